// Cost model of the autotuner: a small multilayer perceptron that predicts
// log2 of a product's device time from its parameters (the only floating point
// in the library; it never touches the arithmetic of a product).
//
// Network: x (F = 12 features) -> h1 = relu(W1 x + b1) (H = 32)
//          -> h2 = relu(W2 h1 + b2) (H) -> y = w3 . h2 + b3.
// Parameters are one float array: W1 [H][F], b1 [H], W2 [H][H], b2 [H],
// w3 [H], b3 [1].  Loss over a batch: mean (y - t)^2.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/dkss.h"

namespace {

constexpr int F = DKSS_MLP_FEATURES;
constexpr int H = DKSS_MLP_HIDDEN;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * F, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == DKSS_MLP_PARAMS, "parameter count");
constexpr int kT = 256;

struct Acts {
    float h1[H], h2[H], y;
};

__device__ void forward_one(const float* p, const float* x, Acts& a) {
    for (int j = 0; j < H; ++j) {
        float s = p[OFF_B1 + j];
        for (int i = 0; i < F; ++i) s += p[OFF_W1 + j * F + i] * x[i];
        a.h1[j] = s > 0.f ? s : 0.f;
    }
    for (int j = 0; j < H; ++j) {
        float s = p[OFF_B2 + j];
        for (int i = 0; i < H; ++i) s += p[OFF_W2 + j * H + i] * a.h1[i];
        a.h2[j] = s > 0.f ? s : 0.f;
    }
    float s = p[OFF_B3];
    for (int i = 0; i < H; ++i) s += p[OFF_W3 + i] * a.h2[i];
    a.y = s;
}

__global__ void __launch_bounds__(kT) k_mlp_forward(const float* __restrict__ params, const float* __restrict__ x,
                                                    uint32_t B, float* __restrict__ y) {
    __shared__ float p[NPARAM];
    for (int i = threadIdx.x; i < NPARAM; i += kT) p[i] = params[i];
    __syncthreads();
    const uint32_t n = blockIdx.x * kT + threadIdx.x;
    if (n >= B) return;
    Acts a;
    forward_one(p, x + (size_t)n * F, a);
    y[n] = a.y;
}

// Gradient of mean (y - t)^2: each CTA sums its samples' contributions in
// shared memory, then adds them to grad (zeroed by the caller) and loss.
__global__ void __launch_bounds__(kT) k_mlp_grad(const float* __restrict__ params, const float* __restrict__ x,
                                                 const float* __restrict__ t, uint32_t B, float* __restrict__ grad,
                                                 float* __restrict__ loss) {
    __shared__ float p[NPARAM];
    __shared__ float g[NPARAM];
    __shared__ float lsum;
    for (int i = threadIdx.x; i < NPARAM; i += kT) {
        p[i] = params[i];
        g[i] = 0.f;
    }
    if (threadIdx.x == 0) lsum = 0.f;
    __syncthreads();
    const uint32_t n = blockIdx.x * kT + threadIdx.x;
    if (n < B) {
        const float* xn = x + (size_t)n * F;
        Acts a;
        forward_one(p, xn, a);
        const float err = a.y - t[n];
        atomicAdd(&lsum, err * err / (float)B);
        const float dy = 2.f * err / (float)B;
        atomicAdd(&g[OFF_B3], dy);
        float dh2[H];
        for (int j = 0; j < H; ++j) {
            atomicAdd(&g[OFF_W3 + j], dy * a.h2[j]);
            dh2[j] = a.h2[j] > 0.f ? dy * p[OFF_W3 + j] : 0.f;
        }
        float dh1[H];
        for (int i = 0; i < H; ++i) dh1[i] = 0.f;
        for (int j = 0; j < H; ++j) {
            if (dh2[j] == 0.f) continue;
            atomicAdd(&g[OFF_B2 + j], dh2[j]);
            for (int i = 0; i < H; ++i) {
                atomicAdd(&g[OFF_W2 + j * H + i], dh2[j] * a.h1[i]);
                dh1[i] += dh2[j] * p[OFF_W2 + j * H + i];
            }
        }
        for (int j = 0; j < H; ++j) {
            const float d = a.h1[j] > 0.f ? dh1[j] : 0.f;
            if (d == 0.f) continue;
            atomicAdd(&g[OFF_B1 + j], d);
            for (int i = 0; i < F; ++i) atomicAdd(&g[OFF_W1 + j * F + i], d * xn[i]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NPARAM; i += kT)
        if (g[i] != 0.f) atomicAdd(&grad[i], g[i]);
    if (threadIdx.x == 0) atomicAdd(loss, lsum);
}

// One Adam step (Kingma & Ba 2015) on every parameter.
__global__ void k_mlp_adam(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m1,
                           float* __restrict__ m2, uint32_t n, float lr, float beta1, float beta2, float eps,
                           float corr1, float corr2) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = grad[i];
    m1[i] = beta1 * m1[i] + (1.f - beta1) * gi;
    m2[i] = beta2 * m2[i] + (1.f - beta2) * gi * gi;
    const float mh = m1[i] / corr1, vh = m2[i] / corr2;
    params[i] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace

extern "C" {

dkss_status dkss_mlp_forward(const float* params, const float* x, size_t B, float* y, dkss_stream_t stream) {
    if (!params || !x || !y || B == 0 || B > (1u << 30)) return DKSS_EINVAL;
    k_mlp_forward<<<(unsigned)((B + kT - 1) / kT), kT, 0, (cudaStream_t)stream>>>(params, x, (uint32_t)B, y);
    return cudaGetLastError() == cudaSuccess ? DKSS_OK : DKSS_ECUDA;
}

dkss_status dkss_mlp_grad(const float* params, const float* x, const float* t, size_t B, float* grad, float* loss,
                          dkss_stream_t stream) {
    if (!params || !x || !t || !grad || !loss || B == 0 || B > (1u << 30)) return DKSS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, st) != cudaSuccess ||
        cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess)
        return DKSS_ECUDA;
    k_mlp_grad<<<(unsigned)((B + kT - 1) / kT), kT, 0, st>>>(params, x, t, (uint32_t)B, grad, loss);
    return cudaGetLastError() == cudaSuccess ? DKSS_OK : DKSS_ECUDA;
}

dkss_status dkss_mlp_adam(float* params, const float* grad, float* m1, float* m2, float lr, uint32_t step,
                          dkss_stream_t stream) {
    if (!params || !grad || !m1 || !m2 || step == 0) return DKSS_EINVAL;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = std::pow(b1, (float)step), c2 = std::pow(b2, (float)step);
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m1, m2, NPARAM, lr, b1, b2, eps,
                                                                        1.f - c1, 1.f - c2);
    return cudaGetLastError() == cudaSuccess ? DKSS_OK : DKSS_ECUDA;
}

}  // extern "C"
