// Stage-boundary range checks (DKSS_DEBUG_CHECKS).
//
// Between kernels every residue of a transformed polynomial is canonical, in
// [0, p^z) (Section 3.2: the coefficients of R live in Z/p^zZ); after the
// backwards transform and the division by 2M they are the exact coefficients
// of the product polynomial, also below p^z (the bound of Section 3.2.2).
// With DKSS_DEBUG_CHECKS a plan runs this kernel over each polynomial at the
// stage boundaries; a residue at or above p^z sets kStatusRange in the plan's
// status word (read by dkss_sync_status as DKSS_EDEVICE) and the product
// continues, so a check never stops or faults the GPU.
#pragma once
#include <cstdint>

#include "status_bits.hpp"

namespace dkss {

struct RangeParams {
    const uint32_t* poly;   // residues of L 32-bit limbs, residue-major
    uint64_t n_res;         // residues to check
    uint32_t q[4];          // p^z, L limbs (limbs >= L zero)
    uint32_t* status;
    uint32_t digit_p;       // nonzero: the residues are p-adic digits, each must be below p
};

// x >= q for L-limb little-endian values
template <int L>
__device__ __forceinline__ bool ge_q(const uint32_t (&x)[L], const uint32_t* q) {
#pragma unroll
    for (int i = L - 1; i >= 0; --i) {
        if (x[i] != q[i]) return x[i] > q[i];
    }
    return true;
}

template <int L>
__global__ void __launch_bounds__(256) k_check_range(RangeParams prm) {
    uint32_t q[L];
#pragma unroll
    for (int i = 0; i < L; ++i) q[i] = prm.q[i];
    bool bad = false;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < prm.n_res; r += stride) {
        uint32_t x[L];
        const uint32_t* p = prm.poly + r * L;
        if constexpr (L == 4) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
            x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
        } else if constexpr (L == 2) {
            const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
            x[0] = v.x; x[1] = v.y;
        } else {
#pragma unroll
            for (int i = 0; i < L; ++i) x[i] = __ldg(p + i);
        }
        if (prm.digit_p) {
#pragma unroll
            for (int i = 0; i < L; ++i) bad |= x[i] >= prm.digit_p;
        } else {
            bad |= ge_q<L>(x, q);
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(prm.status, kStatusRange);
}

}  // namespace dkss
