// Decoding and carry propagation without any allocation (dkss_decode_static).
//
// Callers that must not allocate device memory at the time of the call can
// still turn a product polynomial into the product's words: a latency-bound
// loop whose device memory is fixed before it starts (cudaMalloc and cudaFree
// may synchronize the device and stall its other streams), or code running
// inside a framework that owns the device's memory pool and gives its plugins
// no allocator.  The carry scan's scratch (one word per tile of 2048 output windows
// plus one status word) lives in a file-scope device array instead of
// caller- or plan-owned memory.  Every GPU that loads the library holds this
// array (1 MiB) until the process exits.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "../../include/dkss.h"
#include "decode.cuh"

namespace {

constexpr uint64_t kStaticTiles = DKSS_DECODE_STATIC_MAX_TILES;
constexpr uint64_t kMaxDevices = 64;

// tile aggregates (kStaticTiles words) followed by one status word
static __device__ __align__(256) uint32_t g_decode_scratch[kStaticTiles + 1];

// Device address of g_decode_scratch per device, looked up once per device
// with that device current (a host-side reference to the symbol is not a
// device address and must never reach a kernel).  Atomic: two host threads
// may make their first calls on a device at once (both store the same value).
std::atomic<uint32_t*> g_scratch_ptr[kMaxDevices] = {};

template <int L>
void launch(const dkss::DecodeParams& dp, uint32_t u, cudaStream_t st) {
    // the u = 32 and u = 16 kernels read residues with L-word vector loads
    const bool vec_ok = (uintptr_t)dp.c % (L == 3 ? 4u : 4u * L) == 0;
    if (u == 32 && vec_ok) dkss::k_decode_tiles_aligned<L, 1><<<(unsigned)dp.n_tiles, dkss::kDecThreads, 0, st>>>(dp);
    else if (u == 16 && vec_ok) dkss::k_decode_tiles_aligned<L, 2><<<(unsigned)dp.n_tiles, dkss::kDecThreads, 0, st>>>(dp);
    else dkss::k_decode_tiles<L><<<(unsigned)dp.n_tiles, dkss::kDecThreads, 0, st>>>(dp);
}

}  // namespace

extern "C" dkss_status dkss_decode_static(const uint32_t* c, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u,
                                          uint32_t L, uint64_t* out, dkss_stream_t stream) {
    if (!c || !out || n_bits == 0 || M == 0 || (M & (M - 1)) || m < 2 || (m & (m - 1)) || m > 64 || u == 0 ||
        u > 32 || L < 2 || L > 4 || (uint64_t)M * (m / 2) * u < n_bits)
        return DKSS_EINVAL;
    const uint64_t nw = (n_bits + 63) / 64;
    const uint64_t n_windows = 4 * nw;
    const uint64_t n_tiles = (n_windows + dkss::kDecTile - 1) / dkss::kDecTile;
    if (n_tiles > kStaticTiles) return DKSS_EUNSUPPORTED;   // product longer than the static scratch covers
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || (uint64_t)dev >= kMaxDevices) return DKSS_ECUDA;
    uint32_t* scratch = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!scratch) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_decode_scratch) != cudaSuccess || !p) return DKSS_ECUDA;
        scratch = static_cast<uint32_t*>(p);
        g_scratch_ptr[dev].store(scratch, std::memory_order_release);
    }
    cudaStream_t st = (cudaStream_t)stream;
    // tile aggregates are written before they are read; only the status word must start at zero
    if (cudaMemsetAsync(scratch + kStaticTiles, 0, sizeof(uint32_t), st) != cudaSuccess) return DKSS_ECUDA;
    dkss::DecodeParams dp{};
    dp.c = c;
    dp.out = reinterpret_cast<uint32_t*>(out);
    dp.agg = scratch;
    dp.status = scratch + kStaticTiles;
    dp.P2 = 2 * M;
    dp.n_windows = n_windows;
    dp.n_tiles = n_tiles;
    dp.k_max = 2 * M * (m / 2) + m / 2;
    dp.m = m;
    dp.h = m / 2;
    dp.u = u;
    dp.db = 32 * L + 1;
    dp.out_aligned16 = ((uintptr_t)out & 15) == 0;
    if (L == 2) launch<2>(dp, u, st);
    else if (L == 3) launch<3>(dp, u, st);
    else launch<4>(dp, u, st);
    if (cudaGetLastError() != cudaSuccess) return DKSS_ECUDA;
    dkss::k_decode_scan<<<1, dkss::kScanThreads, 0, st>>>(dp);
    if (cudaGetLastError() != cudaSuccess) return DKSS_ECUDA;
    dkss::k_decode_fix<<<(unsigned)((n_tiles + 255) / 256), 256, 0, st>>>(dp);
    if (cudaGetLastError() != cudaSuccess) return DKSS_ECUDA;
    return DKSS_OK;
}
