// The step of the Lucas-Lehmer test that follows the square (dkss_ll_step).
//
// The thesis checks its DKSS implementation as a whole by testing Mersenne
// numbers M_p = 2^p - 1 for primality (implementation chapter, system test):
// s_0 = 4, s_(k+1) = s_k^2 - 2 mod M_p, and for an odd prime p, M_p is prime
// exactly when s_(p-2) = 0.  A single wrong bit in any square spreads to every
// later residue, so the residues check every code path of the multiplication.
// The square is dkss_sqr; this file reduces it modulo M_p and subtracts 2.
// Because 2^p = 1 mod M_p, c mod M_p is (c mod 2^p) + (c >> p), folded once
// more; the serial word loop is short beside the square and runs on one
// thread.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/dkss.h"
#include "mersenne.cuh"

namespace {

__global__ void k_ll_step(const uint64_t* __restrict__ c, uint64_t* __restrict__ s, uint32_t p, uint32_t w) {
    dkss::ll_fold(c, s, p, w);
}

}  // namespace

extern "C" dkss_status dkss_ll_step(const uint64_t* c, uint64_t* s, uint32_t p, dkss_stream_t stream) {
    if (!c || !s || p <= 2 || p >= (1u << 26)) return DKSS_EINVAL;
    const uint32_t w = (p + 63) / 64;
    const uintptr_t c0 = (uintptr_t)c, c1 = c0 + 16ull * w, s0 = (uintptr_t)s, s1 = s0 + 8ull * w;
    if (s0 < c1 && c0 < s1) return DKSS_EINVAL;
    k_ll_step<<<1, 1, 0, (cudaStream_t)stream>>>(c, s, p, w);
    return cudaGetLastError() == cudaSuccess ? DKSS_OK : DKSS_ECUDA;
}
