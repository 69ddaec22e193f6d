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

namespace {

// bits [pos, pos + 64) of the little-endian number x of n words (zero past its end)
__device__ __forceinline__ uint64_t bits_at(const uint64_t* x, uint64_t n, uint64_t pos) {
    const uint64_t q = pos >> 6;
    const uint32_t r = (uint32_t)(pos & 63);
    const uint64_t lo = q < n ? x[q] : 0ull;
    if (r == 0) return lo;
    const uint64_t hi = q + 1 < n ? x[q + 1] : 0ull;
    return (lo >> r) | (hi << (64 - r));
}

// s = (c - 2) mod (2^p - 1) for c < 2^(2p) of 2w words; s has w words
__global__ void k_ll_step(const uint64_t* __restrict__ c, uint64_t* __restrict__ s, uint32_t p, uint32_t w) {
    const uint32_t top = p - 64 * (w - 1);                       // bits in the top word, 1..64
    const uint64_t top_mask = top == 64 ? ~0ull : (1ull << top) - 1;
    // t = (c mod 2^p) + (c >> p), below 2^(p+1)
    uint64_t carry = 0;
    for (uint32_t i = 0; i < w; ++i) {
        const uint64_t lo = i + 1 == w ? (c[i] & top_mask) : c[i];
        const uint64_t hi = bits_at(c, 2ull * w, (uint64_t)p + 64ull * i);
        uint64_t t = lo + hi;
        uint64_t cout = t < lo ? 1ull : 0ull;
        t += carry;
        cout += t < carry ? 1ull : 0ull;
        s[i] = t;
        carry = cout;
    }
    // fold bit p back: t mod 2^p + (t >> p) <= 2^p - 1
    uint64_t e;
    if (top == 64) {
        e = carry;
    } else {
        e = s[w - 1] >> top;
        s[w - 1] &= top_mask;
    }
    for (uint32_t i = 0; i < w && e != 0; ++i) {
        s[i] += e;
        e = s[i] == 0 ? 1ull : 0ull;
    }
    // 2^p - 1 is 0 mod M_p
    bool all_ones = true;
    for (uint32_t i = 0; i < w; ++i)
        if (s[i] != (i + 1 == w ? top_mask : ~0ull)) all_ones = false;
    if (all_ones)
        for (uint32_t i = 0; i < w; ++i) s[i] = 0;
    // minus 2 mod M_p
    bool ge2 = s[0] >= 2;
    for (uint32_t i = 1; i < w; ++i)
        if (s[i] != 0) ge2 = true;
    if (ge2) {
        uint64_t borrow = 2;
        for (uint32_t i = 0; i < w && borrow != 0; ++i) {
            const uint64_t v = s[i];
            s[i] = v - borrow;
            borrow = v < borrow ? 1ull : 0ull;
        }
    } else {
        // s in {0, 1}: s + M_p - 2 = 2^p - 3 + s
        const uint64_t v = s[0];
        for (uint32_t i = 0; i < w; ++i) s[i] = i + 1 == w ? top_mask : ~0ull;
        s[0] -= 2 - v;
    }
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
