// Reduction step of the Lucas-Lehmer test (dkss_ll_step, mersenne.cu): plain
// integer code, callable on the device and, for the CPU tests, on the host.
//
// s = (c - 2) mod (2^p - 1) for c < 2^(2p).  Because 2^p = 1 mod 2^p - 1,
// c mod (2^p - 1) is (c mod 2^p) + (c >> p), folded once more; 2^p - 1 itself
// maps to 0, then 2 is subtracted modulo 2^p - 1.
#pragma once
#include <cstdint>

namespace dkss {

// bits [pos, pos + 64) of the little-endian number x of n words (zero past its end)
__host__ __device__ inline uint64_t ll_bits_at(const uint64_t* x, uint64_t n, uint64_t pos) {
    const uint64_t q = pos >> 6;
    const uint32_t r = (uint32_t)(pos & 63);
    const uint64_t lo = q < n ? x[q] : 0ull;
    if (r == 0) return lo;
    const uint64_t hi = q + 1 < n ? x[q + 1] : 0ull;
    return (lo >> r) | (hi << (64 - r));
}

// c: 2w words, s: w words (w = ceil(p/64)), not overlapping
__host__ __device__ inline void ll_fold(const uint64_t* c, uint64_t* s, uint32_t p, uint32_t w) {
    const uint32_t top = p - 64 * (w - 1);                       // bits in the top word, 1..64
    const uint64_t top_mask = top == 64 ? ~0ull : (1ull << top) - 1;
    // t = (c mod 2^p) + (c >> p), below 2^(p+1)
    uint64_t carry = 0;
    for (uint32_t i = 0; i < w; ++i) {
        const uint64_t lo = i + 1 == w ? (c[i] & top_mask) : c[i];
        const uint64_t hi = ll_bits_at(c, 2ull * w, (uint64_t)p + 64ull * i);
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

}  // namespace dkss
