// Reduced-radix products for the R-multiplications.
//
// The negacyclic convolution c_k = sum_i x_i y_{k-i} (thesis eq. ncycconv)
// sums m products of residues mod p^z.  Here each factor is split into LR
// limbs of 26 bits and every limb product (< 2^52) is added into a 64-bit
// column accumulator with one 32x32->64 multiply-add: no carry is handled in
// the loop, because a column receives at most m*LR products plus the
// reduction's, which stays below 2^64 for m*LR < 4096.  One Montgomery
// reduction with R' = 2^(26*LR) per output follows; the host guarantees
// m*p^z < R', so its result is below 2 p^z and one subtraction makes it
// canonical.
#pragma once
#include <cstdint>

namespace dkss {

constexpr uint32_t kM26 = (1u << 26) - 1;

// the limb arithmetic below is plain integer code: also callable on the host,
// where the CPU tests check it against exact integers
#define DKSS_HD __host__ __device__ __forceinline__
#define DKSS_HD_DECL __host__ __device__ inline

template <int LR>
struct ModRR {
    uint32_t q[LR];     // p^z in 26-bit limbs
    uint32_t nprime;    // -(p^z)^-1 mod 2^26
    uint64_t qtop_inv;  // floor((2^64 - 1) / Q), Q = q[LR-1] 2^26 + q[LR-2]: quotient estimates
};

// The reciprocal of ModRR::qtop_inv (host and device).
DKSS_HD_DECL uint64_t qtop_reciprocal(uint32_t q_hi, uint32_t q_lo) {
    return ~0ull / (((uint64_t)q_hi << 26) + q_lo);
}

// 32-bit limbs -> 26-bit limbs (x < 2^(26 LR))
template <int L, int LR>
DKSS_HD void to_rr(uint32_t (&out)[LR], const uint32_t (&x)[L]) {
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const int bit = 26 * i, w = bit >> 5, s = bit & 31;
        uint32_t v = w < L ? (x[w] >> s) : 0u;
        if (s > 6 && w + 1 < L) v |= x[w + 1] << (32 - s);
        out[i] = v & kM26;
    }
}

// 26-bit limbs -> 32-bit limbs (value < 2^(32 L))
template <int L, int LR>
DKSS_HD void from_rr(uint32_t (&out)[L], const uint32_t (&r)[LR]) {
#pragma unroll
    for (int w = 0; w < L; ++w) out[w] = 0;
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const int bit = 26 * i, w = bit >> 5, s = bit & 31;
        if (w < L) out[w] |= r[i] << s;
        if (s > 6 && w + 1 < L) out[w + 1] |= r[i] >> (32 - s);
    }
}

// r = (q - y) mod q in 26-bit limbs
template <int LR>
DKSS_HD void neg_rr(uint32_t (&r)[LR], const uint32_t (&y)[LR], const ModRR<LR>& md) {
    uint32_t nz = 0, borrow = 0;
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        nz |= y[i];
        uint32_t d = md.q[i] - y[i] - borrow;
        borrow = d >> 31;
        r[i] = d & kM26;
    }
#pragma unroll
    for (int i = 0; i < LR; ++i) r[i] = nz ? r[i] : 0u;
}

// col[a+b] += x_a * y_b
template <int LR>
DKSS_HD void mac_cols(uint64_t (&col)[2 * LR], const uint32_t (&x)[LR], const uint32_t (&y)[LR]) {
#pragma unroll
    for (int a = 0; a < LR; ++a)
#pragma unroll
        for (int b = 0; b < LR; ++b) col[a + b] += (uint64_t)x[a] * y[b];
}

// Montgomery reduction of the column sum T = sum_t col[t] 2^(26t):
// r = T * 2^(-26 LR) mod q, canonical, for T < q * 2^(26 LR).
template <int LR>
DKSS_HD void redc_cols(uint32_t (&r)[LR], uint64_t (&col)[2 * LR], const ModRR<LR>& md) {
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const uint32_t d = (uint32_t)col[i] & kM26;
        const uint32_t qi = (d * md.nprime) & kM26;
        const uint64_t c = col[i] + (uint64_t)qi * md.q[0];   // low 26 bits become 0
        col[i + 1] += c >> 26;
#pragma unroll
        for (int k = 1; k < LR; ++k) col[i + k] += (uint64_t)qi * md.q[k];
    }
    // normalise the upper half into 26-bit limbs; the value is below 2q
    uint64_t carry = 0;
    uint32_t t[LR + 1];
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const uint64_t v = col[LR + i] + carry;
        t[i] = (uint32_t)v & kM26;
        carry = v >> 26;
    }
    t[LR] = (uint32_t)carry;
    // subtract q once if t >= q
    uint32_t d[LR], borrow = 0;
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const uint32_t v = t[i] - md.q[i] - borrow;
        borrow = v >> 31;
        d[i] = v & kM26;
    }
    const bool ge = t[LR] || !borrow;
#pragma unroll
    for (int i = 0; i < LR; ++i) r[i] = ge ? d[i] : t[i];
}

// r = a * b * 2^(-26 LR) mod q
template <int LR>
DKSS_HD void mont_mul_rr(uint32_t (&r)[LR], const uint32_t (&a)[LR], const uint32_t (&b)[LR],
                                            const ModRR<LR>& md) {
    uint64_t col[2 * LR];
#pragma unroll
    for (int i = 0; i < 2 * LR; ++i) col[i] = 0;
    mac_cols<LR>(col, a, b);
    redc_cols<LR>(r, col, md);
}

// shared-memory residues in 26-bit limbs: LR consecutive words
template <int LR>
__device__ __forceinline__ void ld_rr(uint32_t (&x)[LR], const uint32_t* p) {
    if constexpr (LR == 4) {
        uint4 v = *reinterpret_cast<const uint4*>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else if constexpr (LR == 2) {
        uint2 v = *reinterpret_cast<const uint2*>(p);
        x[0] = v.x; x[1] = v.y;
    } else {
#pragma unroll
        for (int i = 0; i < LR; ++i) x[i] = p[i];
    }
}

template <int LR>
__device__ __forceinline__ void st_rr(uint32_t* p, const uint32_t (&x)[LR]) {
    if constexpr (LR == 4) {
        *reinterpret_cast<uint4*>(p) = make_uint4(x[0], x[1], x[2], x[3]);
    } else if constexpr (LR == 2) {
        *reinterpret_cast<uint2*>(p) = make_uint2(x[0], x[1]);
    } else {
#pragma unroll
        for (int i = 0; i < LR; ++i) p[i] = x[i];
    }
}

}  // namespace dkss
