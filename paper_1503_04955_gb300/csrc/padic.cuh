// Residues mod p^z as z base-p digits (p-adic digits) for the transform in R.
//
// x = sum_{k<z} x_k p^k.  Reducing mod p^z is dropping the digits from z on,
// so a product mod p^z needs only the z(z+1)/2 digit products of the
// truncated columns c_k = sum_{i+j=k} a_i b_j (k < z), then one carry chain
// that writes each column as q_k p + d_k and adds q_k to the next; the top
// column keeps d only.  Each quotient q_k is a Barrett estimate with a
// precomputed reciprocal of p: mu = floor(2^(64+s) / p), s = floor(log2 p),
// q = floor(c mu / 2^(64+s)) is floor(c / p) or one less, so d = c - q p is in
// [0, 2p) and one conditional subtraction makes it canonical.  For z = 4 and
// p < 2^30 that is 10 limb products and 4 carries per product, against
// 5 x 5 limb products and 5 x 6 reduction products for a 26-bit-limb
// Montgomery product of the same 120-bit modulus.
//
// Digits are lazy between products: additions are digitwise (a digit may
// exceed p), a difference x - y is x + D - y with D = K (p, p-1, ..., p-1),
// whose value K p^z is 0 mod p^z and whose digits are at least y's, and
// pd_norm brings digits back near p with one multiply-high per digit.  The
// plan's host check (ntt_bounds.cpp, pd_lazy_bounds) follows the largest
// digit and every column through the schedule below and only then selects
// this form.  Plain integer code: also callable on the host, where the CPU
// tests check it against exact integers.
#pragma once
#include <cstdint>

#include "ntt_rmul.cuh"

namespace dkss {

constexpr int kPdDigits = 4;   // z of the rings that take this form

// F (fast carries): floor(2^32 / p) is a power of two, 2^e; then the
// reciprocal floor(2^64 / p) is 2^e 2^32 + mu_lo and a column's quotient
// takes one wide product and one multiply-high instead of the high half of
// a 64 x 64-bit product (pd_carry).
template <int Z, bool F = false>
struct ModPD {
    uint32_t p;
    uint32_t nmu;     // floor(2^32 / p): quotient estimates of single digits (pd_canon)
    uint32_t nsh;     // ceil(log2 p): quotient estimates of lazy digits (pd_norm)
    uint32_t s;       // floor(log2 p)
    uint64_t mu;      // floor(2^(64 + s) / p): quotient estimates of columns
    uint32_t mu_lo;   // floor(2^64 / p) mod 2^32 (F)
    uint32_t lg_nmu;  // log2 floor(2^32 / p) (F)
};

// The same constants for the fast carries (the fields are those of ModPD<Z, false>).
template <int Z>
DKSS_HD ModPD<Z, true> pd_fast_view(const ModPD<Z, false>& md) {
    ModPD<Z, true> f;
    f.p = md.p;
    f.nmu = md.nmu;
    f.nsh = md.nsh;
    f.s = md.s;
    f.mu = md.mu;
    f.mu_lo = md.mu_lo;
    f.lg_nmu = md.lg_nmu;
    return f;
}

template <class MR>
struct IsPD {
    static constexpr bool value = false;
};
template <int Z, bool F>
struct IsPD<ModPD<Z, F>> {
    static constexpr bool value = true;
};

DKSS_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// A constant of the plan's table: read-only cache on the device.
DKSS_HD uint32_t ld_const(const uint32_t* p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// Carry chain of the columns c_0 .. c_{Z-1} (each below 2^64 with the carry
// it receives): canonical digits of sum_k c_k p^k mod p^Z.
template <int Z, bool F>
DKSS_HD void pd_carry(uint32_t (&r)[Z], uint64_t (&c)[Z], const ModPD<Z, F>& md) {
#pragma unroll
    for (int k = 0; k < Z; ++k) {
        uint64_t q;   // floor(c / p) or one less
        if constexpr (F) {
            // floor(c (2^e 2^32 + mu_lo) / 2^64) from c = c1 2^32 + c0: the
            // integer part of (c1 mu_lo + c0 2^e + hi(c0 mu_lo)) / 2^32 plus
            // c1 2^e (the plan's check keeps the sum below 2^64)
            const uint32_t c0 = (uint32_t)c[k], c1 = (uint32_t)(c[k] >> 32);
            const uint64_t t = (uint64_t)c1 * md.mu_lo + ((uint64_t)c0 << md.lg_nmu) + mulhi32(c0, md.mu_lo);
            q = ((uint64_t)c1 << md.lg_nmu) + (t >> 32);
        } else {
            q = mulhi64(c[k], md.mu) >> md.s;
        }
        uint32_t d = (uint32_t)c[k] - (uint32_t)q * md.p;
        if (d >= md.p) {
            d -= md.p;
            ++q;
        }
        r[k] = d;
        if (k + 1 < Z) c[k + 1] += q;
    }
}

// r = a b mod p^Z, canonical digits
template <int Z, bool F>
DKSS_HD void mmul(uint32_t (&r)[Z], const uint32_t (&a)[Z], const uint32_t (&b)[Z], const ModPD<Z, F>& md) {
    uint64_t c[Z];
#pragma unroll
    for (int k = 0; k < Z; ++k) c[k] = 0;
#pragma unroll
    for (int i = 0; i < Z; ++i)
#pragma unroll
        for (int j = 0; i + j < Z; ++j) c[i + j] += (uint64_t)a[i] * b[j];
    pd_carry<Z>(r, c, md);
}

// Lazy normalisation: digit v = x_k + carry becomes v - k p with
// k = floor(v / 2^ceil(log2 p)) <= v / p (a shift), so below
// v (1 - p / 2^ceil(log2 p)) + p; k moves to the next digit, the top digit's
// is dropped (a multiple of p^Z).  Every x_k + carry must stay below 2^32.
template <int Z, bool F>
DKSS_HD void pd_norm(uint32_t (&x)[Z], const ModPD<Z, F>& md) {
    uint32_t cin = 0;
#pragma unroll
    for (int k = 0; k < Z; ++k) {
        const uint32_t v = x[k] + cin;
        const uint32_t kq = v >> md.nsh;
        x[k] = v - kq * md.p;
        cin = kq;
    }
}

// Canonical digits (each below p) of a lazy value, same limits as pd_norm.
template <int Z, bool F>
DKSS_HD void pd_canon(uint32_t (&r)[Z], const uint32_t (&x)[Z], const ModPD<Z, F>& md) {
    uint32_t cin = 0;
#pragma unroll
    for (int k = 0; k < Z; ++k) {
        const uint32_t v = x[k] + cin;
        uint32_t kq = mulhi32(v, md.nmu);
        uint32_t d = v - kq * md.p;   // below 2p
        if (d >= md.p) {
            d -= md.p;
            ++kq;
        }
        r[k] = d;
        cin = kq;
    }
}

// Digits of a residue held as L 32-bit words w (any value below 2^(32L)):
// w = sum_j w_j 2^(32j) = sum_j w_j P_j (mod p^Z) with P_j the canonical
// digits of 2^(32j) mod p^Z (pw[j * Z + k], from the plan), then one carry
// chain.  Columns stay below L 2^32 p + carry < 2^64 for L <= 4, p < 2^30.
template <int L, int Z, bool F>
DKSS_HD void pd_from_words(uint32_t (&r)[Z], const uint32_t (&w)[L], const uint32_t* pw, const ModPD<Z, F>& md) {
    uint64_t c[Z];
#pragma unroll
    for (int k = 0; k < Z; ++k) c[k] = k == 0 ? w[0] : 0;
#pragma unroll
    for (int j = 1; j < L; ++j)
#pragma unroll
        for (int k = 0; k < Z; ++k) c[k] += (uint64_t)w[j] * ld_const(pw + j * Z + k);
    pd_carry<Z>(r, c, md);
}

// pd_from_words for 4 words and 4 digits where p > 2^22: 2^32 < p^2 and
// 2^64 < p^3, so the digits of 2^32 are zero from the third on and those of
// 2^64 from the fourth on; their products are left out (9 instead of 12).
template <bool F>
DKSS_HD void pd_from_words4_large_p(uint32_t (&r)[4], const uint32_t (&w)[4], const uint32_t* pw,
                                    const ModPD<4, F>& md) {
    uint64_t c[4] = {w[0], 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 2; ++k) c[k] += (uint64_t)w[1] * ld_const(pw + 4 + k);
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] += (uint64_t)w[2] * ld_const(pw + 8 + k);
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] += (uint64_t)w[3] * ld_const(pw + 12 + k);
    pd_carry<4>(r, c, md);
}

// 32-bit words of a residue from its canonical digits (Horner's rule from
// the top digit): the canonical value below p^Z < 2^(32L).
template <int L, int Z, bool F>
DKSS_HD void pd_to_words(uint32_t (&w)[L], const uint32_t (&d)[Z], const ModPD<Z, F>& md) {
#pragma unroll
    for (int j = 0; j < L; ++j) w[j] = j == 0 ? d[Z - 1] : 0u;
#pragma unroll
    for (int k = Z - 2; k >= 0; --k) {
        // the value so far is below p^(Z-1-k) < 2^(30 (Z-1-k)): only its low words are non-zero
        constexpr int kMaxW = L;
        const int nw = (30 * (Z - k) + 31) / 32 < kMaxW ? (30 * (Z - k) + 31) / 32 : kMaxW;
        uint64_t carry = d[k];
#pragma unroll
        for (int j = 0; j < L; ++j) {
            if (j < nw) {
                const uint64_t t = (uint64_t)w[j] * md.p + carry;
                w[j] = (uint32_t)t;
                carry = t >> 32;
            }
        }
    }
}

// Constants of the transform in p-adic digits: NttLayout<m>'s entries (plain
// residues, no Montgomery factor; the biases are digit vectors
// K (p, p-1, ..., p-1)), then the digits of 2^(32j) mod p^Z, j < 4.
template <int m>
struct PdLayout {
    static constexpr int POW32 = NttLayout<m>::COUNT;
    static constexpr int COUNT = POW32 + 4;
};

// Forward negacyclic transform (as ntt_forward): digits grow by at most p
// per stage (t is canonical, the bias digits are at most p), and both
// outputs are normalised after every second stage and after the last.
template <int m, int Z, bool F>
__device__ __forceinline__ void ntt_forward_pd(uint32_t (&v)[4][Z], uint32_t* buf, int lane, unsigned mask,
                                               const uint32_t* cst, const ModPD<Z, F>& md) {
    using NL = NttLayout<m>;
    constexpr int LG = NL::LG;
    uint32_t bf[Z];
    ldg_rr<Z>(bf, cst + NL::BF * Z);
    int h = LG - 1;
#pragma unroll
    for (int b = LG - 1; b >= 0; --b) {
        if ((LG - 1 - b) % 2 == 0 && b != LG - 1) {
            const int hn = b >= 1 ? b : 1;
            ntt_exchange<m, Z>(v, buf, lane, h, hn, mask);
            h = hn;
        }
        const int sbit = b == h ? 2 : 1;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int jl = sbit == 2 ? p : 2 * p, jh = jl + sbit;
            const int k = (1 << (LG - 1 - b)) + (lidx(lane, jl, h) >> (b + 1));
            uint32_t z[Z], t[Z];
            ldg_rr<Z>(z, cst + (NL::ZF + k) * Z);
            mmul<Z>(t, v[jh], z, md);
            lz_sub<Z>(v[jh], v[jl], bf, t);
            lz_add<Z>(v[jl], v[jl], t);
        }
        if ((LG - 1 - b) % 2 == 1 || b == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) pd_norm<Z>(v[j], md);
        }
    }
}

// Backwards transform scaled by a constant (as ntt_backward): the products
// are canonical, the sums are normalised after every stage but the last; a
// difference takes the stage's bias.  The last stage multiplies by cst[lo_c]
// and cst[hi_c] (plain residues), or with RAW_LO leaves slots 0 and 1 as the
// sums (the caller makes them canonical with pd_canon).
template <int m, int Z, bool RAW_LO = false, bool F = false>
__device__ __forceinline__ void ntt_backward_pd(uint32_t (&v)[4][Z], uint32_t* buf, int lane, unsigned mask,
                                                const uint32_t* cst, int lo_c, int hi_c, const ModPD<Z, F>& md) {
    using NL = NttLayout<m>;
    constexpr int LG = NL::LG;
    int h = 1;
#pragma unroll
    for (int b = 0; b < LG; ++b) {
        if (b % 2 == 0 && b != 0) {
            const int hn = b + 1 <= LG - 1 ? b + 1 : LG - 1;
            ntt_exchange<m, Z>(v, buf, lane, h, hn, mask);
            h = hn;
        }
        uint32_t bias[Z];
        ldg_rr<Z>(bias, cst + (NL::BB + b) * Z);
        const int sbit = b == h ? 2 : 1;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int jl = sbit == 2 ? p : 2 * p, jh = jl + sbit;
            uint32_t s[Z], d[Z], z[Z];
            lz_add<Z>(s, v[jl], v[jh]);
            lz_sub<Z>(d, v[jl], bias, v[jh]);
            if (b == LG - 1) {
                ldg_rr<Z>(z, cst + hi_c * Z);
                if constexpr (RAW_LO) {
#pragma unroll
                    for (int w = 0; w < Z; ++w) v[jl][w] = s[w];
                } else {
                    uint32_t c[Z];
                    ldg_rr<Z>(c, cst + lo_c * Z);
                    mmul<Z>(v[jl], s, c, md);
                }
                mmul<Z>(v[jh], d, z, md);
            } else {
                const int k = (1 << (LG - 1 - b)) + (lidx(lane, jl, h) >> (b + 1));
                ldg_rr<Z>(z, cst + (NL::ZI + k) * Z);
                pd_norm<Z>(s, md);
#pragma unroll
                for (int w = 0; w < Z; ++w) v[jl][w] = s[w];
                mmul<Z>(v[jh], d, z, md);
            }
        }
    }
}

}  // namespace dkss
