// R-multiplication through the evaluation map of R.
//
// alpha^m + 1 splits over P = Z/p^zZ: its roots are gamma^(2j+1), j < m, with
// gamma = omega^(2M/2m) a principal 2m-th root of unity (thesis Section 3.2.3,
// the same fact that yields rho by Lagrange interpolation).  So
// x -> (x(gamma^(2j+1)))_j is a ring isomorphism R -> P^m and a product in R
// is: evaluate both factors (a negacyclic number-theoretic transform of
// length m), multiply pointwise, interpolate (the inverse transform, scaled by
// m^-1).  A bad twiddle rho^s has the evaluations rho^s(gamma^(2j+1)) =
// omega^(s(2j+1)) (rho(gamma^(2j+1)) = omega^(2j+1) by construction), so the
// plan tabulates them directly; alpha^r is applied before the transform as a
// negacyclic coefficient shift, as in the direct form.
//
// One team of m/2 lanes owns an element; lane l holds two coefficients.
// Forward stages use Cooley-Tukey butterflies with psi^brv(k) (psi = gamma),
// which leave evaluations in bit-reversed order; backwards stages use
// Gentleman-Sande butterflies with psi^-brv(k) and return natural order.
// Between stages lanes l and l ^ 2^b swap one value with a shuffle.
//
// Arithmetic is lazy: residues are vectors of LR limbs of nominally 26 bits,
// a sum is a limbwise addition (limbs may grow past 26 bits), a difference
// x - y is x + B - y with a bias B = K p^z whose limbs are each at least
// y's, and a Montgomery product (R' = 2^(26 LR)) leaves normalised limbs of a
// value below 2 p^z without a final subtraction.  The plan's host check
// (ntt_bounds.cpp) follows the worst case of every limb through both
// transforms and picks the biases; only the results written back are made
// canonical.
#pragma once
#include <cstdint>

#include "rr_arith.cuh"

namespace dkss {

// Layout of a plan's transform constants, in residues of LR words.
template <int m>
struct NttLayout {
    static constexpr int LG = (m >= 64) ? 6 : (m >= 32) ? 5 : (m >= 16) ? 4 : (m >= 8) ? 3 : 2;
    static constexpr int ZF = 0;            // psi^brv(k) R', k in [1, m)
    static constexpr int ZI = m;            // psi^-brv(k) R'
    static constexpr int BB = 2 * m;        // backwards stage biases, LG of them
    static constexpr int BF = BB + LG;      // forward butterfly bias
    static constexpr int BN = BF + 1;       // bias of negated input coefficients
    static constexpr int Q = BN + 1;        // p^z (normalised)
    static constexpr int TW_LO = Q + 1;     // m^-1 R'            (last backwards stage, twiddles)
    static constexpr int TW_HI = Q + 2;     // psi^-1 m^-1 R'
    static constexpr int PW_LO = Q + 3;     // m^-1 (2M)^-1 R'^2  (componentwise products of
    static constexpr int PW_HI = Q + 4;     // psi^-1 m^-1 (2M)^-1 R'^2   two normal-form factors)
    static constexpr int ONE = Q + 5;       // R'                 (last backwards stage after a
    static constexpr int ZLAST = Q + 6;     // psi^-1 R'           prescaled componentwise product)
    static constexpr int COUNT = Q + 7;
};

template <int LR>
__device__ __forceinline__ void ldg_rr(uint32_t (&x)[LR], const uint32_t* p) {
#pragma unroll
    for (int i = 0; i < LR; ++i) x[i] = __ldg(p + i);
}

// r = a + b, limbwise
template <int LR>
__device__ __forceinline__ void lz_add(uint32_t (&r)[LR], const uint32_t (&a)[LR], const uint32_t (&b)[LR]) {
#pragma unroll
    for (int i = 0; i < LR; ++i) r[i] = a[i] + b[i];
}

// r = a + B - b, limbwise (B[i] >= b[i] for every i)
template <int LR>
__device__ __forceinline__ void lz_sub(uint32_t (&r)[LR], const uint32_t (&a)[LR], const uint32_t (&B)[LR],
                                       const uint32_t (&b)[LR]) {
#pragma unroll
    for (int i = 0; i < LR; ++i) r[i] = a[i] + B[i] - b[i];
}

// Montgomery product a b 2^(-26 LR) mod q as normalised limbs of a value
// below a b / R' + q (the top limb holds every bit above 26 (LR - 1)).
template <int LR>
__device__ __forceinline__ void mmul(uint32_t (&r)[LR], const uint32_t (&a)[LR], const uint32_t (&b)[LR],
                                     const ModRR<LR>& md) {
    uint64_t col[2 * LR];
#pragma unroll
    for (int i = 0; i < 2 * LR; ++i) col[i] = 0;
    mac_cols<LR>(col, a, b);
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const uint32_t qi = ((uint32_t)col[i] * md.nprime) & kM26;
        const uint64_t c = col[i] + (uint64_t)qi * md.q[0];   // low 26 bits become 0
        col[i + 1] += c >> 26;
#pragma unroll
        for (int k = 1; k < LR; ++k) col[i + k] += (uint64_t)qi * md.q[k];
    }
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const uint64_t v = col[LR + i] + carry;
        r[i] = i + 1 < LR ? ((uint32_t)v & kM26) : (uint32_t)v;
        carry = v >> 26;
    }
}

// canonical residue of normalised limbs of a value below 2q
template <int LR>
__device__ __forceinline__ void canon(uint32_t (&r)[LR], const uint32_t (&x)[LR], const ModRR<LR>& md) {
    uint32_t d[LR], borrow = 0;
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const uint32_t v = x[i] - md.q[i] - borrow;
        borrow = v >> 31;
        d[i] = i + 1 < LR ? (v & kM26) : v;
    }
#pragma unroll
    for (int i = 0; i < LR; ++i) r[i] = borrow ? x[i] : d[i];
}

// carry-propagate limbs (each below 2^32) to 26 bits; the top limb keeps the rest
template <int LR>
__device__ __forceinline__ void lz_norm(uint32_t (&x)[LR]) {
    uint32_t carry = 0;
#pragma unroll
    for (int i = 0; i + 1 < LR; ++i) {
        const uint32_t v = x[i] + carry;
        carry = (v >> 26) + (v < carry ? 64u : 0u);
        x[i] = v & kM26;
    }
    x[LR - 1] += carry;
}

template <int m, int LR>
__device__ __forceinline__ void team_swap(uint32_t (&lo)[LR], uint32_t (&hi)[LR], int lane, int b, unsigned mask) {
    const bool bit = (lane >> b) & 1;
#pragma unroll
    for (int w = 0; w < LR; ++w) {
        const uint32_t send = bit ? lo[w] : hi[w];
        const uint32_t recv = __shfl_xor_sync(mask, send, 1 << b, m / 2);
        if (bit) lo[w] = recv;
        else hi[w] = recv;
    }
}

// Forward negacyclic transform: on entry lane l holds coefficients l, l+m/2;
// on exit the evaluations with bit-reversed indices 2l, 2l+1 (lazy).
template <int m, int LR>
__device__ __forceinline__ void ntt_forward(uint32_t (&lo)[LR], uint32_t (&hi)[LR], int lane, unsigned mask,
                                            const uint32_t* cst, const ModRR<LR>& md) {
    using NL = NttLayout<m>;
    uint32_t bf[LR];
    ldg_rr<LR>(bf, cst + NL::BF * LR);
#pragma unroll
    for (int b = NL::LG - 1; b >= 0; --b) {
        if (b < NL::LG - 1) team_swap<m, LR>(lo, hi, lane, b, mask);
        const int k = (1 << (NL::LG - 1 - b)) + (lane >> b);
        uint32_t z[LR], t[LR];
        ldg_rr<LR>(z, cst + (NL::ZF + k) * LR);
        mmul<LR>(t, hi, z, md);
        lz_sub<LR>(hi, lo, bf, t);        // lo - t
        lz_add<LR>(lo, lo, t);            // lo + t
    }
}

// Backwards transform scaled by a constant: on entry lane l holds the
// evaluations 2l, 2l+1 (bit-reversed order); on exit the coefficients l,
// l+m/2 of the interpolated element times c (normalised, below 2q), where the
// last stage multiplies by cst[lo_c] and cst[hi_c] (= c and psi^-1 c, times R').
template <int m, int LR>
__device__ __forceinline__ void ntt_backward(uint32_t (&lo)[LR], uint32_t (&hi)[LR], int lane, unsigned mask,
                                             const uint32_t* cst, int lo_c, int hi_c, const ModRR<LR>& md) {
    using NL = NttLayout<m>;
#pragma unroll
    for (int b = 0; b < NL::LG; ++b) {
        if (b > 0) team_swap<m, LR>(lo, hi, lane, b - 1, mask);
        uint32_t bias[LR], s[LR], d[LR], z[LR];
        if (b == NL::LG - 1) {          // sums of m/2 values: bring the limbs back to 26 bits
            lz_norm<LR>(lo);
            lz_norm<LR>(hi);
        }
        ldg_rr<LR>(bias, cst + (NL::BB + b) * LR);
        lz_add<LR>(s, lo, hi);                  // u + v
        lz_sub<LR>(d, lo, bias, hi);            // u - v
        if (b == NL::LG - 1) {
            uint32_t c[LR];
            ldg_rr<LR>(c, cst + lo_c * LR);
            ldg_rr<LR>(z, cst + hi_c * LR);
            mmul<LR>(lo, s, c, md);
            mmul<LR>(hi, d, z, md);
        } else {
            const int k = (1 << (NL::LG - 1 - b)) + (lane >> b);
            ldg_rr<LR>(z, cst + (NL::ZI + k) * LR);
#pragma unroll
            for (int w = 0; w < LR; ++w) lo[w] = s[w];
            mmul<LR>(hi, d, z, md);
        }
    }
}

}  // namespace dkss
