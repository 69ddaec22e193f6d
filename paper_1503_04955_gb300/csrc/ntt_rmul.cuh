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
// Residues are 26-bit limbs (rr_arith.cuh); sums stay below 2^lg(m) p^z and
// the plan picks LR with 4 m p^z < 2^(26 LR), so every Montgomery product
// input is in range.
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
    static constexpr int BIAS = 2 * m;      // 2^b p^z, b < LG (normalised)
    static constexpr int Q = BIAS + LG;     // p^z
    static constexpr int TW_LO = Q + 1;     // m^-1 R'            (last backwards stage, twiddles)
    static constexpr int TW_HI = Q + 2;     // psi^-1 m^-1 R'
    static constexpr int PW_LO = Q + 3;     // m^-1 (2M)^-1 R'^2  (componentwise products of
    static constexpr int PW_HI = Q + 4;     // psi^-1 m^-1 (2M)^-1 R'^2   two normal-form factors)
    static constexpr int COUNT = Q + 5;
};

template <int LR>
__device__ __forceinline__ void ldg_rr(uint32_t (&x)[LR], const uint32_t* p) {
#pragma unroll
    for (int i = 0; i < LR; ++i) x[i] = __ldg(p + i);
}

// r = a + b, limbs normalised to 26 bits (the value must fit in LR limbs)
template <int LR>
__device__ __forceinline__ void add_norm(uint32_t (&r)[LR], const uint32_t (&a)[LR], const uint32_t (&b)[LR]) {
    uint32_t carry = 0;
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const uint32_t s = a[i] + b[i] + carry;
        r[i] = i + 1 < LR ? (s & kM26) : s;
        carry = s >> 26;
    }
}

// r = c - v for normalised c >= v
template <int LR>
__device__ __forceinline__ void sub_norm(uint32_t (&r)[LR], const uint32_t (&c)[LR], const uint32_t (&v)[LR]) {
    uint32_t borrow = 0;
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const uint32_t d = c[i] - v[i] - borrow;
        borrow = d >> 31;
        r[i] = d & kM26;
    }
}

// canonical product a * b * 2^(-26 LR) mod q (a b < q 2^(26 LR))
template <int LR>
__device__ __forceinline__ void mmul(uint32_t (&r)[LR], const uint32_t (&a)[LR], const uint32_t (&b)[LR],
                                     const ModRR<LR>& md) {
    mont_mul_rr<LR>(r, a, b, md);
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
// on exit the evaluations with bit-reversed indices 2l, 2l+1.
template <int m, int LR>
__device__ __forceinline__ void ntt_forward(uint32_t (&lo)[LR], uint32_t (&hi)[LR], int lane, unsigned mask,
                                            const uint32_t* cst, const ModRR<LR>& md) {
    using NL = NttLayout<m>;
    uint32_t q[LR];
    ldg_rr<LR>(q, cst + NL::Q * LR);
#pragma unroll
    for (int b = NL::LG - 1; b >= 0; --b) {
        if (b < NL::LG - 1) team_swap<m, LR>(lo, hi, lane, b, mask);
        const int k = (1 << (NL::LG - 1 - b)) + (lane >> b);
        uint32_t z[LR], t[LR], d[LR];
        ldg_rr<LR>(z, cst + (NL::ZF + k) * LR);
        mmul<LR>(t, hi, z, md);           // canonical, < q
        sub_norm<LR>(d, q, t);            // q - t
        add_norm<LR>(hi, lo, d);          // lo - t + q
        add_norm<LR>(lo, lo, t);          // lo + t
    }
}

// Backwards transform scaled by a constant: on entry lane l holds the
// evaluations 2l, 2l+1 (bit-reversed order); on exit the canonical
// coefficients l, l+m/2 of the interpolated element times c, where the last
// stage multiplies by cst[lo_c] and cst[hi_c] (= c and psi^-1 c, times R').
template <int m, int LR>
__device__ __forceinline__ void ntt_backward(uint32_t (&lo)[LR], uint32_t (&hi)[LR], int lane, unsigned mask,
                                             const uint32_t* cst, int lo_c, int hi_c, const ModRR<LR>& md) {
    using NL = NttLayout<m>;
#pragma unroll
    for (int b = 0; b < NL::LG; ++b) {
        if (b > 0) team_swap<m, LR>(lo, hi, lane, b - 1, mask);
        uint32_t bias[LR], s[LR], dd[LR], d[LR], z[LR];
        ldg_rr<LR>(bias, cst + (NL::BIAS + b) * LR);   // 2^b q >= hi
        add_norm<LR>(s, lo, hi);                        // u + v
        sub_norm<LR>(dd, bias, hi);
        add_norm<LR>(d, lo, dd);                        // u - v + 2^b q
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
