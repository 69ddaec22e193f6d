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
// One team of m/4 lanes owns an element; each lane holds four residues whose
// indices differ in two "local" index bits, so two butterfly stages run in
// registers (two independent butterflies per lane and stage), after which the
// team exchanges values through its shared-memory buffer to make the next two
// index bits local.  Forward stages use Cooley-Tukey butterflies with
// psi^brv(k) (psi = gamma), which leave evaluations in bit-reversed order;
// backwards stages use Gentleman-Sande butterflies with psi^-brv(k) and
// return natural order.
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
    static constexpr int EVB = Q + 7;       // biases of the DFTs in evaluation coordinates, LG + 1 stages
    static constexpr int PSI = EVB + LG + 1;  // psi^t R', t in [0, 2m)
    static constexpr int COUNT = PSI + 2 * m;
};

template <int LR>
__device__ __forceinline__ void ldg_rr(uint32_t (&x)[LR], const uint32_t* p) {
#pragma unroll
    for (int i = 0; i < LR; ++i) x[i] = __ldg(p + i);
}

// r = a + b, limbwise
template <int LR>
DKSS_HD void lz_add(uint32_t (&r)[LR], const uint32_t (&a)[LR], const uint32_t (&b)[LR]) {
#pragma unroll
    for (int i = 0; i < LR; ++i) r[i] = a[i] + b[i];
}

// r = a + B - b, limbwise (B[i] >= b[i] for every i)
template <int LR>
DKSS_HD void lz_sub(uint32_t (&r)[LR], const uint32_t (&a)[LR], const uint32_t (&B)[LR],
                                       const uint32_t (&b)[LR]) {
#pragma unroll
    for (int i = 0; i < LR; ++i) r[i] = a[i] + B[i] - b[i];
}

// Montgomery product a b 2^(-26 LR) mod q as normalised limbs of a value
// below a b / R' + q (the top limb holds every bit above 26 (LR - 1)).
template <int LR>
DKSS_HD void mmul(uint32_t (&r)[LR], const uint32_t (&a)[LR], const uint32_t (&b)[LR],
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

// A modulus p^z = 1 (mod 2^26) whose 26-bit limbs 1 .. LR-2 are zero: a Proth
// prime p = h 2^n + 1 with z = 1 and 26 (LR-1) <= n (the thesis's primes,
// Section 4.1; its outlook proposes exploiting their form in the modular
// reductions).  Then -(p^z)^-1 = -1 (mod 2^26): the Montgomery digit of a
// column is its negated low 26 bits (no product), and adding digit * p^z
// touches the column itself and the top limb only (one limb product per
// digit instead of LR + 1).  The digits and the result are those of mmul with
// the same modulus; only products by zero limbs are left out.
template <int LR>
struct ModRRSparse : ModRR<LR> {};

template <int LR>
DKSS_HD void mmul(uint32_t (&r)[LR], const uint32_t (&a)[LR], const uint32_t (&b)[LR],
                                     const ModRRSparse<LR>& md) {
    uint64_t col[2 * LR];
#pragma unroll
    for (int i = 0; i < 2 * LR; ++i) col[i] = 0;
    mac_cols<LR>(col, a, b);
    const uint32_t qtop = md.q[LR - 1];
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const uint32_t qi = (0u - (uint32_t)col[i]) & kM26;
        const uint64_t c = col[i] + qi;                       // low 26 bits become 0
        col[i + 1] += c >> 26;
        col[i + LR - 1] += (uint64_t)qi * qtop;
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
DKSS_HD void canon(uint32_t (&r)[LR], const uint32_t (&x)[LR], const ModRR<LR>& md) {
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
DKSS_HD void lz_norm(uint32_t (&x)[LR]) {
    uint32_t carry = 0;
#pragma unroll
    for (int i = 0; i + 1 < LR; ++i) {
        const uint32_t v = x[i] + carry;
        carry = (v >> 26) + (v < carry ? 64u : 0u);
        x[i] = v & kM26;
    }
    x[LR - 1] += carry;
}

// Canonical residue of a lazy value x (limbs below 2^32, value below 2^20 q):
// quotient estimate k from the top two limbs, one multi-limb subtraction of
// (k - 1) q, then two conditional subtractions.  With V the top two limbs of x
// (after carrying to 26-bit limbs) and Q those of q, k = floor(V / Q) -- a
// multiply-high by the plan's reciprocal floor((2^64 - 1) / Q), which is k or
// k - 1, and one correction -- is within one of floor(x / q) because Q is at
// least 2^18 and the quotient below 2^12 (the plan's limb choice and host
// check), so x - (k - 1) q is in [0, 3q).  Integer arithmetic only.
DKSS_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

template <int LR>
DKSS_HD void reduce_raw(uint32_t (&r)[LR], const uint32_t (&x)[LR], const ModRR<LR>& md) {
    uint32_t y[LR];
#pragma unroll
    for (int i = 0; i < LR; ++i) y[i] = x[i];
    lz_norm<LR>(y);
    const uint64_t V = ((uint64_t)y[LR - 1] << 26) + y[LR - 2];          // below 2^58
    const uint64_t Q = ((uint64_t)md.q[LR - 1] << 26) + md.q[LR - 2];
    uint64_t ke = mulhi64(V, md.qtop_inv);                               // floor(V / Q) or one less
    if (V - ke * Q >= Q) ++ke;
    const uint32_t k = ke > 0 ? (uint32_t)ke - 1 : 0;
    int64_t carry = 0;
#pragma unroll
    for (int i = 0; i < LR; ++i) {
        const int64_t acc = (int64_t)y[i] - (int64_t)((uint64_t)k * md.q[i]) + carry;
        if (i + 1 < LR) {
            r[i] = (uint32_t)acc & kM26;
            carry = acc >> 26;
        } else {
            r[i] = (uint32_t)acc;
        }
    }
    canon<LR>(r, r, md);
    canon<LR>(r, r, md);
}

// Position of index i in a team's exchange buffer: an XOR swizzle of its
// low bits by its high bits, so that in every layout below the eight lanes of
// a quarter warp touch eight different 16-byte bank groups (m = 32, 64).
template <int m>
__device__ __forceinline__ int xpos(int i) {
    if constexpr (m == 32) return i ^ (((i >> 3) & 1) * 2) ^ (((i >> 4) & 1) * 5);
    else if constexpr (m == 64) return i ^ ((i >> 3) & 1) ^ (((i >> 4) & 1) * 6);
    else return i;
}

// Residues of 3 or 5 limbs (m = 64) do not fit the 16-byte layout above: the
// exchange buffer then holds one plane of m words per limb (limb w of index
// i at w m + xplane(i)).  With i = (A, B, C) in 2-bit fields, xplane keeps A
// and replaces the low four bits by (A ^ C, B ^ C): in each of the three
// exchange patterns the 16 lanes of a team vary two of the fields, and the
// map is one-to-one on them, so the lanes hit 16 different banks modulo 16;
// the warp's second team flips bit 4 and takes the other 16 banks.
template <int m, int LR>
struct XchgPlanes {
    static constexpr bool value = m == 64 && (LR == 3 || LR == 5);
};

__device__ __forceinline__ int xplane(int i) {
    const int a = i >> 4, b = (i >> 2) & 3, c = i & 3;
    return (a << 4) | ((a ^ c) << 2) | (b ^ c);
}

// Bit 4 for the second team of a warp (teams of 16 lanes, m = 64).
__device__ __forceinline__ int xteam_flip() { return (threadIdx.x & 16); }

// Index held in slot j (0..3) by lane l when the local index bits are (h, h-1).
__device__ __forceinline__ int lidx(int l, int j, int h) {
    const int low = (1 << (h - 1)) - 1;
    return ((l & ~low) << 2) | (j << (h - 1)) | (l & low);
}

// Re-deal the team's 4 m/4 residues from local bits (h_from, h_from - 1) to
// (h_to, h_to - 1) through the team's buffer (m residues of LR words).
template <int m, int LR>
__device__ __forceinline__ void ntt_exchange(uint32_t (&v)[4][LR], uint32_t* buf, int lane, int h_from, int h_to,
                                             unsigned mask) {
    __syncwarp(mask);   // the team's last reads of buf are done
    if constexpr (XchgPlanes<m, LR>::value) {
        const int f = xteam_flip();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = xplane(lidx(lane, j, h_from)) ^ f;
#pragma unroll
            for (int w = 0; w < LR; ++w) buf[w * m + q] = v[j][w];
        }
        __syncwarp(mask);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = xplane(lidx(lane, j, h_to)) ^ f;
#pragma unroll
            for (int w = 0; w < LR; ++w) v[j][w] = buf[w * m + q];
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) st_rr<LR>(buf + xpos<m>(lidx(lane, j, h_from)) * LR, v[j]);
        __syncwarp(mask);
#pragma unroll
        for (int j = 0; j < 4; ++j) ld_rr<LR>(v[j], buf + xpos<m>(lidx(lane, j, h_to)) * LR);
    }
}

// Forward negacyclic transform (lazy).  On entry slot j of lane l holds
// coefficient l + j m/4; on exit the evaluations at bit-reversed positions
// 4l + j.
template <int m, int LR, class MD>
__device__ __forceinline__ void ntt_forward(uint32_t (&v)[4][LR], uint32_t* buf, int lane, unsigned mask,
                                            const uint32_t* cst, const MD& md) {
    using NL = NttLayout<m>;
    constexpr int LG = NL::LG;
    uint32_t bf[LR];
    ldg_rr<LR>(bf, cst + NL::BF * LR);
    int h = LG - 1;
#pragma unroll
    for (int b = LG - 1; b >= 0; --b) {
        if ((LG - 1 - b) % 2 == 0 && b != LG - 1) {   // a new pair of stages: make bits (b, b-1) local
            const int hn = b >= 1 ? b : 1;
            ntt_exchange<m, LR>(v, buf, lane, h, hn, mask);
            h = hn;
        }
        const int sbit = b == h ? 2 : 1;               // slot bit of index bit b
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int jl = sbit == 2 ? p : 2 * p, jh = jl + sbit;
            const int k = (1 << (LG - 1 - b)) + (lidx(lane, jl, h) >> (b + 1));
            uint32_t z[LR], t[LR];
            ldg_rr<LR>(z, cst + (NL::ZF + k) * LR);
            mmul<LR>(t, v[jh], z, md);
            lz_sub<LR>(v[jh], v[jl], bf, t);       // lo - t
            lz_add<LR>(v[jl], v[jl], t);           // lo + t
        }
    }
}

// Backwards transform scaled by a constant.  On entry slot j of lane l holds
// the evaluation at bit-reversed position 4l + j; on exit coefficient
// l + j m/4 of the interpolated element times c (normalised, below 2q), where
// the last stage multiplies by cst[lo_c] and cst[hi_c] (= c and psi^-1 c,
// times R').  With RAW_LO (c = 1, already folded into the inputs) the last
// stage leaves slots 0 and 1 as the plain sums, unreduced (reduce_raw), and
// multiplies only slots 2 and 3 by cst[hi_c].
template <int m, int LR, bool RAW_LO = false, class MD = ModRR<LR>>
__device__ __forceinline__ void ntt_backward(uint32_t (&v)[4][LR], uint32_t* buf, int lane, unsigned mask,
                                             const uint32_t* cst, int lo_c, int hi_c, const MD& md) {
    using NL = NttLayout<m>;
    constexpr int LG = NL::LG;
    int h = 1;
#pragma unroll
    for (int b = 0; b < LG; ++b) {
        if (b % 2 == 0 && b != 0) {                      // make bits (b+1, b) local
            const int hn = b + 1 <= LG - 1 ? b + 1 : LG - 1;
            ntt_exchange<m, LR>(v, buf, lane, h, hn, mask);
            h = hn;
        }
        if (b == LG - 1) {                               // sums of m/2 values: limbs back to 26 bits
#pragma unroll
            for (int j = 0; j < 4; ++j) lz_norm<LR>(v[j]);
        }
        uint32_t bias[LR];
        ldg_rr<LR>(bias, cst + (NL::BB + b) * LR);
        const int sbit = b == h ? 2 : 1;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int jl = sbit == 2 ? p : 2 * p, jh = jl + sbit;
            uint32_t s[LR], d[LR], z[LR];
            lz_add<LR>(s, v[jl], v[jh]);                 // u + v
            lz_sub<LR>(d, v[jl], bias, v[jh]);           // u - v
            if (b == LG - 1) {
                ldg_rr<LR>(z, cst + hi_c * LR);
                if constexpr (RAW_LO) {
#pragma unroll
                    for (int w = 0; w < LR; ++w) v[jl][w] = s[w];
                } else {
                    uint32_t c[LR];
                    ldg_rr<LR>(c, cst + lo_c * LR);
                    mmul<LR>(v[jl], s, c, md);
                }
                mmul<LR>(v[jh], d, z, md);
            } else {
                const int k = (1 << (LG - 1 - b)) + (lidx(lane, jl, h) >> (b + 1));
                ldg_rr<LR>(z, cst + (NL::ZI + k) * LR);
#pragma unroll
                for (int w = 0; w < LR; ++w) v[jl][w] = s[w];
                mmul<LR>(v[jh], d, z, md);
            }
        }
    }
}

}  // namespace dkss
