// Levels of the transform in the evaluation coordinates of R (DKSS_LEVELS_EVAL;
// by default every level runs on coefficients with alpha-shift inner DFTs).
//
// The map x -> (x(gamma^(2j+1)))_j, j < m, is a ring isomorphism R -> P^m
// (P = Z/p^zZ; the thesis builds rho through it, Section 3.2.3).  Under it
// alpha goes to gamma^(2j+1), so an inner DFT of a level, X_v = sum_j x_j
// alpha^(jv), becomes m independent DFTs over P, one per coordinate with root
// gamma^(2j+1), and a bad twiddle rho^e becomes the pointwise factors
// rho^e(gamma^(2j+1)) = omega^(e(2j+1)).  The transform computed is the same
// one (a linear map over R); only the coordinates of the inner levels change:
//   level 0 forward   inner DFT by alpha-shifts (coefficients), then each
//                     element is mapped to evaluation coordinates (the
//                     forward NTT of ntt_rmul.cuh) and multiplied by its
//                     twiddle there;
//   levels d >= 1     DFTs over P per coordinate, pointwise twiddles;
//   last level        DFTs over P, the componentwise products, inverse DFTs;
//   level 0 backwards twiddle pointwise, back to coefficients (the backward
//                     NTT, scaled by m^-1), alpha^r as a coefficient shift,
//                     then the inner DFT by alpha-shifts.
// Between kernels an element is m canonical residues of L words in
// bit-reversed coordinate order: index i holds x(gamma^(2 brv(i) + 1)).  Inside
// a kernel residues are 26-bit limbs with the lazy sums of ntt_rmul.cuh; the
// plan's host check (ntt_bounds.cpp) covers DFTs of up to 2m points.
#pragma once
#include <cstdint>

namespace dkss {

// coordinates per CTA of the evaluation-coordinate DFT kernels: a whole element
// for m <= 32 (contiguous loads and stores of m residues)
template <int m>
struct EvalKC {
    static constexpr int value = m < 32 ? m : 32;
};

// Radix-2 DIT over `arrays` consecutive arrays of n elements, each element
// KC = EvalKC<m> coordinates of LR words: residue (array a, slot s, coordinate c) at
// buf + ((a n + s) KC + c) LR.  Input in bit-reversed slots, output in
// natural slots.  Coordinate c is storage index i0 + c of the element, whose
// root is gamma^((2 brv(i) + 1) rexp) (rexp: exponent of alpha of the DFT's
// root).  Butterflies (t = b w; a + t; a + B_s - t) are lazy; where the
// twiddle is 1 (k = 0) and bit s of `skip` is set, t = b without a product (the
// plan admits a stage only where its bounds allow).  Butterflies are dealt so
// that the two of a warp share k, which keeps those warps uniform.
template <int m, int LR>
__device__ void eval_dit(uint32_t* buf, int arrays, int n, int rexp, int i0, const uint32_t* cst, uint32_t skip,
                         const ModRR<LR>& md) {
    constexpr int KC = EvalKC<m>::value;
    using NL = NttLayout<m>;
    const int log2n = 31 - __clz(n);
    const int tasks = arrays * (n / 2) * KC;
    for (int lh = 0; lh < log2n; ++lh) {
        const int half = 1 << lh;
        const int scale = n >> (lh + 1);
        const int lg_groups = log2n - lh - 1;       // blocks of 2 half slots: n >> (lh + 1)
        uint32_t bs[LR];
        ldg_rr<LR>(bs, cst + (NL::EVB + lh) * LR);
        for (int task = threadIdx.x; task < tasks; task += kThreads) {
            const int c = task % KC, rest = task / KC;
            const int arr = rest >> (log2n - 1), idx = rest & (n / 2 - 1);
            const int g = idx & ((1 << lg_groups) - 1), k_in = idx >> lg_groups;
            const int ia = g * 2 * half + k_in, ib = ia + half;
            uint32_t* pa = buf + ((arr * n + ia) * KC + c) * LR;
            uint32_t* pb = buf + ((arr * n + ib) * KC + c) * LR;
            uint32_t a[LR], b[LR], t[LR];
            ld_rr<LR>(a, pa);
            ld_rr<LR>(b, pb);
            if (k_in == 0 && ((skip >> lh) & 1)) {
#pragma unroll
                for (int w = 0; w < LR; ++w) t[w] = b[w];
            } else {
                const int sh = (rexp * scale * k_in) & (2 * m - 1);
                const int ex = ((2 * (int)bitrev((uint32_t)(i0 + c), NL::LG) + 1) * sh) & (2 * m - 1);
                uint32_t z[LR];
                ldg_rr<LR>(z, cst + (NL::PSI + ex) * LR);
                mmul<LR>(t, b, z, md);
            }
            uint32_t s0[LR], s1[LR];
            lz_add<LR>(s0, a, t);
            lz_sub<LR>(s1, a, bs, t);
            st_rr<LR>(pa, s0);
            st_rr<LR>(pb, s1);
        }
        __syncthreads();
    }
}

// canonical residue of x (lazy, limbs as left by mmul) in L words at dst
template <int L, int LR>
__device__ __forceinline__ void store_canon(uint32_t* dst, const uint32_t (&x)[LR], const ModRR<LR>& mr) {
    uint32_t c[LR], o[L];
    canon<LR>(c, x, mr);
    from_rr<L, LR>(o, c);
    st_res<L>(dst, o);
}

// ---------------------------------------------------------------------------
// Level 0 forward: inner DFT of a column by alpha-shifts (encoding its
// inputs), then each of its 2m outputs times its bad twiddle in evaluation
// coordinates (forward NTT, pointwise product), written in storage order.
// ---------------------------------------------------------------------------
template <int m, int L, int LR>
__device__ __forceinline__ void level0_fwd_eval(const LevelParams& prm, const Mod<L>& md, const ModRR<LR>& mr,
                                                uint32_t* smem, uint64_t column, int op) {
    using G = Geo<m, L>;
    using NT = NttTeam<m>;
    uint32_t* col = smem;
    uint32_t* xbuf = smem + G::TWO_M * G::ES;
    uint32_t* poly = prm.data + (op ? prm.poly_words : 0);
    const int lg_mu = (__ffsll((long long)prm.len) - 1) - ilog2<G::TWO_M>();
    const uint64_t mu_d = 1ull << lg_mu;
    const uint64_t blk = column >> lg_mu, l = column & (mu_d - 1);
    const uint64_t base = blk * prm.len;
    column_load_fwd<m, L, true>(prm, col, column, op);
    __syncthreads();
    dft_dit<m, L>(col, 1, G::TWO_M, 1, md);     // ends with __syncthreads: output v in slot v
    NT nt;
    uint32_t* buf = xbuf + nt.id * m * LR;
    const int lane = nt.lane;
    uint32_t bn[LR];
    ldg_rr<LR>(bn, prm.ntt_cst + NttLayout<m>::BN * LR);
    for (int v = nt.id; v < G::TWO_M; v += NT::NTEAMS) {
        const uint32_t* src = col + v * G::ES;
        uint32_t* dst = poly + (base + (uint64_t)v * mu_d + l) * G::EW;
        const uint64_t e = (uint64_t)v * l * prm.bp;      // rho^e = alpha^r rho^s
        const int r = (int)(e >> prm.log2_mu_top);
        const uint64_t sidx = e & (prm.mu_top - 1);
        uint32_t vv[4][LR];
#pragma unroll
        for (int j = 0; j < 4; ++j) load_shifted_rr<m, L, LR>(vv[j], src, lane + j * NT::TEAM, r, bn);
        ntt_forward<m, LR>(vv, buf, lane, nt.mask, prm.ntt_cst, mr);
        const uint32_t* tw = prm.table_eval + (sidx * m + 4 * lane) * LR;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t t[LR];
            ldg_rr<LR>(t, tw + j * LR);
            mmul<LR>(vv[j], vv[j], t, mr);
            store_canon<L, LR>(dst + (4 * lane + j) * L, vv[j], mr);
        }
    }
}

template <int m, int L, int LR>
__global__ void __launch_bounds__(kThreads, 4) k_level0_fwd_eval(LevelParams prm, Mod<L> md, ModRR<LR> mr) {
    extern __shared__ __align__(16) uint32_t smem[];
    level0_fwd_eval<m, L, LR>(prm, md, mr, smem, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Level d >= 1 forward in evaluation coordinates: one CTA per (column,
// KC coordinates): 2m-point DFTs over P, then the pointwise twiddles
// omega^(v l b_d (2j+1)) from the level's table (prm.tw_lvl).
// ---------------------------------------------------------------------------
template <int m, int L, int LR>
__global__ void __launch_bounds__(kThreads) k_level_eval_fwd(LevelParams prm, ModRR<LR> mr) {
    constexpr int KC = EvalKC<m>::value;
    using G = Geo<m, L>;
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int LOG2_TWO_M = ilog2<G::TWO_M>();
    const uint64_t column = blockIdx.x;
    const int i0 = blockIdx.y * KC;
    uint32_t* poly = prm.data + (blockIdx.z ? prm.poly_words : 0);
    const int lg_mu = (__ffsll((long long)prm.len) - 1) - LOG2_TWO_M;
    const uint64_t mu_d = 1ull << lg_mu;
    const uint64_t blk = column >> lg_mu, l = column & (mu_d - 1);
    const uint64_t base = blk * prm.len;
    for (int idx = threadIdx.x; idx < G::TWO_M * KC; idx += kThreads) {
        const int j = idx / KC, c = idx % KC;
        uint32_t x[L], y[LR];
        ld_res<L>(x, poly + (base + (uint64_t)j * mu_d + l) * G::EW + (i0 + c) * L);
        to_rr<L, LR>(y, x);
        st_rr<LR>(smem + ((int)bitrev(j, LOG2_TWO_M) * KC + c) * LR, y);
    }
    __syncthreads();
    eval_dit<m, LR>(smem, 1, G::TWO_M, 1, i0, prm.ntt_cst, prm.eval_skip, mr);
    for (int idx = threadIdx.x; idx < G::TWO_M * KC; idx += kThreads) {
        const int v = idx / KC, c = idx % KC;
        uint32_t x[LR], t[LR];
        ld_rr<LR>(x, smem + (v * KC + c) * LR);
        ldg_rr<LR>(t, prm.tw_lvl + ((uint64_t)v * l * m + i0 + c) * LR);
        mmul<LR>(x, x, t, mr);
        store_canon<L, LR>(poly + (base + (uint64_t)v * mu_d + l) * G::EW + (i0 + c) * L, x, mr);
    }
}

// ---------------------------------------------------------------------------
// Level d >= 1 backwards: pointwise twiddles omega^(-v l b_d (2j+1)), then
// 2m-point DFTs over P with root gamma^(-(2j+1)).
// ---------------------------------------------------------------------------
template <int m, int L, int LR>
__global__ void __launch_bounds__(kThreads) k_level_eval_inv(LevelParams prm, ModRR<LR> mr) {
    constexpr int KC = EvalKC<m>::value;
    using G = Geo<m, L>;
    using NL = NttLayout<m>;
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int LOG2_TWO_M = ilog2<G::TWO_M>();
    const uint64_t column = blockIdx.x;
    const int i0 = blockIdx.y * KC;
    uint32_t* poly = prm.data;
    const int lg_mu = (__ffsll((long long)prm.len) - 1) - LOG2_TWO_M;
    const uint64_t mu_d = 1ull << lg_mu;
    const uint64_t blk = column >> lg_mu, l = column & (mu_d - 1);
    const uint64_t base = blk * prm.len;
    const uint64_t n_tw = prm.P2 / prm.bp;             // entries of the level's table
    for (int idx = threadIdx.x; idx < G::TWO_M * KC; idx += kThreads) {
        const int j = idx / KC, c = idx % KC;
        uint32_t x[L], y[LR], t[LR];
        ld_res<L>(x, poly + (base + (uint64_t)j * mu_d + l) * G::EW + (i0 + c) * L);
        to_rr<L, LR>(y, x);
        const uint64_t e = (n_tw - (uint64_t)j * l) & (n_tw - 1);
        ldg_rr<LR>(t, prm.tw_lvl + (e * m + i0 + c) * LR);
        mmul<LR>(y, y, t, mr);
        st_rr<LR>(smem + ((int)bitrev(j, LOG2_TWO_M) * KC + c) * LR, y);
    }
    __syncthreads();
    eval_dit<m, LR>(smem, 1, G::TWO_M, G::TWO_M - 1, i0, prm.ntt_cst, prm.eval_skip, mr);
    uint32_t one[LR];
    ldg_rr<LR>(one, prm.ntt_cst + NL::ONE * LR);
    for (int idx = threadIdx.x; idx < G::TWO_M * KC; idx += kThreads) {
        const int v = idx / KC, c = idx % KC;
        uint32_t x[LR];
        ld_rr<LR>(x, smem + (v * KC + c) * LR);
        mmul<LR>(x, x, one, mr);
        store_canon<L, LR>(poly + (base + (uint64_t)v * mu_d + l) * G::EW + (i0 + c) * L, x, mr);
    }
}

// Elements of the last level per CTA of k_final_eval (whole blocks of n).
template <int m>
__host__ __device__ constexpr int final_eval_elems(int n) {
    return n >= 32 ? n : 32;
}

// ---------------------------------------------------------------------------
// Last level in evaluation coordinates: n-point DFTs over P (root
// gamma^((2j+1) 2m/n)) of a and b, componentwise products scaled by (2M)^-1,
// inverse DFTs; one CTA per (final_eval_elems elements, KC coordinates).
// smem: A, B and C, final_eval_elems x KC residues each.
// ---------------------------------------------------------------------------
template <int m, int L, int LR>
__global__ void __launch_bounds__(kThreads) k_final_eval(LevelParams prm, ModRR<LR> mr) {
    constexpr int KC = EvalKC<m>::value;
    using G = Geo<m, L>;
    using NL = NttLayout<m>;
    extern __shared__ __align__(16) uint32_t smem[];
    const int n = (int)prm.len;
    const int log2n = 31 - __clz(n);
    const int nn = final_eval_elems<m>(n);
    const int i0 = blockIdx.y * KC;
    const uint64_t base = (uint64_t)blockIdx.x * nn;
    uint32_t* sa = smem;
    uint32_t* sb = sa + nn * KC * LR;
    uint32_t* sc = sb + nn * KC * LR;
    uint32_t* pa = prm.data;
    uint32_t* pb = prm.data + prm.poly_words;
    for (int idx = threadIdx.x; idx < nn * KC; idx += kThreads) {
        const int j = idx / KC, c = idx % KC;
        const int slot = ((j >> log2n) << log2n) + (int)bitrev(j & (n - 1), log2n);
        uint32_t x[L], y[LR];
        ld_res<L>(x, pa + (base + j) * G::EW + (i0 + c) * L);
        to_rr<L, LR>(y, x);
        st_rr<LR>(sa + (slot * KC + c) * LR, y);
        ld_res<L>(x, pb + (base + j) * G::EW + (i0 + c) * L);
        to_rr<L, LR>(y, x);
        st_rr<LR>(sb + (slot * KC + c) * LR, y);
    }
    __syncthreads();
    const int rexp = G::TWO_M / n;
    eval_dit<m, LR>(sa, 2 * (nn / n), n, rexp, i0, prm.ntt_cst, prm.eval_skip, mr);   // a and b (sb follows sa)
    // componentwise products a b (2M)^-1: b scaled first, or, where the plan's
    // bounds allow, a b unscaled and (2M)^-1 taken by the final reduction
    uint32_t ks[LR];
#pragma unroll
    for (int w = 0; w < LR; ++w) ks[w] = prm.kscale[w];      // (2M)^-1 R'^2
    const bool noscale = prm.eval_noscale != 0;
    for (int idx = threadIdx.x; idx < nn * KC; idx += kThreads) {
        const int v = idx / KC, c = idx % KC;
        uint32_t x[LR], y[LR];
        ld_rr<LR>(x, sa + (v * KC + c) * LR);
        ld_rr<LR>(y, sb + (v * KC + c) * LR);
        if (!noscale) mmul<LR>(y, y, ks, mr);                 // b (2M)^-1 R'
        mmul<LR>(x, x, y, mr);
        const int slot = ((v >> log2n) << log2n) + (int)bitrev(v & (n - 1), log2n);
        st_rr<LR>(sc + (slot * KC + c) * LR, x);
    }
    __syncthreads();
    eval_dit<m, LR>(sc, nn / n, n, (G::TWO_M - rexp) & (G::TWO_M - 1), i0, prm.ntt_cst, prm.eval_skip, mr);
    // final reduction: by 1, or by (2M)^-1 R'^2 where the products were unscaled
    // (a Montgomery product of two plain residues leaves a factor R'^-1)
    uint32_t one[LR];
    ldg_rr<LR>(one, prm.ntt_cst + NL::ONE * LR);
    if (noscale) {
#pragma unroll
        for (int w = 0; w < LR; ++w) one[w] = ks[w];
    }
    for (int idx = threadIdx.x; idx < nn * KC; idx += kThreads) {
        const int v = idx / KC, c = idx % KC;
        uint32_t x[LR];
        ld_rr<LR>(x, sc + (v * KC + c) * LR);
        mmul<LR>(x, x, one, mr);
        store_canon<L, LR>(pa + (base + v) * G::EW + (i0 + c) * L, x, mr);
    }
}

// ---------------------------------------------------------------------------
// Level 0 backwards: each element of a column times its bad twiddle rho^s in
// evaluation coordinates, back to coefficients (backward NTT with m^-1), times
// alpha^r as a coefficient shift, into the column's slot; then the inner DFT by
// alpha^-1-shifts and the write-back (as k_dft_inv).
// ---------------------------------------------------------------------------
template <int m, int L, int LR>
__device__ __forceinline__ void level0_inv_eval(const LevelParams& prm, const Mod<L>& md, const ModRR<LR>& mr,
                                                uint32_t* smem, uint64_t column) {
    using G = Geo<m, L>;
    using NT = NttTeam<m>;
    constexpr int LOG2_TWO_M = ilog2<G::TWO_M>();
    uint32_t* col = smem;
    uint32_t* xbuf = smem + G::TWO_M * G::ES;
    uint32_t* poly = prm.data;
    const int lg_mu = (__ffsll((long long)prm.len) - 1) - LOG2_TWO_M;
    const uint64_t mu_d = 1ull << lg_mu;
    const uint64_t blk = column >> lg_mu, l = column & (mu_d - 1);
    const uint64_t base = blk * prm.len;
    NT nt;
    uint32_t* buf = xbuf + nt.id * m * LR;
    const int lane = nt.lane;
    for (int v = nt.id; v < G::TWO_M; v += NT::NTEAMS) {
        const uint32_t* src = poly + (base + (uint64_t)v * mu_d + l) * G::EW;
        const uint64_t e = (prm.P2 - (uint64_t)v * l * prm.bp) & (prm.P2 - 1);   // rho^-vl b = alpha^r rho^s
        const int r = (int)(e >> prm.log2_mu_top);
        const uint64_t sidx = e & (prm.mu_top - 1);
        const uint32_t* tw = prm.table_eval + (sidx * m + 4 * lane) * LR;
        uint32_t vv[4][LR];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t x[L], t[LR];
            ld_res<L>(x, src + (4 * lane + j) * L);
            to_rr<L, LR>(vv[j], x);
            ldg_rr<LR>(t, tw + j * LR);
            mmul<LR>(vv[j], vv[j], t, mr);
        }
        ntt_backward<m, LR>(vv, buf, lane, nt.mask, prm.ntt_cst, NttLayout<m>::TW_LO, NttLayout<m>::TW_HI, mr);
        // coefficient k of alpha^r y is +-y[k - r]: y's coefficient t goes to (t + r) mod m
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = lane + j * NT::TEAM;
            int pos = t + r;
            bool neg = false;
            if (pos >= m) {
                pos -= m;
                neg = true;
                if (pos >= m) {
                    pos -= m;
                    neg = false;
                }
            }
            uint32_t c[LR], o[L];
            canon<LR>(c, vv[j], mr);
            if (neg) neg_rr<LR>(c, c, mr);
            from_rr<L, LR>(o, c);
            st_res<L>(col + v * G::ES + pos * L, o);
        }
    }
    __syncthreads();
    dft_dif<m, L>(col, 1, G::TWO_M, G::TWO_M - 1, md);
    for (int idx = threadIdx.x; idx < G::TWO_M * m; idx += kThreads) {
        int j = idx / m, t = idx % m;
        uint32_t x[L];
        ld_res<L>(x, col + bitrev(j, LOG2_TWO_M) * G::ES + t * L);
        st_res<L>(poly + ((base + (uint64_t)j * mu_d + l) * m + t) * L, x);
    }
}

template <int m, int L, int LR>
__global__ void __launch_bounds__(kThreads, 4) k_level0_inv_eval(LevelParams prm, Mod<L> md, ModRR<LR> mr) {
    extern __shared__ __align__(16) uint32_t smem[];
    level0_inv_eval<m, L, LR>(prm, md, mr, smem, blockIdx.x);
}

template <int m, int L, int LR>
constexpr size_t level_eval_smem_bytes() {
    return sizeof(uint32_t) * (size_t)Geo<m, L>::TWO_M * EvalKC<m>::value * LR;
}

template <int m, int L, int LR>
size_t final_eval_smem_bytes(int n) {
    return sizeof(uint32_t) * 3 * (size_t)final_eval_elems<m>(n) * EvalKC<m>::value * LR;
}

}  // namespace dkss
