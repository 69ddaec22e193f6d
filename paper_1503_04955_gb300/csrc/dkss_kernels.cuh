// DKSS_MUL stage kernels (thesis Section 3.2 steps 4-8, Section 4.2).
//
// Layout in HBM: a polynomial over R is 2M elements, element e holds m
// residues (inner coefficients) of L 32-bit limbs, residue-major:
// word (e*m + t)*L + l.  Every kernel below works on that layout.
//
// The forward 2M-point transform is the thesis's radix-2m decimation in time
// (Section 3.2.5 i.-iii.), done in place level by level: level d splits each
// block of len = 2M/(2m)^(d-1) elements into 2m rows of len/2m columns; one
// CTA takes one column and runs the 2m-point inner DFT with root alpha (shifts
// only) in shared memory, then multiplies output v of column l by the bad
// twiddle rho^(v*l*(2m)^(d-1)) (k_level_fwd_ntt; for m = 64, or the direct and
// INT8 forms, a column-DFT kernel followed by an element-parallel twiddle
// kernel).  After the last level the elements sit in
// mixed-radix digit-reversed order.  Componentwise products do not care about
// order; the backwards transform runs the same levels in reverse as
// decimation in frequency with rho^-1 and alpha^-1 (the backwards transform
// of Section 2.7), which returns natural order.
#pragma once
#include <cstdint>

#include "arith.cuh"
#include "i8_rmul.cuh"
#include "ntt_rmul.cuh"
#include "padic.cuh"
#include "rr_arith.cuh"

namespace dkss {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <int m, int L>
struct Geo {
    static constexpr int TWO_M = 2 * m;
    static constexpr int EW = m * L;                     // words per element of R
    // Shared-memory stride of an element: EW, padded for 3-word residues at
    // m <= 32 so that the teams of a warp (2 of 16 lanes for m = 32, 4 of 8
    // for m = 16), which work on different elements with scalar accesses,
    // start in different banks (96 + 16 and 48 + 8 words).  The layout in HBM
    // keeps EW.
    static constexpr int ES = EW + ((L == 3 && m == 32) ? 16 : (L == 3 && m == 16) ? 8 : 0);
    static constexpr int TEAM = m / 2;                   // lanes per element in the DFTs and the direct
                                                         // form (2 coefficients each)
    static constexpr int TEAMS_PER_WARP = 32 / TEAM;
    static constexpr int NTEAMS = kWarps * TEAMS_PER_WARP;
    static constexpr int CPL = m / TEAM;                 // coefficients per lane
};

// Per-team shared buffers of an R-multiplication in 26-bit limbs: the first
// factor x (m residues) and the extended second factor E (2m residues).
template <int m, int LR>
struct TeamBuf {
    static constexpr int WORDS = 3 * m * LR;
};

struct LevelParams {
    uint32_t* data;            // one or two polynomials (operand b at data + poly_words)
    const uint64_t* raw_a;     // encode source of operand a (first forward level)
    const uint64_t* raw_b;
    const uint32_t* table;     // rho^s R' mod p^z, s < mu_top: m residues of LR 26-bit limbs each
    uint64_t poly_words;
    uint64_t P2;               // 2M
    uint64_t mu_top;           // 2M / 2m
    uint64_t len;              // block length at this level
    uint64_t bp;               // (2m)^(level-1)
    uint64_t M;
    uint64_t n_bits;
    uint64_t raw_words;
    uint32_t u;
    uint32_t log2_mu_top;
    uint32_t kscale[5];        // (2M)^-1 R'^2 mod p^z in 26-bit limbs, R' = 2^(26 LR)
    const uint32_t* table_eval;  // rho^s(gamma^(2 brv(i)+1)) R', s < mu_top, i < m: LR words each
    const uint32_t* ntt_cst;     // NttLayout<m> constants, LR words each
    uint32_t i8_S;               // bytes per residue (INT8 tensor-core form)
    uint32_t ntt_prescale;       // NTT form: scale b before the componentwise product
    const uint32_t* tw_lvl;      // inner levels in evaluation coordinates: this level's twiddles
    uint32_t eval_skip;          // their DFTs: bit s = stage s adds t = b unreduced where the twiddle is 1
    uint32_t eval_noscale;       // last level: multiply a b unscaled, scale by (2M)^-1 at the end
    uint32_t square;             // last level of a square (b is a): one forward transform per element
    uint32_t dft_lazy;           // m = 64 forward half-column DFTs with unreduced sums (2^7 p^z fits the words)
    uint32_t red_rcp;            // floor(2^40 / (q_top + 1)), q_top the top word of p^z (their final reduction)
    uint32_t pd_io;              // the forward levels keep p-adic digits in HBM (4 words, padic.cuh)
    uint32_t pd_fast;            // their conversions may take the fast carries (ModPD<4, true>)
    ModPD<kPdDigits> pd;         // the conversions' constants (generic carries; same fields for fast ones)
    const uint32_t* pd_pw;       // digits of 2^(32j) mod p^4, j < 4 (the plan's constant table)
};

// How R-multiplications are computed.
enum : int {
    kFormDirect = 0,   // negacyclic convolution on the integer pipe (26-bit limbs)
    kFormNtt = 1,      // through the evaluation map of R (ntt_rmul.cuh)
    kFormI8 = 2        // as INT8 tensor-core products (i8_rmul.cuh)
};

// Per-warp shared words of an INT8 R-multiplication: x and E in 26-bit
// limbs, then the byte planes and diagonal sums of i8_rmul.cuh.  Rounded up
// to 4 words so that every warp's buffer starts 16-byte aligned (residues of
// 4 limbs are stored with 16-byte vector accesses).
template <int m, int LR>
__host__ __device__ constexpr int i8_warp_words(int S) {
    return (3 * m * LR + i8_warp_bytes<m>(S) / 4 + 3) & ~3;
}

__device__ __forceinline__ uint32_t bitrev(uint32_t x, int bits) { return __brev(x) >> (32 - bits); }

template <int n>
__device__ __forceinline__ constexpr int ilog2() {
    int r = 0;
    int v = n;
    while (v > 1) { v >>= 1; ++r; }
    return r;
}

// u bits of the operand starting at bit pos (bits at or above n_bits read as 0).
__device__ __forceinline__ uint32_t get_field(const uint64_t* raw, uint64_t raw_words, uint64_t n_bits, uint64_t pos,
                                              uint32_t u) {
    if (pos >= n_bits) return 0;
    uint64_t w = pos >> 6;
    uint32_t off = (uint32_t)(pos & 63);
    uint64_t v = raw[w] >> off;
    if (off + u > 64 && w + 1 < raw_words) v |= raw[w + 1] << (64 - off);
    uint64_t avail = n_bits - pos;
    uint32_t width = avail < u ? (uint32_t)avail : u;
    return (uint32_t)(v & ((width == 64 ? ~0ull : ((1ull << width) - 1))));
}

// Team-local view: which lanes of which warp serve which element.
template <int m, int L>
struct Team {
    int id;         // team index in the CTA
    int lane;       // lane within the team
    unsigned mask;  // lanes of this team in its warp (for __syncwarp)
    __device__ __forceinline__ Team() {
        using G = Geo<m, L>;
        int warp = threadIdx.x >> 5;
        int l = threadIdx.x & 31;
        id = warp * G::TEAMS_PER_WARP + l / G::TEAM;
        lane = l % G::TEAM;
        mask = G::TEAM == 32 ? 0xffffffffu : (((1u << G::TEAM) - 1u) << (l / G::TEAM * G::TEAM));
    }
};

// Team of the NTT-form R-multiplication (ntt_rmul.cuh): m/4 lanes per element.
template <int m>
struct NttTeam {
    static constexpr int TEAM = m / 4;
    static constexpr int TEAMS_PER_WARP = 32 / TEAM;
    static constexpr int NTEAMS = kWarps * TEAMS_PER_WARP;
    static constexpr int BUF_WORDS_PER_LR = m;   // exchange buffer: m residues
    int id, lane;
    unsigned mask;
    __device__ __forceinline__ NttTeam() {
        const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
        id = warp * TEAMS_PER_WARP + l / TEAM;
        lane = l % TEAM;
        mask = TEAM == 32 ? 0xffffffffu : (((1u << TEAM) - 1u) << (l / TEAM * TEAM));
    }
};

// Blocks of the last level (n elements each) per CTA of the NTT-form fused
// kernel: enough that every team of the CTA owns an element.
template <int m>
__host__ __device__ constexpr int final_blocks_per_cta(int n) {
    return n >= NttTeam<m>::NTEAMS ? 1 : NttTeam<m>::NTEAMS / n;
}

// Coefficient t of alpha^sh * y (sh in [0, 2m)): +-y[src] (negacyclic shift).
template <int m, int L>
__device__ __forceinline__ void shifted(uint32_t (&out)[L], bool& neg, const uint32_t* y, int t, int sh) {
    int src = t - sh;
    neg = false;
    if (src < 0) {
        src += m;
        neg = true;
        if (src < 0) {
            src += m;
            neg = false;
        }
    }
    ld_res<L>(out, y + src * L);
}

// In-place radix-2 DIT over n elements held in shared memory in bit-reversed
// slots, for `arrays` consecutive arrays of n elements transformed together;
// leaves X_v = sum_j x_j (alpha^root)^(j v) in slot v.  root is a shift
// amount in [0, 2m).  Butterflies are spread over teams; a team owns whole
// butterflies, so one __syncwarp separates its reads from its writes.
template <int m, int L>
__device__ void dft_dit(uint32_t* base, int arrays, int n, int root, const Mod<L>& md) {
    using G = Geo<m, L>;
    Team<m, L> tm;
    const int log2n = 31 - __clz(n);
    for (int lh = 0; lh < log2n; ++lh) {          // half = 2^lh (powers of two: shifts, no division)
        const int half = 1 << lh;
        const int scale = n >> (lh + 1);
        for (int bfa = tm.id; bfa < arrays * (n / 2); bfa += G::NTEAMS) {
            uint32_t* s = base + (bfa >> (log2n - 1)) * n * G::ES;
            int bf = bfa & (n / 2 - 1);
            int k_in = bf & (half - 1);
            int ia = ((bf >> lh) << (lh + 1)) + k_in;
            int ib = ia + half;
            int sh = (root * scale * k_in) & (G::TWO_M - 1);
            uint32_t* pa = s + ia * G::ES;
            uint32_t* pb = s + ib * G::ES;
            uint32_t a[G::CPL][L], y[G::CPL][L];
            bool ng[G::CPL];
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                ld_res<L>(a[c], pa + t * L);
                shifted<m, L>(y[c], ng[c], pb, t, sh);
            }
            __syncwarp(tm.mask);
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                // a + y and a - y; where the shifted coefficient carries a minus
                // sign the two results trade places (the store addresses swap)
                uint32_t pl[L], mi[L];
                add_mod<L>(pl, a[c], y[c], md);
                sub_mod<L>(mi, a[c], y[c], md);
                uint32_t* d0 = (ng[c] ? pb : pa) + t * L;
                uint32_t* d1 = (ng[c] ? pa : pb) + t * L;
                st_res<L>(d0, pl);
                st_res<L>(d1, mi);
            }
            __syncwarp(tm.mask);
        }
        __syncthreads();
    }
}

// In-place radix-2 DIF over n elements in natural slots, for `arrays`
// consecutive arrays of n elements; leaves X_v = sum_j x_j (alpha^root)^(j v)
// in slot bitrev(v).
template <int m, int L>
__device__ void dft_dif(uint32_t* base, int arrays, int n, int root, const Mod<L>& md) {
    using G = Geo<m, L>;
    Team<m, L> tm;
    const int log2n = 31 - __clz(n);
    for (int lh = log2n - 1; lh >= 0; --lh) {     // half = 2^lh
        const int half = 1 << lh;
        const int scale = n >> (lh + 1);
        for (int bfa = tm.id; bfa < arrays * (n / 2); bfa += G::NTEAMS) {
            uint32_t* s = base + (bfa >> (log2n - 1)) * n * G::ES;
            const int bf = bfa & (n / 2 - 1);
            int k_in = bf & (half - 1);
            int ia = ((bf >> lh) << (lh + 1)) + k_in;
            int ib = ia + half;
            int sh = (root * scale * k_in) & (G::TWO_M - 1);
            uint32_t sa[G::CPL][L], db[G::CPL][L];
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                uint32_t a[L], b[L];
                ld_res<L>(a, s + ia * G::ES + t * L);
                ld_res<L>(b, s + ib * G::ES + t * L);
                add_mod<L>(sa[c], a, b, md);
                // coefficient t of alpha^sh * (a - b)
                int src = t - sh;
                bool neg = false;
                if (src < 0) {
                    src += m;
                    neg = true;
                    if (src < 0) {
                        src += m;
                        neg = false;
                    }
                }
                // b - a instead of a - b where the coefficient carries a minus sign
                const uint32_t* pa = s + (neg ? ib : ia) * G::ES + src * L;
                const uint32_t* pb = s + (neg ? ia : ib) * G::ES + src * L;
                ld_res<L>(a, pa);
                ld_res<L>(b, pb);
                sub_mod<L>(db[c], a, b, md);
            }
            __syncwarp(tm.mask);
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                st_res<L>(s + ia * G::ES + t * L, sa[c]);
                st_res<L>(s + ib * G::ES + t * L, db[c]);
            }
            __syncwarp(tm.mask);
        }
        __syncthreads();
    }
}

// Negacyclic product in R (Section 2.9.2, eq. ncycconv) times alpha^r, in
// 26-bit limbs: out_k = REDC(sum_i x_i E[(k - r - i) mod 2m]) where
// E[t] = y_t and E[t+m] = -y_t, so that the wrapped terms carry their minus
// sign.  X and E are the team's shared buffers.  Lane l computes the two
// consecutive outputs k = 2l and 2l+1: the factor E[k - r - i] used for
// output k at step i is the one output k+1 needs at step i+1, so each step
// loads one x_i (broadcast) and one E value for two outputs.
template <int m, int LR>
__device__ __forceinline__ void negacyclic_mul_rr(uint32_t (&out)[2][LR], const uint32_t* X, const uint32_t* E, int r,
                                                  const ModRR<LR>& md, int lane) {
    const int k0 = 2 * lane;
    uint64_t c0[2 * LR], c1[2 * LR];
#pragma unroll
    for (int i = 0; i < 2 * LR; ++i) c0[i] = c1[i] = 0;
    uint32_t prev[LR];
    ld_rr<LR>(prev, E + ((k0 + 1 - r) & (2 * m - 1)) * LR);
#pragma unroll 4
    for (int i = 0; i < m; ++i) {
        uint32_t xi[LR], cur[LR];
        ld_rr<LR>(xi, X + i * LR);
        ld_rr<LR>(cur, E + ((k0 - r - i) & (2 * m - 1)) * LR);
        mac_cols<LR>(c0, xi, cur);
        mac_cols<LR>(c1, xi, prev);
#pragma unroll
        for (int w = 0; w < LR; ++w) prev[w] = cur[w];
    }
    redc_cols<LR>(out[0], c0, md);
    redc_cols<LR>(out[1], c1, md);
}

// Stage element x (radix-2^32 residues, L words) into X as 26-bit limbs.
template <int m, int L, int LR>
__device__ __forceinline__ void stage_x_rr(uint32_t* X, const uint32_t* x, int lane) {
    constexpr int CPL = Geo<m, L>::CPL, TEAM = Geo<m, L>::TEAM;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int t = lane + c * TEAM;
        uint32_t v[L], w[LR];
        ld_res<L>(v, x + t * L);
        to_rr<L, LR>(w, v);
        st_rr<LR>(X + t * LR, w);
    }
}

// Stage E from a factor already in 26-bit limbs (the rho^s table).
template <int m, int LR>
__device__ __forceinline__ void stage_ext_rr(uint32_t* E, const uint32_t* y, const ModRR<LR>& md, int lane) {
    constexpr int CPL = Geo<m, 1>::CPL, TEAM = Geo<m, 1>::TEAM;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int t = lane + c * TEAM;
        uint32_t v[LR], nv[LR];
#pragma unroll
        for (int i = 0; i < LR; ++i) v[i] = y[t * LR + i];
        neg_rr<LR>(nv, v, md);
        st_rr<LR>(E + t * LR, v);
        st_rr<LR>(E + (t + m) * LR, nv);
    }
}

// Stage E from a factor in radix-2^32 residues (a transformed operand).
template <int m, int L, int LR>
__device__ __forceinline__ void stage_ext_from32(uint32_t* E, const uint32_t* y, const ModRR<LR>& md, int lane) {
    constexpr int CPL = Geo<m, L>::CPL, TEAM = Geo<m, L>::TEAM;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int t = lane + c * TEAM;
        uint32_t v32[L], v[LR], nv[LR];
        ld_res<L>(v32, y + t * L);
        to_rr<L, LR>(v, v32);
        neg_rr<LR>(nv, v, md);
        st_rr<LR>(E + t * LR, v);
        st_rr<LR>(E + (t + m) * LR, nv);
    }
}

// Warp-owned staging (one warp per element, INT8 form): x from radix-2^32
// residues; E = (y, -y) from 26-bit limbs (the coefficient table) or from
// radix-2^32 residues (a transformed operand).
template <int m, int L, int LR>
__device__ __forceinline__ void i8_stage_x_from32(uint32_t* X, const uint32_t* x, int lane) {
    for (int t = lane; t < m; t += 32) {
        uint32_t v[L], w[LR];
        ld_res<L>(v, x + t * L);
        to_rr<L, LR>(w, v);
        st_rr<LR>(X + t * LR, w);
    }
}

template <int m, int LR>
__device__ __forceinline__ void i8_stage_ext_rr(uint32_t* E, const uint32_t* y, const ModRR<LR>& md, int lane) {
    for (int t = lane; t < m; t += 32) {
        uint32_t v[LR], nv[LR];
#pragma unroll
        for (int i = 0; i < LR; ++i) v[i] = y[t * LR + i];
        neg_rr<LR>(nv, v, md);
        st_rr<LR>(E + t * LR, v);
        st_rr<LR>(E + (t + m) * LR, nv);
    }
}

template <int m, int L, int LR>
__device__ __forceinline__ void i8_stage_ext_from32(uint32_t* E, const uint32_t* y, const ModRR<LR>& md, int lane) {
    for (int t = lane; t < m; t += 32) {
        uint32_t v32[L], v[LR], nv[LR];
        ld_res<L>(v32, y + t * L);
        to_rr<L, LR>(v, v32);
        neg_rr<LR>(nv, v, md);
        st_rr<LR>(E + t * LR, v);
        st_rr<LR>(E + (t + m) * LR, nv);
    }
}

// ---------------------------------------------------------------------------
// Forward level d, step i.: the 2m-point inner DFT of one column with root
// alpha (shifts and additions only), in shared memory.  Grid: x = column
// (2M/2m of them), y = operand (0: a, 1: b).  The first level reads the
// operand words and encodes them (Section 3.2.4) on the fly.
// ---------------------------------------------------------------------------
template <int m, int L, bool FIRST>
__device__ __forceinline__ void column_load_fwd(const LevelParams& prm, uint32_t* col, uint64_t column, int op) {
    using G = Geo<m, L>;
    constexpr int LOG2_TWO_M = ilog2<G::TWO_M>();
    uint32_t* poly = prm.data + (op ? prm.poly_words : 0);
    const int lg_mu = (__ffsll((long long)prm.len) - 1) - LOG2_TWO_M;
    const uint64_t mu_d = 1ull << lg_mu;
    const uint64_t blk = column >> lg_mu, l = column & (mu_d - 1);
    const uint64_t base = blk * prm.len;
    // element j of the column sits at base + j*mu_d + l; load it into slot bitrev(j)
    if constexpr (FIRST) {
        const uint64_t* raw = op ? prm.raw_b : prm.raw_a;
        const int h = m / 2;
        for (int idx = threadIdx.x; idx < G::TWO_M * m; idx += kThreads) {
            int j = idx / m, t = idx % m;
            uint64_t i = (uint64_t)j * mu_d + l;        // outer coefficient index
            uint32_t v = 0;
            if (i < prm.M && t < h) v = get_field(raw, prm.raw_words, prm.n_bits, (uint64_t)prm.u * (i * h + t), prm.u);
            uint32_t* dst = col + bitrev(j, LOG2_TWO_M) * G::ES + t * L;
            dst[0] = v;
#pragma unroll
            for (int w = 1; w < L; ++w) dst[w] = 0;
        }
    } else {
        for (int idx = threadIdx.x; idx < G::TWO_M * m; idx += kThreads) {
            int j = idx / m, t = idx % m;
            uint32_t x[L];
            ld_res<L>(x, poly + ((base + (uint64_t)j * mu_d + l) * m + t) * L);
            st_res<L>(col + bitrev(j, LOG2_TWO_M) * G::ES + t * L, x);
        }
    }
}

template <int m, int L, bool FIRST>
__device__ __forceinline__ void dft_fwd_column(const LevelParams& prm, const Mod<L>& md, uint32_t* col, uint64_t column,
                                               int op) {
    using G = Geo<m, L>;
    uint32_t* poly = prm.data + (op ? prm.poly_words : 0);
    const int lg_mu = (__ffsll((long long)prm.len) - 1) - ilog2<G::TWO_M>();
    const uint64_t mu_d = 1ull << lg_mu;
    const uint64_t blk = column >> lg_mu, l = column & (mu_d - 1);
    const uint64_t base = blk * prm.len;
    column_load_fwd<m, L, FIRST>(prm, col, column, op);
    __syncthreads();
    dft_dit<m, L>(col, 1, G::TWO_M, 1, md);
    for (int idx = threadIdx.x; idx < G::TWO_M * m; idx += kThreads) {
        int v = idx / m, t = idx % m;
        uint32_t x[L];
        ld_res<L>(x, col + v * G::ES + t * L);
        st_res<L>(poly + ((base + (uint64_t)v * mu_d + l) * m + t) * L, x);
    }
}

template <int m, int L, bool FIRST>
__global__ void __launch_bounds__(kThreads) k_dft_fwd(LevelParams prm, Mod<L> md) {
    extern __shared__ __align__(16) uint32_t smem[];
    dft_fwd_column<m, L, FIRST>(prm, md, smem, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Bad multiplications of level d (Section 3.2.5 ii.): element (v, l) of every
// block times rho^(+-v l bp) = alpha^r rho^s, in place.  Element-parallel: one
// team per element, only the (2m-1)(mu_d-1) elements per block whose twiddle
// is not 1.  Grid: x = element groups, y = operand.
// ---------------------------------------------------------------------------
template <int m, int L, int LR, bool INV>
__global__ void __launch_bounds__(kThreads) k_twiddle(LevelParams prm, ModRR<LR> mr) {
    using G = Geo<m, L>;
    extern __shared__ __align__(16) uint32_t smem[];
    Team<m, L> tm;
    uint32_t* X = smem + tm.id * TeamBuf<m, LR>::WORDS;
    uint32_t* E = X + m * LR;
    uint32_t* poly = prm.data + (blockIdx.y ? prm.poly_words : 0);
    const uint64_t mu_d = prm.len / G::TWO_M;
    const uint64_t per_blk = (uint64_t)(G::TWO_M - 1) * (mu_d - 1);
    const uint64_t total = per_blk * (prm.P2 / prm.len);
    const uint64_t idx = (uint64_t)blockIdx.x * G::NTEAMS + tm.id;
    if (idx >= total) return;
    const uint64_t blk = idx / per_blk, rem = idx % per_blk;
    const uint64_t v = 1 + rem / (mu_d - 1), l = 1 + rem % (mu_d - 1);
    uint64_t e = v * l * prm.bp;                          // in (0, 2M)
    if (INV) e = prm.P2 - e;
    const int r = (int)(e >> prm.log2_mu_top);
    const uint64_t sidx = e & (prm.mu_top - 1);
    uint32_t* x = poly + (blk * prm.len + v * mu_d + l) * G::EW;
    stage_x_rr<m, L, LR>(X, x, tm.lane);
    stage_ext_rr<m, LR>(E, prm.table + sidx * m * LR, mr, tm.lane);
    __syncwarp(tm.mask);
    uint32_t out[2][LR];
    negacyclic_mul_rr<m, LR>(out, X, E, r, mr, tm.lane);
    uint32_t o32[2][L];
    from_rr<L, LR>(o32[0], out[0]);
    from_rr<L, LR>(o32[1], out[1]);
    st_res<L>(x + (2 * tm.lane) * L, o32[0]);
    st_res<L>(x + (2 * tm.lane + 1) * L, o32[1]);
}

// Coefficients l and l + m/2 of alpha^r x (x: m residues of L words) in
// 26-bit limbs: coefficient t of alpha^r x is +-x[(t - r) mod m]; a negated
// one is the lazy bias(K p^z) - x (ntt_rmul.cuh).
template <int m, int L, int LR>
__device__ __forceinline__ void load_shifted_rr(uint32_t (&out)[LR], const uint32_t* x, int t, int r,
                                                const uint32_t (&bn)[LR]) {
    int src = t - r;
    bool neg = false;
    if (src < 0) {
        src += m;
        neg = true;
        if (src < 0) {
            src += m;
            neg = false;
        }
    }
    uint32_t v[L], y[LR];
    ld_res<L>(v, x + src * L);
    to_rr<L, LR>(y, v);
#pragma unroll
    for (int i = 0; i < LR; ++i) out[i] = neg ? bn[i] - y[i] : y[i];
}

// ---------------------------------------------------------------------------
// Bad multiplications of level d through the evaluation map of R
// (ntt_rmul.cuh): same element set as k_twiddle, one team of m/4 lanes per
// element, xbuf = the CTA's exchange buffers (NttTeam<m>::NTEAMS of m
// residues of LR words).
// ---------------------------------------------------------------------------
template <int m, int L, int LR, bool INV, class MR>
__device__ __forceinline__ void twiddle_ntt_group(const LevelParams& prm, const MR& mr, uint64_t group, int op,
                                                  uint32_t* xbuf) {
    using G = Geo<m, L>;
    using NT = NttTeam<m>;
    NT tm;
    uint32_t* poly = prm.data + (op ? prm.poly_words : 0);
    // element (blk, v, l) of the level, all P2 of them (len, mu_d powers of two:
    // shifts, no division); the twiddle of v = 0 or l = 0 is 1
    const int lg_len = __ffsll((long long)prm.len) - 1;
    const int lg_mu = lg_len - ilog2<G::TWO_M>();
    const uint64_t idx = group * NT::NTEAMS + tm.id;
    if (idx >= prm.P2) return;
    const uint64_t blk = idx >> lg_len, rem = idx & (prm.len - 1);
    const uint64_t v = rem >> lg_mu, l = rem & ((1ull << lg_mu) - 1);
    if (v == 0 || l == 0) return;
    const uint64_t mu_d = 1ull << lg_mu;
    uint64_t e = v * l * prm.bp;                          // in (0, 2M)
    if (INV) e = prm.P2 - e;
    const int r = (int)(e >> prm.log2_mu_top);
    const uint64_t sidx = e & (prm.mu_top - 1);
    uint32_t* x = poly + (blk * prm.len + v * mu_d + l) * G::EW;
    uint32_t* buf = xbuf + tm.id * m * LR;
    const int lane = tm.lane;
    uint32_t bn[LR];
    ldg_rr<LR>(bn, prm.ntt_cst + NttLayout<m>::BN * LR);
    uint32_t vv[4][LR];
#pragma unroll
    for (int j = 0; j < 4; ++j) load_shifted_rr<m, L, LR>(vv[j], x, lane + j * NT::TEAM, r, bn);
    ntt_forward<m, LR>(vv, buf, lane, tm.mask, prm.ntt_cst, mr);
    const uint32_t* tw = prm.table_eval + (sidx * m + 4 * lane) * LR;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t t[LR];
        ldg_rr<LR>(t, tw + j * LR);
        mmul<LR>(vv[j], vv[j], t, mr);
    }
    // the table carries m^-1: the last stage multiplies only by psi^-1 and
    // slots 0 and 1 are reduced without a product
    ntt_backward<m, LR, true>(vv, buf, lane, tm.mask, prm.ntt_cst, 0, NttLayout<m>::ZLAST, mr);
    __syncwarp(tm.mask);   // every lane has read its shifted inputs before any write
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t c[LR], o[L];
        if (j < 2) reduce_raw<LR>(c, vv[j], mr);
        else canon<LR>(c, vv[j], mr);
        from_rr<L, LR>(o, c);
        st_res<L>(x + (lane + j * NT::TEAM) * L, o);
    }
}

// Coefficient t of alpha^r x in p-adic digits (padic.cuh): x's residue
// converted from its L words (pw: digits of 2^(32j) mod p^z), a negated one
// as the bias bn - y (bn = (p, p-1, ..., p-1), y canonical).
template <int m, int L, int Z, bool F>
__device__ __forceinline__ void load_shifted_pd(uint32_t (&out)[Z], const uint32_t* x, int t, int r,
                                                const uint32_t (&bn)[Z], const uint32_t* pw, const ModPD<Z, F>& md) {
    int src = t - r;
    bool neg = false;
    if (src < 0) {
        src += m;
        neg = true;
        if (src < 0) {
            src += m;
            neg = false;
        }
    }
    uint32_t v[L], y[Z];
    ld_res<L>(v, x + src * L);
    // 4-word residues: p^4 >= 2^95, so p > 2^23 and the short conversion applies
    if constexpr (L == 4 && Z == 4) pd_from_words4_large_p(y, v, pw, md);
    else pd_from_words<L, Z>(y, v, pw, md);
#pragma unroll
    for (int i = 0; i < Z; ++i) out[i] = neg ? bn[i] - y[i] : y[i];
}

// The same coefficient where the residues in HBM already are canonical digits.
template <int m, int Z>
__device__ __forceinline__ void load_shifted_digits(uint32_t (&out)[Z], const uint32_t* x, int t, int r,
                                                    const uint32_t (&bn)[Z]) {
    int src = t - r;
    bool neg = false;
    if (src < 0) {
        src += m;
        neg = true;
        if (src < 0) {
            src += m;
            neg = false;
        }
    }
    uint32_t y[Z];
    ld_res<Z>(y, x + src * Z);
#pragma unroll
    for (int i = 0; i < Z; ++i) out[i] = neg ? bn[i] - y[i] : y[i];
}

// The bad multiplications of twiddle_ntt_group with the transform in R in
// p-adic digits: the element's residues are converted on load and back on
// store, the twiddle table and the transform constants hold digits.
template <int m, int L, bool INV, int Z, bool F>
__device__ __forceinline__ void twiddle_pd_group(const LevelParams& prm, const ModPD<Z, F>& md, uint64_t group, int op,
                                                 uint32_t* xbuf) {
    using G = Geo<m, L>;
    using NT = NttTeam<m>;
    NT tm;
    uint32_t* poly = prm.data + (op ? prm.poly_words : 0);
    const int lg_len = __ffsll((long long)prm.len) - 1;
    const int lg_mu = lg_len - ilog2<G::TWO_M>();
    const uint64_t idx = group * NT::NTEAMS + tm.id;
    if (idx >= prm.P2) return;
    const uint64_t blk = idx >> lg_len, rem = idx & (prm.len - 1);
    const uint64_t v = rem >> lg_mu, l = rem & ((1ull << lg_mu) - 1);
    if (v == 0 || l == 0) return;
    const uint64_t mu_d = 1ull << lg_mu;
    uint64_t e = v * l * prm.bp;
    if (INV) e = prm.P2 - e;
    const int r = (int)(e >> prm.log2_mu_top);
    const uint64_t sidx = e & (prm.mu_top - 1);
    uint32_t* x = poly + (blk * prm.len + v * mu_d + l) * G::EW;
    uint32_t* buf = xbuf + tm.id * m * Z;
    const int lane = tm.lane;
    const uint32_t* cst = prm.ntt_cst;
    uint32_t bn[Z];
    ldg_rr<Z>(bn, cst + NttLayout<m>::BN * Z);
    const uint32_t* pw = cst + PdLayout<m>::POW32 * Z;
    // forward levels with digits in HBM (L = Z words): no conversions at either edge
    bool dio = false;
    if constexpr (!INV && L == Z) dio = prm.pd_io != 0;
    uint32_t vv[4][Z];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (dio) load_shifted_digits<m, Z>(vv[j], x, lane + j * NT::TEAM, r, bn);
        else load_shifted_pd<m, L, Z>(vv[j], x, lane + j * NT::TEAM, r, bn, pw, md);
    }
    ntt_forward_pd<m, Z>(vv, buf, lane, tm.mask, cst, md);
    const uint32_t* tw = prm.table_eval + (sidx * m + 4 * lane) * Z;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t t[Z];
        ldg_rr<Z>(t, tw + j * Z);
        mmul<Z>(vv[j], vv[j], t, md);
    }
    // the table carries m^-1: the last stage multiplies only by psi^-1
    ntt_backward_pd<m, Z, true>(vv, buf, lane, tm.mask, cst, 0, NttLayout<m>::ZLAST, md);
    __syncwarp(tm.mask);   // every lane has read its shifted inputs before any write
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t c[Z], o[L];
        if (j < 2) pd_canon<Z>(c, vv[j], md);
        else {
#pragma unroll
            for (int w = 0; w < Z; ++w) c[w] = vv[j][w];
        }
        if constexpr (L == Z) {
            if (dio) {
                st_res<L>(x + (lane + j * NT::TEAM) * L, c);
                continue;
            }
        }
        pd_to_words<L, Z>(o, c, md);
        st_res<L>(x + (lane + j * NT::TEAM) * L, o);
    }
}

template <int m, int L, int LR, bool INV, class MR = ModRR<LR>>
__global__ void __launch_bounds__(kThreads, (LR >= 5 || m >= 64) ? 3 : 4) k_twiddle_ntt(LevelParams prm, MR mr) {
    extern __shared__ __align__(16) uint32_t smem[];
    if constexpr (IsPD<MR>::value)
        twiddle_pd_group<m, L, INV, LR>(prm, mr, blockIdx.x, blockIdx.y, smem);
    else
        twiddle_ntt_group<m, L, LR, INV, MR>(prm, mr, blockIdx.x, blockIdx.y, smem);
}

// ---------------------------------------------------------------------------
// A radix-2m level fused with its bad multiplications (NTT form), one CTA per
// column: forward, the column's inner DFT (integer ALU) and then the
// R-multiplications of its 2m outputs (multiply pipe); backwards, the
// R-multiplications of the column's inputs and then its inner DFT.  Several
// CTAs per SM sit in different phases, so the two pipes overlap, and each
// level reads and writes the polynomial once.  smem: the column (2m elements)
// and the teams' exchange buffers.
// ---------------------------------------------------------------------------
template <int m, int L, int LR, class MR>
__device__ __forceinline__ void level_rmul_element(const LevelParams& prm, const MR& mr, const uint32_t* src,
                                                   uint32_t* dst, uint64_t e, uint32_t* buf, int lane, unsigned mask,
                                                   const uint32_t (&bn)[LR]) {
    using NT = NttTeam<m>;
    const int r = (int)(e >> prm.log2_mu_top);
    const uint64_t sidx = e & (prm.mu_top - 1);
    uint32_t vv[4][LR];
#pragma unroll
    for (int j = 0; j < 4; ++j) load_shifted_rr<m, L, LR>(vv[j], src, lane + j * NT::TEAM, r, bn);
    ntt_forward<m, LR>(vv, buf, lane, mask, prm.ntt_cst, mr);
    const uint32_t* tw = prm.table_eval + (sidx * m + 4 * lane) * LR;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t t[LR];
        ldg_rr<LR>(t, tw + j * LR);
        mmul<LR>(vv[j], vv[j], t, mr);
    }
    // the table carries m^-1: the last stage multiplies only by psi^-1 and
    // slots 0 and 1 are reduced without a product
    ntt_backward<m, LR, true>(vv, buf, lane, mask, prm.ntt_cst, 0, NttLayout<m>::ZLAST, mr);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t c[LR], o[L];
        if (j < 2) reduce_raw<LR>(c, vv[j], mr);
        else canon<LR>(c, vv[j], mr);
        from_rr<L, LR>(o, c);
        st_res<L>(dst + (lane + j * NT::TEAM) * L, o);
    }
}

template <int m, int L, int LR, bool FIRST, class MR>
__device__ __forceinline__ void level_fwd_ntt(const LevelParams& prm, const Mod<L>& md, const MR& mr,
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
    column_load_fwd<m, L, FIRST>(prm, col, column, op);
    __syncthreads();
    dft_dit<m, L>(col, 1, G::TWO_M, 1, md);     // ends with __syncthreads: output v in slot v
    NT nt;
    uint32_t* buf = xbuf + nt.id * m * LR;
    uint32_t bn[LR];
    ldg_rr<LR>(bn, prm.ntt_cst + NttLayout<m>::BN * LR);
    for (int v = nt.id; v < G::TWO_M; v += NT::NTEAMS) {
        const uint32_t* src = col + v * G::ES;
        uint32_t* dst = poly + (base + (uint64_t)v * mu_d + l) * G::EW;
        if (v == 0 || l == 0) {                  // twiddle 1
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t x[L];
                ld_res<L>(x, src + (nt.lane + j * NT::TEAM) * L);
                st_res<L>(dst + (nt.lane + j * NT::TEAM) * L, x);
            }
            continue;
        }
        level_rmul_element<m, L, LR, MR>(prm, mr, src, dst, (uint64_t)v * l * prm.bp, buf, nt.lane, nt.mask, bn);
    }
}

template <int m, int L, int LR, bool FIRST, class MR = ModRR<LR>>
__global__ void __launch_bounds__(kThreads, m >= 64 ? 1 : 4)
    k_level_fwd_ntt(LevelParams prm, Mod<L> md, MR mr) {
    extern __shared__ __align__(16) uint32_t smem[];
    level_fwd_ntt<m, L, LR, FIRST, MR>(prm, md, mr, smem, blockIdx.x, blockIdx.y);
}

template <int m, int L, int LR, class MR>
__device__ __forceinline__ void level_inv_ntt(const LevelParams& prm, const Mod<L>& md, const MR& mr,
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
    uint32_t bn[LR];
    ldg_rr<LR>(bn, prm.ntt_cst + NttLayout<m>::BN * LR);
    // element v of the column times rho^(-v l bp), into slot v
    for (int v = nt.id; v < G::TWO_M; v += NT::NTEAMS) {
        const uint32_t* src = poly + (base + (uint64_t)v * mu_d + l) * G::EW;
        uint32_t* dst = col + v * G::ES;
        if (v == 0 || l == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t x[L];
                ld_res<L>(x, src + (nt.lane + j * NT::TEAM) * L);
                st_res<L>(dst + (nt.lane + j * NT::TEAM) * L, x);
            }
            continue;
        }
        level_rmul_element<m, L, LR, MR>(prm, mr, src, dst, prm.P2 - (uint64_t)v * l * prm.bp, buf, nt.lane, nt.mask,
                                     bn);
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

template <int m, int L, int LR, class MR = ModRR<LR>>
__global__ void __launch_bounds__(kThreads, m >= 64 ? 1 : 4)
    k_level_inv_ntt(LevelParams prm, Mod<L> md, MR mr) {
    extern __shared__ __align__(16) uint32_t smem[];
    level_inv_ntt<m, L, LR, MR>(prm, md, mr, smem, blockIdx.x);
}

template <int m, int L, int LR>
constexpr size_t level_ntt_smem_bytes() {
    return sizeof(uint32_t) * ((size_t)Geo<m, L>::TWO_M * Geo<m, L>::ES + (size_t)NttTeam<m>::NTEAMS * m * LR);
}

// dft_dit over residues held as p-adic digits (padic.cuh): sums digitwise,
// a difference adds 2 (p, p-1, ..., p-1) (zero mod p^z, digits at least those
// of a normalised residue), every stage normalises its outputs and the last
// makes them canonical; the plan's check (pd_lazy_bounds) keeps every digit
// below 2^32.  Inputs canonical digits.
template <int m, int Z, bool F>
__device__ void dft_dit_pd(uint32_t* base, int arrays, int n, int root, const ModPD<Z, F>& md) {
    using G = Geo<m, Z>;
    Team<m, Z> tm;
    const int log2n = 31 - __clz(n);
    uint32_t D2[Z];
#pragma unroll
    for (int k = 0; k < Z; ++k) D2[k] = 2 * (k == 0 ? md.p : md.p - 1);
    for (int lh = 0; lh < log2n; ++lh) {
        const int half = 1 << lh;
        const int scale = n >> (lh + 1);
        const bool last = lh + 1 == log2n;
        for (int bfa = tm.id; bfa < arrays * (n / 2); bfa += G::NTEAMS) {
            uint32_t* s = base + (bfa >> (log2n - 1)) * n * G::ES;
            int bf = bfa & (n / 2 - 1);
            int k_in = bf & (half - 1);
            int ia = ((bf >> lh) << (lh + 1)) + k_in;
            int ib = ia + half;
            int sh = (root * scale * k_in) & (G::TWO_M - 1);
            uint32_t* pa = s + ia * G::ES;
            uint32_t* pb = s + ib * G::ES;
            uint32_t a[G::CPL][Z], y[G::CPL][Z];
            bool ng[G::CPL];
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                ld_res<Z>(a[c], pa + t * Z);
                shifted<m, Z>(y[c], ng[c], pb, t, sh);
            }
            __syncwarp(tm.mask);
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                uint32_t pl[Z], mi[Z];
                lz_add<Z>(pl, a[c], y[c]);
                lz_sub<Z>(mi, a[c], D2, y[c]);
                if (last) {
                    pd_canon<Z>(pl, pl, md);
                    pd_canon<Z>(mi, mi, md);
                } else {
                    pd_norm<Z>(pl, md);
                    pd_norm<Z>(mi, md);
                }
                uint32_t* d0 = (ng[c] ? pb : pa) + t * Z;
                uint32_t* d1 = (ng[c] ? pa : pb) + t * Z;
                st_res<Z>(d0, pl);
                st_res<Z>(d1, mi);
            }
            __syncwarp(tm.mask);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Last level of both forward transforms, componentwise products scaled by
// (2M)^-1 (Section 3.2.6), and the first level of the backwards transform,
// fused.  One CTA per block of n = len contiguous elements (len <= 2m, root
// alpha^(2m/len)).  For a square the caller passes poly_words = 0 (b is a) and
// square = 1: the NTT form then reuses a's evaluations for both factors.
// ---------------------------------------------------------------------------
template <int m, int L, int LR, int FORM, class MR>
__device__ __forceinline__ void final_block(const LevelParams& prm, const Mod<L>& md, const MR& mr,
                                            uint32_t* smem, uint64_t block) {
    using G = Geo<m, L>;
    const int n = (int)prm.len;
    const int log2n = 31 - __clz(n);
    // the NTT form takes nb consecutive blocks per CTA so that every team has an element
    const int nb = FORM == kFormNtt ? final_blocks_per_cta<m>(n) : 1;
    const int nn = nb * n;
    uint32_t* sa = smem;
    uint32_t* sb = smem + nn * G::ES;
    uint32_t* tbuf = sb + nn * G::ES;
    const uint64_t base = block * nn;
    uint32_t* pa = prm.data;
    uint32_t* pb = prm.data + prm.poly_words;
    for (int idx = threadIdx.x; idx < nn * m; idx += kThreads) {
        int j = idx / m, t = idx % m;
        uint32_t x[L];
        int slot = ((j >> log2n) << log2n) + bitrev(j & (n - 1), log2n);
        ld_res<L>(x, pa + ((base + j) * m + t) * L);
        st_res<L>(sa + slot * G::ES + t * L, x);
        ld_res<L>(x, pb + ((base + j) * m + t) * L);
        st_res<L>(sb + slot * G::ES + t * L, x);
    }
    __syncthreads();
    const int root = G::TWO_M / n;
    // forward levels with digits in HBM: the last level's DFT on digits too
    bool pdio = false;
    if constexpr (FORM == kFormNtt && IsPD<MR>::value && L == LR) pdio = prm.pd_io != 0;
    if (pdio) {
        if constexpr (FORM == kFormNtt && IsPD<MR>::value && L == LR) dft_dit_pd<m, LR>(sa, 2 * nb, n, root, mr);
    } else {
        dft_dit<m, L>(sa, 2 * nb, n, root, md);
    }
    // componentwise products c_v = a_v * b_v * (2M)^-1
    Team<m, L> tm;
    if constexpr (FORM == kFormI8) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        uint32_t* X = tbuf + warp * i8_warp_words<m, LR>((int)prm.i8_S);
        uint32_t* E = X + m * LR;
        uint8_t* xb = reinterpret_cast<uint8_t*>(E + 2 * m * LR);
        uint8_t* fb = xb + ((prm.i8_S * m + 3) / 4) * 4;
        uint32_t* D = reinterpret_cast<uint32_t*>(fb + ((prm.i8_S * (2 * m + 4) + 3) / 4) * 4);
        uint32_t ks[LR];
#pragma unroll
        for (int w = 0; w < LR; ++w) ks[w] = prm.kscale[w];
        for (int v = warp; v < n; v += kWarps) {
            i8_stage_x_from32<m, L, LR>(X, sa + v * G::ES, lane);
            i8_stage_ext_from32<m, L, LR>(E, sb + v * G::ES, mr, lane);
            __syncwarp();
            i8_stage<m, LR>(xb, fb, (int)prm.i8_S, X, E, lane);
            __syncwarp();
            uint32_t out[m / 32][LR];
            i8_rmul_warp<m, LR>(out, xb, fb, D, (int)prm.i8_S, 0, mr, lane);
#pragma unroll
            for (int c = 0; c < m / 32; ++c) {
                uint32_t scaled[LR], o32[L];
                mont_mul_rr<LR>(scaled, out[c], ks, mr);
                from_rr<L, LR>(o32, scaled);
                st_res<L>(sa + v * G::ES + (lane + 32 * c) * L, o32);
            }
            __syncwarp();
        }
    } else if constexpr (FORM == kFormNtt && IsPD<MR>::value) {
        // the transform in R in p-adic digits (padic.cuh): per team an exchange
        // buffer, then b's canonical evaluations while a is transformed
        using NT = NttTeam<m>;
        NT nt;
        uint32_t* buf = tbuf + nt.id * 2 * m * LR;
        const int lane = nt.lane;
        uint32_t* park = buf + m * LR + nt.lane * LR;
        const uint32_t* cst = prm.ntt_cst;
        const uint32_t* pw = cst + PdLayout<m>::POW32 * LR;
#pragma unroll 1
        for (int v = nt.id; v < nn; v += NT::NTEAMS) {
            uint32_t x[4][LR], w[L];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ld_res<L>(w, sb + v * G::ES + (lane + j * NT::TEAM) * L);
                if (pdio) {
#pragma unroll
                    for (int k = 0; k < LR; ++k) x[j][k] = w[k < L ? k : 0];
                } else {
                    pd_from_words<L, LR>(x[j], w, pw, mr);
                }
            }
            ntt_forward_pd<m, LR>(x, buf, lane, nt.mask, cst, mr);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pd_canon<LR>(x[j], x[j], mr);
                st_rr<LR>(park + j * NT::TEAM * LR, x[j]);
            }
            // a square keeps a = b's evaluations in registers
            if (!prm.square) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    ld_res<L>(w, sa + v * G::ES + (lane + j * NT::TEAM) * L);
                    if (pdio) {
#pragma unroll
                        for (int k = 0; k < LR; ++k) x[j][k] = w[k < L ? k : 0];
                    } else {
                        pd_from_words<L, LR>(x[j], w, pw, mr);
                    }
                }
                ntt_forward_pd<m, LR>(x, buf, lane, nt.mask, cst, mr);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t y[LR];
                ld_rr<LR>(y, park + j * NT::TEAM * LR);
                mmul<LR>(x[j], x[j], y, mr);
            }
            ntt_backward_pd<m, LR>(x, buf, lane, nt.mask, cst, NttLayout<m>::PW_LO, NttLayout<m>::PW_HI, mr);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pd_to_words<L, LR>(w, x[j], mr);
                st_res<L>(sa + v * G::ES + (lane + j * NT::TEAM) * L, w);
            }
        }
    } else if constexpr (FORM == kFormNtt) {
        // per team: an exchange buffer, then a buffer holding b's evaluations
        // while a is transformed (one element in registers at a time)
        using NT = NttTeam<m>;
        NT nt;
        uint32_t* buf = tbuf + nt.id * 2 * m * LR;
        const int lane = nt.lane;
        // b's evaluations: residue j of the lane at park + j * TEAM * LR, or with
        // limb planes (3 or 5 limbs, m = 64) limb w at pbase + w * m + (j * TEAM + lane) ^ flip
        uint32_t* park = buf + m * LR + nt.lane * LR;
        uint32_t* pbase = buf + m * LR;
        constexpr bool PLANES = XchgPlanes<m, LR>::value;
#pragma unroll 1
        for (int v = nt.id; v < nn; v += NT::NTEAMS) {
            uint32_t x[4][LR], w[L];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ld_res<L>(w, sb + v * G::ES + (lane + j * NT::TEAM) * L);
                to_rr<L, LR>(x[j], w);
            }
            ntt_forward<m, LR>(x, buf, lane, nt.mask, prm.ntt_cst, mr);
            if (prm.ntt_prescale) {
                // scale b first so that the product of two lazy evaluations stays in range
                uint32_t c[LR];
                ldg_rr<LR>(c, prm.ntt_cst + NttLayout<m>::PW_LO * LR);
#pragma unroll
                for (int j = 0; j < 4; ++j) mmul<LR>(x[j], x[j], c, mr);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if constexpr (PLANES) {
#pragma unroll
                    for (int w = 0; w < LR; ++w) pbase[w * m + ((j * NT::TEAM + lane) ^ xteam_flip())] = x[j][w];
                } else {
                    st_rr<LR>(park + j * NT::TEAM * LR, x[j]);
                }
            }
            // a square keeps the unscaled evaluations of a = b in registers
            if (!prm.square || prm.ntt_prescale) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    ld_res<L>(w, sa + v * G::ES + (lane + j * NT::TEAM) * L);
                    to_rr<L, LR>(x[j], w);
                }
                ntt_forward<m, LR>(x, buf, lane, nt.mask, prm.ntt_cst, mr);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t y[LR];
                if constexpr (PLANES) {
#pragma unroll
                    for (int w = 0; w < LR; ++w) y[w] = pbase[w * m + ((j * NT::TEAM + lane) ^ xteam_flip())];
                } else {
                    ld_rr<LR>(y, park + j * NT::TEAM * LR);
                }
                mmul<LR>(x[j], x[j], y, mr);
            }
            if (prm.ntt_prescale)
                ntt_backward<m, LR>(x, buf, lane, nt.mask, prm.ntt_cst, NttLayout<m>::ONE, NttLayout<m>::ZLAST, mr);
            else
                ntt_backward<m, LR>(x, buf, lane, nt.mask, prm.ntt_cst, NttLayout<m>::PW_LO, NttLayout<m>::PW_HI, mr);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t c[LR];
                canon<LR>(c, x[j], mr);
                from_rr<L, LR>(w, c);
                st_res<L>(sa + v * G::ES + (lane + j * NT::TEAM) * L, w);
            }
        }
    } else {
        uint32_t* X = tbuf + tm.id * TeamBuf<m, LR>::WORDS;
        uint32_t* E = X + m * LR;
        uint32_t ks[LR];
#pragma unroll
        for (int w = 0; w < LR; ++w) ks[w] = prm.kscale[w];
        for (int v = tm.id; v < n; v += G::NTEAMS) {
            stage_x_rr<m, L, LR>(X, sa + v * G::ES, tm.lane);
            stage_ext_from32<m, L, LR>(E, sb + v * G::ES, mr, tm.lane);
            __syncwarp(tm.mask);
            uint32_t out[2][LR];
            negacyclic_mul_rr<m, LR>(out, X, E, 0, mr, tm.lane);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                uint32_t scaled[LR], o32[L];
                mont_mul_rr<LR>(scaled, out[c], ks, mr);
                from_rr<L, LR>(o32, scaled);
                st_res<L>(sa + v * G::ES + (2 * tm.lane + c) * L, o32);
            }
            __syncwarp(tm.mask);
        }
    }
    __syncthreads();
    // first backwards level: DFT with root alpha^(-2m/n), natural in, bit-reversed out
    dft_dif<m, L>(sa, nb, n, (G::TWO_M - root) % G::TWO_M, md);
    for (int idx = threadIdx.x; idx < nn * m; idx += kThreads) {
        int j = idx / m, t = idx % m;
        uint32_t x[L];
        const int slot = ((j >> log2n) << log2n) + bitrev(j & (n - 1), log2n);
        ld_res<L>(x, sa + slot * G::ES + t * L);
        st_res<L>(pa + ((base + j) * m + t) * L, x);
    }
}

template <int m, int L, int LR, int FORM, class MR = ModRR<LR>>
__global__ void __launch_bounds__(kThreads, FORM == kFormNtt ? ((LR >= 5 || IsPD<MR>::value) ? 2 : 3) : 1)
    k_final_pointwise(LevelParams prm, Mod<L> md, MR mr) {
    extern __shared__ __align__(16) uint32_t smem[];
    final_block<m, L, LR, FORM, MR>(prm, md, mr, smem, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Bad multiplications of level d as INT8 tensor-core products: one warp per
// element (same element set as k_twiddle), twiddles from the coefficient
// table.  Grid: x = groups of kWarps elements, y = operand.
// ---------------------------------------------------------------------------
template <int m, int L, int LR, bool INV>
__global__ void __launch_bounds__(kThreads) k_twiddle_i8(LevelParams prm, ModRR<LR> mr) {
    using G = Geo<m, L>;
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* X = smem + warp * i8_warp_words<m, LR>((int)prm.i8_S);
    uint32_t* E = X + m * LR;
    uint8_t* xb = reinterpret_cast<uint8_t*>(E + 2 * m * LR);
    uint8_t* fb = xb + ((prm.i8_S * m + 3) / 4) * 4;
    uint32_t* D = reinterpret_cast<uint32_t*>(fb + ((prm.i8_S * (2 * m + 4) + 3) / 4) * 4);
    uint32_t* poly = prm.data + (blockIdx.y ? prm.poly_words : 0);
    const uint64_t mu_d = prm.len / G::TWO_M;
    const uint64_t per_blk = (uint64_t)(G::TWO_M - 1) * (mu_d - 1);
    const uint64_t total = per_blk * (prm.P2 / prm.len);
    const uint64_t idx = (uint64_t)blockIdx.x * kWarps + warp;
    if (idx >= total) return;
    const uint64_t blk = idx / per_blk, rem = idx % per_blk;
    const uint64_t v = 1 + rem / (mu_d - 1), l = 1 + rem % (mu_d - 1);
    uint64_t e = v * l * prm.bp;
    if (INV) e = prm.P2 - e;
    const int r = (int)(e >> prm.log2_mu_top);
    const uint64_t sidx = e & (prm.mu_top - 1);
    uint32_t* x = poly + (blk * prm.len + v * mu_d + l) * G::EW;
    i8_stage_x_from32<m, L, LR>(X, x, lane);
    i8_stage_ext_rr<m, LR>(E, prm.table + sidx * m * LR, mr, lane);
    __syncwarp();
    i8_stage<m, LR>(xb, fb, (int)prm.i8_S, X, E, lane);
    __syncwarp();
    uint32_t out[m / 32][LR];
    i8_rmul_warp<m, LR>(out, xb, fb, D, (int)prm.i8_S, r, mr, lane);
#pragma unroll
    for (int c = 0; c < m / 32; ++c) {
        uint32_t o32[L];
        from_rr<L, LR>(o32, out[c]);
        st_res<L>(x + (lane + 32 * c) * L, o32);
    }
}

// ---------------------------------------------------------------------------
// Backwards level d, after its twiddles: the 2m-point DFT with root alpha^-1
// over each column (decimation in frequency: natural in, bit-reversed out),
// written back in natural element order.
// ---------------------------------------------------------------------------
template <int m, int L>
__device__ __forceinline__ void dft_inv_column(const LevelParams& prm, const Mod<L>& md, uint32_t* col, uint64_t column) {
    using G = Geo<m, L>;
    constexpr int LOG2_TWO_M = ilog2<G::TWO_M>();
    uint32_t* poly = prm.data;
    const uint64_t mu_d = prm.len / G::TWO_M;
    const uint64_t blk = column / mu_d, l = column % mu_d;
    const uint64_t base = blk * prm.len;
    for (int idx = threadIdx.x; idx < G::TWO_M * m; idx += kThreads) {
        int j = idx / m, t = idx % m;
        uint32_t x[L];
        ld_res<L>(x, poly + ((base + (uint64_t)j * mu_d + l) * m + t) * L);
        st_res<L>(col + j * G::ES + t * L, x);
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

template <int m, int L>
__global__ void __launch_bounds__(kThreads) k_dft_inv(LevelParams prm, Mod<L> md) {
    extern __shared__ __align__(16) uint32_t smem[];
    dft_inv_column<m, L>(prm, md, smem, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Column DFTs in halves, for columns too large for several CTAs per SM (m = 64:
// 2m elements of 64 residues of 3 or 4 words are 96 or 128 KiB).  The 2m-point
// DFT with root alpha^r splits into two m-point DFTs with root alpha^(2r):
// forward (decimation in time) over the even and the odd elements, then
// X_v = E_v + alpha^(r v) O_v and X_(v+m) = E_v - alpha^(r v) O_v; backwards
// (decimation in frequency) first s_k = x_k + x_(k+m) and
// d_k = alpha^(r k) (x_k - x_(k+m)), whose m-point DFTs give the even and the
// odd outputs.  One half sits in shared memory while the other waits in the
// CTA's slice of a plan-owned scratch buffer (m elements; L2-resident, since
// only the resident CTAs own slices), so a CTA needs m elements of shared
// memory and three or four CTAs fit per SM.  Persistent grid: CTA b owns
// scratch slice b and takes columns b, b + gridDim.x, ...
// ---------------------------------------------------------------------------
template <int m, int L>
__device__ __forceinline__ void copy_words_block(uint32_t* dst, const uint32_t* src, int words) {
    for (int i = 4 * threadIdx.x; i < words; i += 4 * kThreads)
        *reinterpret_cast<uint4*>(dst + i) = *reinterpret_cast<const uint4*>(src + i);
}

// Asynchronous 16-byte copies global -> shared (cp.async, L2 only): a thread
// issues all of its copies before it waits, so many loads are in flight
// without staging registers.
__device__ __forceinline__ void cp_async16(uint32_t* smem_dst, const uint32_t* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// n elements of EW words (a multiple of 4; 16-byte aligned in global and
// shared memory): element i from src(i) to dst + slot(i) * ES, in 16-byte
// pieces spread over the CTA; the caller synchronises the CTA afterwards.
template <int m, int L, class Src, class Slot>
__device__ __forceinline__ void cp_async_elements(uint32_t* dst, int n, Src src, Slot slot) {
    using G = Geo<m, L>;
    static_assert(G::EW % 4 == 0 && G::ES % 4 == 0, "elements move in 16-byte pieces");
    constexpr int PIECES = G::EW / 4;
    for (int idx = threadIdx.x; idx < n * PIECES; idx += kThreads) {
        const int i = idx / PIECES, pc = idx % PIECES;
        cp_async16(dst + slot(i) * G::ES + 4 * pc, src(i) + 4 * pc);
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// Lazy DFT arithmetic of the forward half-column kernel: residues stay
// unreduced L-word integers congruent mod q = p^z.  A sum is a plain carry
// chain; a difference at a stage whose inputs are below 2^s q is
// a - b + 2^s q (nonnegative), so both results stay below 2^(s+1) q.  The
// host enables this only where 2^7 q fits the L words (dft_lazy), and every
// value is reduced once when it is written back (lz32_reduce).
// ---------------------------------------------------------------------------
// The carries run in the condition-code chain (one asm block per chain, so
// nothing comes between its instructions): one instruction per word.
template <int L>
__device__ __forceinline__ void lz32_add(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L]) {
    static_assert(L == 3 || L == 4, "half-column kernels hold 3- or 4-word residues");
    if constexpr (L == 4) {
        asm("add.cc.u32 %0, %4, %8;\n\taddc.cc.u32 %1, %5, %9;\n\taddc.cc.u32 %2, %6, %10;\n\taddc.u32 %3, %7, %11;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]));
    } else {
        asm("add.cc.u32 %0, %3, %6;\n\taddc.cc.u32 %1, %4, %7;\n\taddc.u32 %2, %5, %8;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]));
    }
}

// r = a - b (no borrow out: a >= b as integers)
template <int L>
__device__ __forceinline__ void lz32_sub_n(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L]) {
    static_assert(L == 3 || L == 4, "half-column kernels hold 3- or 4-word residues");
    if constexpr (L == 4) {
        asm("sub.cc.u32 %0, %4, %8;\n\tsubc.cc.u32 %1, %5, %9;\n\tsubc.cc.u32 %2, %6, %10;\n\tsubc.u32 %3, %7, %11;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]));
    } else {
        asm("sub.cc.u32 %0, %3, %6;\n\tsubc.cc.u32 %1, %4, %7;\n\tsubc.u32 %2, %5, %8;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]));
    }
}

// r = a - b + B (B >= b as integers, the result below 2^(32L))
template <int L>
__device__ __forceinline__ void lz32_sub(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                                         const uint32_t (&B)[L]) {
    uint32_t t[L];
    lz32_sub_n<L>(t, B, b);
    lz32_add<L>(r, a, t);
}

// B = q 2^s (s <= 7, no overflow: checked on the host)
template <int L>
__device__ __forceinline__ void lz32_bias(uint32_t (&B)[L], const Mod<L>& md, int s) {
#pragma unroll
    for (int i = L - 1; i >= 0; --i)
        B[i] = s == 0 ? md.q[i] : (md.q[i] << s) | (i > 0 ? md.q[i - 1] >> (32 - s) : 0u);
}

// Canonical residue of x < 2^7 q: k = floor(x_top rcp / 2^40), rcp =
// floor(2^40 / (q_top + 1)), is floor(x / q) or up to two less (x_top and
// q_top the top words; q_top >= 2^8 on the host), so x - k q is below 3q and
// two conditional subtractions finish.
template <int L>
__device__ __forceinline__ void lz32_reduce(uint32_t (&r)[L], const uint32_t (&x)[L], const Mod<L>& md,
                                            uint32_t rcp) {
    const uint32_t k = (uint32_t)(((uint64_t)x[L - 1] * rcp) >> 40);
    uint32_t kq[L];
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        const uint64_t t = (uint64_t)k * md.q[i] + carry;
        kq[i] = (uint32_t)t;
        carry = t >> 32;
    }
    lz32_sub_n<L>(r, x, kq);
    // r below 3q: two conditional subtractions of q.  sub_mod(r, q) computes
    // r - q and adds q back where that borrows, i.e. r - q if r >= q, else r.
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        uint32_t d[L];
        sub_mod<L>(d, r, md.q, md);
#pragma unroll
        for (int i = 0; i < L; ++i) r[i] = d[i];
    }
}

// dft_dit with lazy arithmetic: the inputs below 2^s0 q, stage lh's below
// 2^(s0+lh) q; the outputs below 2^(s0+log2 n) q, unreduced.  With pd_in
// (L = 4) the inputs are canonical p-adic digits, converted to words as the
// first stage loads them (each residue once).
template <int m, int L>
__device__ void dft_dit_lazy(uint32_t* base, int n, int root, int s0, const Mod<L>& md, bool pd_in,
                             const ModPD<kPdDigits>& pd) {
    using G = Geo<m, L>;
    Team<m, L> tm;
    const int log2n = 31 - __clz(n);
    for (int lh = 0; lh < log2n; ++lh) {
        const int half = 1 << lh;
        const int scale = n >> (lh + 1);
        uint32_t B[L];
        lz32_bias<L>(B, md, s0 + lh);
        for (int bf = tm.id; bf < n / 2; bf += G::NTEAMS) {
            int k_in = bf & (half - 1);
            int ia = ((bf >> lh) << (lh + 1)) + k_in;
            int ib = ia + half;
            int sh = (root * scale * k_in) & (G::TWO_M - 1);
            uint32_t* pa = base + ia * G::ES;
            uint32_t* pb = base + ib * G::ES;
            uint32_t a[G::CPL][L], y[G::CPL][L];
            bool ng[G::CPL];
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                ld_res<L>(a[c], pa + t * L);
                shifted<m, L>(y[c], ng[c], pb, t, sh);
                if constexpr (L == kPdDigits) {
                    if (pd_in && lh == 0) {
                        uint32_t w[L];
                        pd_to_words<L, L>(w, a[c], pd);
#pragma unroll
                        for (int k = 0; k < L; ++k) a[c][k] = w[k];
                        pd_to_words<L, L>(w, y[c], pd);
#pragma unroll
                        for (int k = 0; k < L; ++k) y[c][k] = w[k];
                    }
                }
            }
            __syncwarp(tm.mask);
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                uint32_t pl[L], mi[L];
                lz32_add<L>(pl, a[c], y[c]);
                lz32_sub<L>(mi, a[c], y[c], B);
                uint32_t* d0 = (ng[c] ? pb : pa) + t * L;
                uint32_t* d1 = (ng[c] ? pa : pb) + t * L;
                st_res<L>(d0, pl);
                st_res<L>(d1, mi);
            }
            __syncwarp(tm.mask);
        }
        __syncthreads();
    }
}

// Elements j = 2i + parity (i < m) of the column into slot bitrev(i) (log2 m bits).
template <int m, int L, bool FIRST>
__device__ __forceinline__ void half_load_fwd(const LevelParams& prm, uint32_t* half, uint64_t base, uint64_t l,
                                              uint64_t mu_d, int op, int parity) {
    using G = Geo<m, L>;
    constexpr int LOG2_M = ilog2<m>();
    const uint32_t* poly = prm.data + (op ? prm.poly_words : 0);
    const uint64_t* raw = op ? prm.raw_b : prm.raw_a;
    const int h = m / 2;
    if constexpr (!FIRST) {
        cp_async_elements<m, L>(
            half, m, [&](int i) { return poly + (base + (2 * (uint64_t)i + parity) * mu_d + l) * G::EW; },
            [&](int i) { return bitrev(i, LOG2_M); });
        if constexpr (L == kPdDigits) {
            // canonical digits in HBM: words for the DFT's arithmetic (the lazy DFT
            // converts in its first stage, where it loads every residue once)
            if (prm.pd_io && !prm.dft_lazy) {
                __syncthreads();
                for (int idx = threadIdx.x; idx < m * m; idx += kThreads) {
                    uint32_t* r = half + (idx / m) * G::ES + (idx % m) * L;
                    uint32_t d[L], w[L];
                    ld_res<L>(d, r);
                    pd_to_words<L, L>(w, d, prm.pd);
                    st_res<L>(r, w);
                }
            }
        }
        return;
    }
    for (int idx = threadIdx.x; idx < m * m; idx += kThreads) {
        const int i = idx / m, t = idx % m;
        const uint64_t j = 2 * (uint64_t)i + parity;
        uint32_t* dst = half + bitrev(i, LOG2_M) * G::ES + t * L;
        if constexpr (FIRST) {
            const uint64_t io = j * mu_d + l;           // outer coefficient index
            uint32_t v = 0;
            if (io < prm.M && t < h) v = get_field(raw, prm.raw_words, prm.n_bits, (uint64_t)prm.u * (io * h + t), prm.u);
            dst[0] = v;
#pragma unroll
            for (int w = 1; w < L; ++w) dst[w] = 0;
        } else {
            uint32_t x[L];
            ld_res<L>(x, poly + ((base + j * mu_d + l) * m + t) * L);
            st_res<L>(dst, x);
        }
    }
}

template <int m, int L, bool FIRST>
__global__ void __launch_bounds__(kThreads, 3) k_dft_fwd_half(LevelParams prm, Mod<L> md, uint32_t* scratch,
                                                           uint32_t operands) {
    using G = Geo<m, L>;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* E = scratch + (uint64_t)blockIdx.x * m * G::EW;
    const int lg_mu = (__ffsll((long long)prm.len) - 1) - ilog2<G::TWO_M>();
    const uint64_t mu_d = 1ull << lg_mu;
    const uint64_t cols = prm.P2 / G::TWO_M;
    Team<m, L> tm;
    for (uint64_t item = blockIdx.x; item < cols * operands; item += gridDim.x) {
        const int op = (int)(item / cols);
        const uint64_t column = item % cols;
        const uint64_t blk = column >> lg_mu, l = column & (mu_d - 1);
        const uint64_t base = blk * prm.len;
        uint32_t* poly = prm.data + (op ? prm.poly_words : 0);
        const bool lazy = prm.dft_lazy != 0;   // unreduced sums, one reduction per output
        // even elements: E_v, v < m, to the scratch slice
        half_load_fwd<m, L, FIRST>(prm, smem, base, l, mu_d, op, 0);
        __syncthreads();
        const bool pd_in = !FIRST && prm.pd_io;
        if (lazy) dft_dit_lazy<m, L>(smem, m, 2, 0, md, pd_in, prm.pd);
        else dft_dit<m, L>(smem, 1, m, 2, md);
        copy_words_block<m, L>(E, smem, m * G::EW);
        __syncthreads();
        // odd elements: O_v in shared memory
        half_load_fwd<m, L, FIRST>(prm, smem, base, l, mu_d, op, 1);
        __syncthreads();
        if (lazy) dft_dit_lazy<m, L>(smem, m, 2, 0, md, pd_in, prm.pd);
        else dft_dit<m, L>(smem, 1, m, 2, md);
        uint32_t B6[L];   // the lazy halves are below 2^6 q
        lz32_bias<L>(B6, md, ilog2<m>());
        // X_v = E_v + alpha^v O_v, X_(v+m) = E_v - alpha^v O_v.  A thread loads the inputs
        // of VB elements (CPL coefficients each) before it stores any output: the stores to
        // the polynomial may alias the scratch slice for the compiler, which would
        // otherwise keep every scratch load behind the previous output's stores.
        constexpr int VB = 2;
        static_assert(m % (VB * G::NTEAMS) == 0, "whole batches of elements");
        for (int v0 = tm.id; v0 < m; v0 += VB * G::NTEAMS) {
            uint32_t ea[VB][G::CPL][L], oy[VB][G::CPL][L];
            bool ngs[VB][G::CPL];
#pragma unroll
            for (int b = 0; b < VB; ++b)
#pragma unroll
                for (int c = 0; c < G::CPL; ++c) {
                    const int v = v0 + b * G::NTEAMS, t = tm.lane + c * G::TEAM;
                    ld_res<L>(ea[b][c], E + v * G::EW + t * L);
                    shifted<m, L>(oy[b][c], ngs[b][c], smem + v * G::ES, t, v);
                }
#pragma unroll
            for (int b = 0; b < VB; ++b)
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                const int v = v0 + b * G::NTEAMS, t = tm.lane + c * G::TEAM;
                uint32_t pl[L], mi[L];
                const uint32_t(&a)[L] = ea[b][c];
                const uint32_t(&y)[L] = oy[b][c];
                const bool ng = ngs[b][c];
                if (lazy) {
                    uint32_t x[L];
                    lz32_add<L>(x, a, y);
                    lz32_reduce<L>(pl, x, md, prm.red_rcp);
                    lz32_sub<L>(x, a, y, B6);
                    lz32_reduce<L>(mi, x, md, prm.red_rcp);
                } else {
                    add_mod<L>(pl, a, y, md);
                    sub_mod<L>(mi, a, y, md);
                }
                // where the shifted coefficient carries a minus sign the two results trade places
                uint32_t* d0 = poly + ((base + (uint64_t)v * mu_d + l) * m + t) * L;
                uint32_t* d1 = poly + ((base + (uint64_t)(v + m) * mu_d + l) * m + t) * L;
                if constexpr (L == kPdDigits) {
                    if (prm.pd_io) {   // canonical digits for the bad multiplications
                        uint32_t dg[L];
                        // 4-word residues: p^4 >= 2^96, so p > 2^24 and the short conversion applies
                        if (prm.pd_fast) {
                            const ModPD<L, true> f = pd_fast_view(prm.pd);
                            pd_from_words4_large_p(dg, pl, prm.pd_pw, f);
#pragma unroll
                            for (int w = 0; w < L; ++w) pl[w] = dg[w];
                            pd_from_words4_large_p(dg, mi, prm.pd_pw, f);
                        } else {
                            pd_from_words4_large_p(dg, pl, prm.pd_pw, prm.pd);
#pragma unroll
                            for (int w = 0; w < L; ++w) pl[w] = dg[w];
                            pd_from_words4_large_p(dg, mi, prm.pd_pw, prm.pd);
                        }
#pragma unroll
                        for (int w = 0; w < L; ++w) mi[w] = dg[w];
                    }
                }
                st_res<L>(ng ? d1 : d0, pl);
                st_res<L>(ng ? d0 : d1, mi);
            }
        }
        __syncthreads();   // shared memory and the scratch slice are reused by the next column
    }
}

template <int m, int L>
__global__ void __launch_bounds__(kThreads) k_dft_inv_half(LevelParams prm, Mod<L> md, uint32_t* scratch) {
    using G = Geo<m, L>;
    constexpr int LOG2_M = ilog2<m>();
    constexpr int ROOT = G::TWO_M - 1;                 // alpha^-1
    constexpr int SUB_ROOT = (2 * ROOT) % G::TWO_M;    // alpha^-2 for the half DFTs
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* D = scratch + (uint64_t)blockIdx.x * m * G::EW;
    const uint64_t mu_d = prm.len / G::TWO_M;
    const uint64_t cols = prm.P2 / G::TWO_M;
    uint32_t* poly = prm.data;
    for (uint64_t column = blockIdx.x; column < cols; column += gridDim.x) {
        const uint64_t blk = column / mu_d, l = column % mu_d;
        const uint64_t base = blk * prm.len;
        // s_k = x_k + x_(k+m) to shared memory, d_k = alpha^(ROOT k) (x_k - x_(k+m)) to the scratch slice.
        // A thread loads the residues of IB items before it stores any result: the stores
        // to the scratch slice may alias the polynomial for the compiler, which would
        // otherwise keep every load behind the previous item's store.
        constexpr int IB = 4;
        static_assert((m * m) % (IB * kThreads) == 0, "whole batches of items");
        for (int idx0 = threadIdx.x; idx0 < m * m; idx0 += IB * kThreads) {
            uint32_t a[IB][L], b[IB][L], a2[IB][L], b2[IB][L];
#pragma unroll
            for (int i = 0; i < IB; ++i) {
                const int idx = idx0 + i * kThreads;
                const int k = idx / m, t = idx % m;
                const uint32_t* pa = poly + (base + (uint64_t)k * mu_d + l) * G::EW;
                const uint32_t* pb = poly + (base + (uint64_t)(k + m) * mu_d + l) * G::EW;
                ld_res<L>(a[i], pa + t * L);
                ld_res<L>(b[i], pb + t * L);
                // coefficient t of alpha^sh (a - b): +-(a - b)[t - sh]; b - a where the sign is negative
                const int sh = (ROOT * k) & (G::TWO_M - 1);
                int src = t - sh;
                bool neg = false;
                if (src < 0) {
                    src += m;
                    neg = true;
                    if (src < 0) {
                        src += m;
                        neg = false;
                    }
                }
                ld_res<L>(a2[i], (neg ? pb : pa) + src * L);
                ld_res<L>(b2[i], (neg ? pa : pb) + src * L);
            }
#pragma unroll
            for (int i = 0; i < IB; ++i) {
                const int idx = idx0 + i * kThreads;
                const int k = idx / m, t = idx % m;
                uint32_t r[L];
                add_mod<L>(r, a[i], b[i], md);
                st_res<L>(smem + k * G::ES + t * L, r);
                sub_mod<L>(r, a2[i], b2[i], md);
                st_res<L>(D + k * G::EW + t * L, r);
            }
        }
        __syncthreads();
        // even outputs X_(2v), from slot bitrev(v)
        dft_dif<m, L>(smem, 1, m, SUB_ROOT, md);
        for (int idx = threadIdx.x; idx < m * m; idx += kThreads) {
            const int v = idx / m, t = idx % m;
            uint32_t x[L];
            ld_res<L>(x, smem + bitrev(v, LOG2_M) * G::ES + t * L);
            st_res<L>(poly + ((base + (uint64_t)(2 * v) * mu_d + l) * m + t) * L, x);
        }
        __syncthreads();
        // odd outputs X_(2v+1)
        cp_async_elements<m, L>(
            smem, m, [&](int i) { return D + (uint64_t)i * G::EW; }, [](int i) { return i; });
        __syncthreads();
        dft_dif<m, L>(smem, 1, m, SUB_ROOT, md);
        for (int idx = threadIdx.x; idx < m * m; idx += kThreads) {
            const int v = idx / m, t = idx % m;
            uint32_t x[L];
            ld_res<L>(x, smem + bitrev(v, LOG2_M) * G::ES + t * L);
            st_res<L>(poly + ((base + (uint64_t)(2 * v + 1) * mu_d + l) * m + t) * L, x);
        }
        __syncthreads();
    }
}

template <int m, int L>
constexpr size_t half_column_smem_bytes() {
    static_assert(Geo<m, L>::ES == Geo<m, L>::EW, "half columns are copied to and from their scratch word for word");
    return sizeof(uint32_t) * (size_t)m * Geo<m, L>::ES;
}

template <int m, int L>
constexpr size_t column_smem_bytes() {
    return sizeof(uint32_t) * (size_t)Geo<m, L>::TWO_M * Geo<m, L>::ES;
}

template <int m, int L, int LR>
constexpr size_t twiddle_smem_bytes() {
    return sizeof(uint32_t) * (size_t)Geo<m, L>::NTEAMS * TeamBuf<m, LR>::WORDS;
}

template <int m, int L, int LR>
size_t final_smem_bytes(int n, int form = kFormDirect, int S = 0) {
    using G = Geo<m, L>;
    const size_t tb = form == kFormI8    ? (size_t)kWarps * i8_warp_words<m, LR>(S)
                      : form == kFormNtt ? (size_t)NttTeam<m>::NTEAMS * 2 * m * LR
                                         : (size_t)G::NTEAMS * TeamBuf<m, LR>::WORDS;
    const size_t nn = (size_t)n * (form == kFormNtt ? final_blocks_per_cta<m>(n) : 1);
    return sizeof(uint32_t) * (2 * nn * G::ES + tb);
}

template <int m, int L, int LR>
constexpr size_t twiddle_ntt_smem_bytes() {
    return sizeof(uint32_t) * (size_t)NttTeam<m>::NTEAMS * m * LR;
}

template <int m, int L, int LR>
size_t twiddle_i8_smem_bytes(int S) {
    return sizeof(uint32_t) * (size_t)kWarps * i8_warp_words<m, LR>(S);
}

}  // namespace dkss
