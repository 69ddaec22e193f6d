// DKSS_MUL stage kernels (thesis Section 3.2 steps 4-8, Section 4.2).
//
// Layout in HBM: a polynomial over R is 2M elements, element e holds m
// residues (inner coefficients) of L 32-bit limbs, residue-major:
// word (e*m + t)*L + l.  Every kernel below works on that layout.
//
// The forward 2M-point transform is the thesis's radix-2m decimation in time
// (Section 3.2.5 i.-iii.), done in place level by level: level d splits each
// block of len = 2M/(2m)^(d-1) elements into 2m rows of len/2m columns; one
// CTA takes one column, runs the 2m-point inner DFT with root alpha (shifts
// only) in shared memory and multiplies output v of column l by the bad
// twiddle rho^(v*l*(2m)^(d-1)).  After the last level the elements sit in
// mixed-radix digit-reversed order.  Componentwise products do not care about
// order; the backwards transform runs the same levels in reverse as
// decimation in frequency with rho^-1 and alpha^-1 (the backwards transform
// of Section 2.7), which returns natural order.
#pragma once
#include <cstdint>

#include "arith.cuh"
#include "rr_arith.cuh"

namespace dkss {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <int m, int L>
struct Geo {
    static constexpr int TWO_M = 2 * m;
    static constexpr int EW = m * L;                     // words per element of R
    static constexpr int TEAM = m < 32 ? m : 32;         // lanes per element
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
};

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
// slots (one array, or two arrays transformed together); leaves
// X_v = sum_j x_j (alpha^root)^(j v) in slot v.  root is a shift amount in
// [0, 2m).  Butterflies are spread over teams; a team owns whole butterflies,
// so one __syncwarp separates its reads from its writes.
template <int m, int L>
__device__ void dft_dit(uint32_t* s0, uint32_t* s1, int arrays, int n, int root, const Mod<L>& md) {
    using G = Geo<m, L>;
    Team<m, L> tm;
    for (int half = 1; half < n; half <<= 1) {
        const int scale = n / (2 * half);
        for (int bfa = tm.id; bfa < arrays * (n / 2); bfa += G::NTEAMS) {
            uint32_t* s = bfa < n / 2 ? s0 : s1;
            int bf = bfa < n / 2 ? bfa : bfa - n / 2;
            int k_in = bf % half;
            int ia = (bf / half) * 2 * half + k_in;
            int ib = ia + half;
            int sh = (root * scale * k_in) % G::TWO_M;
            uint32_t a[G::CPL][L], y[G::CPL][L];
            bool ng[G::CPL];
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                ld_res<L>(a[c], s + ia * G::EW + t * L);
                shifted<m, L>(y[c], ng[c], s + ib * G::EW, t, sh);
            }
            __syncwarp(tm.mask);
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                uint32_t sa[L], sb[L];
                if (ng[c]) {
                    sub_mod<L>(sa, a[c], y[c], md);
                    add_mod<L>(sb, a[c], y[c], md);
                } else {
                    add_mod<L>(sa, a[c], y[c], md);
                    sub_mod<L>(sb, a[c], y[c], md);
                }
                st_res<L>(s + ia * G::EW + t * L, sa);
                st_res<L>(s + ib * G::EW + t * L, sb);
            }
            __syncwarp(tm.mask);
        }
        __syncthreads();
    }
}

// In-place radix-2 DIF over n elements in natural slots; leaves
// X_v = sum_j x_j (alpha^root)^(j v) in slot bitrev(v).
template <int m, int L>
__device__ void dft_dif(uint32_t* s, int n, int root, const Mod<L>& md) {
    using G = Geo<m, L>;
    Team<m, L> tm;
    for (int half = n / 2; half >= 1; half >>= 1) {
        const int scale = n / (2 * half);
        for (int bf = tm.id; bf < n / 2; bf += G::NTEAMS) {
            int k_in = bf % half;
            int ia = (bf / half) * 2 * half + k_in;
            int ib = ia + half;
            int sh = (root * scale * k_in) % G::TWO_M;
            uint32_t sa[G::CPL][L], db[G::CPL][L];
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                uint32_t a[L], b[L];
                ld_res<L>(a, s + ia * G::EW + t * L);
                ld_res<L>(b, s + ib * G::EW + t * L);
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
                ld_res<L>(a, s + ia * G::EW + src * L);
                ld_res<L>(b, s + ib * G::EW + src * L);
                if (neg) sub_mod<L>(db[c], b, a, md);
                else sub_mod<L>(db[c], a, b, md);
            }
            __syncwarp(tm.mask);
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                st_res<L>(s + ia * G::EW + t * L, sa[c]);
                st_res<L>(s + ib * G::EW + t * L, db[c]);
            }
            __syncwarp(tm.mask);
        }
        __syncthreads();
    }
}

// Negacyclic product in R (Section 2.9.2, eq. ncycconv) times alpha^r, in
// 26-bit limbs: out_k = REDC(sum_i x_i E[(k - r - i) mod 2m]) where
// E[t] = y_t and E[t+m] = -y_t, so that the wrapped terms carry their minus
// sign.  X and E are the team's shared buffers; results stay in registers.
template <int m, int LR>
__device__ __forceinline__ void negacyclic_mul_rr(uint32_t (&out)[Geo<m, 1>::CPL][LR], const uint32_t* X,
                                                  const uint32_t* E, int r, const ModRR<LR>& md, int lane) {
    constexpr int CPL = Geo<m, 1>::CPL, TEAM = Geo<m, 1>::TEAM;
    uint64_t col[CPL][2 * LR];
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int i = 0; i < 2 * LR; ++i) col[c][i] = 0;
#pragma unroll 4
    for (int i = 0; i < m; ++i) {
        uint32_t xi[LR];
        ld_rr<LR>(xi, X + i * LR);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int k = lane + c * TEAM;
            uint32_t y[LR];
            ld_rr<LR>(y, E + ((k - r - i) & (2 * m - 1)) * LR);
            mac_cols<LR>(col[c], xi, y);
        }
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) redc_cols<LR>(out[c], col[c], md);
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

// ---------------------------------------------------------------------------
// Forward level: inner DFT of one column (root alpha) + bad multiplications.
// Grid: x = column (2M/2m of them), y = operand (0: a, 1: b).
// ---------------------------------------------------------------------------
template <int m, int L, int LR, bool FIRST>
__global__ void __launch_bounds__(kThreads) k_fwd_level(LevelParams prm, Mod<L> md, ModRR<LR> mr) {
    using G = Geo<m, L>;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* col = smem;                                   // 2m elements
    uint32_t* tbuf = smem + G::TWO_M * G::EW;               // per-team product buffers
    constexpr int LOG2_TWO_M = ilog2<G::TWO_M>();
    const uint64_t column = blockIdx.x;
    const int op = blockIdx.y;
    uint32_t* poly = prm.data + (op ? prm.poly_words : 0);
    const uint64_t mu_d = prm.len / G::TWO_M;
    const uint64_t blk = column / mu_d, l = column % mu_d;
    const uint64_t base = blk * prm.len;

    // load the column e_l: element j at position base + j*mu_d + l, into slot bitrev(j)
    if constexpr (FIRST) {
        const uint64_t* raw = op ? prm.raw_b : prm.raw_a;
        const int h = m / 2;
        for (int idx = threadIdx.x; idx < G::TWO_M * m; idx += kThreads) {
            int j = idx / m, t = idx % m;
            uint64_t i = (uint64_t)j * mu_d + l;        // outer coefficient index
            uint32_t v = 0;
            if (i < prm.M && t < h) v = get_field(raw, prm.raw_words, prm.n_bits, (uint64_t)prm.u * (i * h + t), prm.u);
            uint32_t* dst = col + bitrev(j, LOG2_TWO_M) * G::EW + t * L;
            dst[0] = v;
#pragma unroll
            for (int w = 1; w < L; ++w) dst[w] = 0;
        }
    } else {
        for (int idx = threadIdx.x; idx < G::TWO_M * m; idx += kThreads) {
            int j = idx / m, t = idx % m;
            uint32_t x[L];
            ld_res<L>(x, poly + ((base + (uint64_t)j * mu_d + l) * m + t) * L);
            st_res<L>(col + bitrev(j, LOG2_TWO_M) * G::EW + t * L, x);
        }
    }
    __syncthreads();
    dft_dit<m, L>(col, col, 1, G::TWO_M, 1, md);

    // bad multiplications: output v of column l times rho^(v l bp) = alpha^r rho^s
    Team<m, L> tm;
    uint32_t* X = tbuf + tm.id * TeamBuf<m, LR>::WORDS;
    uint32_t* E = X + m * LR;
    for (int v = tm.id; v < G::TWO_M; v += G::NTEAMS) {
        const uint64_t e = (uint64_t)v * l * prm.bp;      // < 2M
        uint32_t* dst = poly + (base + (uint64_t)v * mu_d + l) * G::EW;
        const uint32_t* x = col + v * G::EW;
        if (e == 0) {
#pragma unroll
            for (int c = 0; c < G::CPL; ++c) {
                int t = tm.lane + c * G::TEAM;
                uint32_t y[L];
                ld_res<L>(y, x + t * L);
                st_res<L>(dst + t * L, y);
            }
            continue;
        }
        const int r = (int)(e >> prm.log2_mu_top);
        const uint64_t sidx = e & (prm.mu_top - 1);
        stage_x_rr<m, L, LR>(X, x, tm.lane);
        stage_ext_rr<m, LR>(E, prm.table + sidx * m * LR, mr, tm.lane);
        __syncwarp(tm.mask);
        uint32_t out[G::CPL][LR];
        negacyclic_mul_rr<m, LR>(out, X, E, r, mr, tm.lane);
#pragma unroll
        for (int c = 0; c < G::CPL; ++c) {
            uint32_t o32[L];
            from_rr<L, LR>(o32, out[c]);
            st_res<L>(dst + (tm.lane + c * G::TEAM) * L, o32);
        }
        __syncwarp(tm.mask);
    }
}

// ---------------------------------------------------------------------------
// Last level of both forward transforms, componentwise products scaled by
// (2M)^-1, and the first level of the backwards transform, fused.  One CTA
// per block of r = len contiguous elements (len <= 2m, root alpha^(2m/len)).
// ---------------------------------------------------------------------------
template <int m, int L, int LR>
__global__ void __launch_bounds__(kThreads) k_final_pointwise(LevelParams prm, Mod<L> md, ModRR<LR> mr) {
    using G = Geo<m, L>;
    extern __shared__ __align__(16) uint32_t smem[];
    const int n = (int)prm.len;
    const int log2n = 31 - __clz(n);
    uint32_t* sa = smem;
    uint32_t* sb = smem + n * G::EW;
    uint32_t* tbuf = sb + n * G::EW;
    const uint64_t base = (uint64_t)blockIdx.x * n;
    uint32_t* pa = prm.data;
    uint32_t* pb = prm.data + prm.poly_words;
    for (int idx = threadIdx.x; idx < n * m; idx += kThreads) {
        int j = idx / m, t = idx % m;
        uint32_t x[L];
        int slot = bitrev(j, log2n);
        ld_res<L>(x, pa + ((base + j) * m + t) * L);
        st_res<L>(sa + slot * G::EW + t * L, x);
        ld_res<L>(x, pb + ((base + j) * m + t) * L);
        st_res<L>(sb + slot * G::EW + t * L, x);
    }
    __syncthreads();
    const int root = G::TWO_M / n;
    dft_dit<m, L>(sa, sb, 2, n, root, md);
    // componentwise products c_v = a_v * b_v * (2M)^-1
    Team<m, L> tm;
    uint32_t* X = tbuf + tm.id * TeamBuf<m, LR>::WORDS;
    uint32_t* E = X + m * LR;
    uint32_t ks[LR];
#pragma unroll
    for (int w = 0; w < LR; ++w) ks[w] = prm.kscale[w];
    for (int v = tm.id; v < n; v += G::NTEAMS) {
        stage_x_rr<m, L, LR>(X, sa + v * G::EW, tm.lane);
        stage_ext_from32<m, L, LR>(E, sb + v * G::EW, mr, tm.lane);
        __syncwarp(tm.mask);
        uint32_t out[G::CPL][LR];
        negacyclic_mul_rr<m, LR>(out, X, E, 0, mr, tm.lane);
#pragma unroll
        for (int c = 0; c < G::CPL; ++c) {
            uint32_t scaled[LR], o32[L];
            mont_mul_rr<LR>(scaled, out[c], ks, mr);
            from_rr<L, LR>(o32, scaled);
            st_res<L>(sa + v * G::EW + (tm.lane + c * G::TEAM) * L, o32);
        }
        __syncwarp(tm.mask);
    }
    __syncthreads();
    // first backwards level: DFT with root alpha^(-2m/n), natural in, bit-reversed out
    dft_dif<m, L>(sa, n, (G::TWO_M - root) % G::TWO_M, md);
    for (int idx = threadIdx.x; idx < n * m; idx += kThreads) {
        int j = idx / m, t = idx % m;
        uint32_t x[L];
        ld_res<L>(x, sa + bitrev(j, log2n) * G::EW + t * L);
        st_res<L>(pa + ((base + j) * m + t) * L, x);
    }
}

// ---------------------------------------------------------------------------
// Backwards level (decimation in frequency): twiddle by rho^-(v l bp) first,
// then the 2m-point DFT with root alpha^-1 over the column.
// ---------------------------------------------------------------------------
template <int m, int L, int LR>
__global__ void __launch_bounds__(kThreads) k_inv_level(LevelParams prm, Mod<L> md, ModRR<LR> mr) {
    using G = Geo<m, L>;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* col = smem;
    uint32_t* tbuf = smem + G::TWO_M * G::EW;
    constexpr int LOG2_TWO_M = ilog2<G::TWO_M>();
    const uint64_t column = blockIdx.x;
    uint32_t* poly = prm.data;
    const uint64_t mu_d = prm.len / G::TWO_M;
    const uint64_t blk = column / mu_d, l = column % mu_d;
    const uint64_t base = blk * prm.len;
    for (int idx = threadIdx.x; idx < G::TWO_M * m; idx += kThreads) {
        int j = idx / m, t = idx % m;
        uint32_t x[L];
        ld_res<L>(x, poly + ((base + (uint64_t)j * mu_d + l) * m + t) * L);
        st_res<L>(col + j * G::EW + t * L, x);
    }
    __syncthreads();
    Team<m, L> tm;
    uint32_t* X = tbuf + tm.id * TeamBuf<m, LR>::WORDS;
    uint32_t* E = X + m * LR;
    for (int v = tm.id; v < G::TWO_M; v += G::NTEAMS) {
        uint64_t e = (uint64_t)v * l * prm.bp;
        if (e == 0) continue;
        e = prm.P2 - e;
        const int r = (int)(e >> prm.log2_mu_top);
        const uint64_t sidx = e & (prm.mu_top - 1);
        stage_x_rr<m, L, LR>(X, col + v * G::EW, tm.lane);
        stage_ext_rr<m, LR>(E, prm.table + sidx * m * LR, mr, tm.lane);
        __syncwarp(tm.mask);
        uint32_t out[G::CPL][LR];
        negacyclic_mul_rr<m, LR>(out, X, E, r, mr, tm.lane);
#pragma unroll
        for (int c = 0; c < G::CPL; ++c) {
            uint32_t o32[L];
            from_rr<L, LR>(o32, out[c]);
            st_res<L>(col + v * G::EW + (tm.lane + c * G::TEAM) * L, o32);
        }
        __syncwarp(tm.mask);
    }
    __syncthreads();
    dft_dif<m, L>(col, G::TWO_M, G::TWO_M - 1, md);
    for (int idx = threadIdx.x; idx < G::TWO_M * m; idx += kThreads) {
        int j = idx / m, t = idx % m;
        uint32_t x[L];
        ld_res<L>(x, col + bitrev(j, LOG2_TWO_M) * G::EW + t * L);
        st_res<L>(poly + ((base + (uint64_t)j * mu_d + l) * m + t) * L, x);
    }
}

template <int m, int L, int LR>
constexpr size_t level_smem_bytes() {
    using G = Geo<m, L>;
    return sizeof(uint32_t) * ((size_t)G::TWO_M * G::EW + (size_t)G::NTEAMS * TeamBuf<m, LR>::WORDS);
}

template <int m, int L, int LR>
size_t final_smem_bytes(int n) {
    using G = Geo<m, L>;
    return sizeof(uint32_t) * (2 * (size_t)n * G::EW + (size_t)G::NTEAMS * TeamBuf<m, LR>::WORDS);
}

}  // namespace dkss
