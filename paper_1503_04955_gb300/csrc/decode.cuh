// Decoding and carry propagation (thesis Section 3.2.8): evaluate the inner
// polynomials at alpha = 2^u and the outer ones at x = 2^(um/2).  Digit k of
// weight 2^(uk) is D_k = c_{k div h, k mod h} + c_{k div h - 1, k mod h + h}
// (h = m/2); the product is sum_k D_k 2^(uk).
//
// The sum is formed per 32-bit output window j: S_j adds the pieces of every
// D_k overlapping bits [32j, 32j+32).  T_j = (S_j mod 2^32) + (S_{j-1} div 2^32)
// leaves a binary carry g_j = T_j div 2^32, which a device-wide scan resolves:
// carry-in of window j+1 = g_j | (p_j & carry-in of j), p_j = (T_j mod 2^32 ==
// 2^32-1).  The scan is reduce-then-scan over tiles of 2048 windows (three
// launches, no inter-CTA waiting): tile aggregates, one CTA scanning them,
// then a fix-up of the windows a tile's carry-in reaches.
#pragma once
#include <cstdint>

#include "arith.cuh"
#include "status_bits.hpp"

namespace dkss {

constexpr int kDecThreads = 256;
constexpr int kDecWPT = 8;
constexpr int kDecTile = kDecThreads * kDecWPT;
constexpr int kScanThreads = 1024;

struct DecodeParams {
    const uint32_t* c;     // 2M elements x m residues x L words, natural order
    uint32_t* out;         // product as 32-bit windows
    uint32_t* agg;         // per tile: bit0 generate, bit1 propagate; then carry-in
    uint32_t* status;
    uint64_t P2;
    uint64_t n_windows;
    uint64_t n_tiles;
    uint64_t k_max;        // number of digits D_k
    uint32_t m, h, u, db;  // db: bit bound of any D_k
    uint32_t out_aligned16;
};

template <int L>
__device__ __forceinline__ void load_digit(uint32_t (&D)[L + 1], const DecodeParams& p, uint64_t k) {
    uint64_t i = k / p.h;
    uint32_t t = (uint32_t)(k % p.h);
#pragma unroll
    for (int w = 0; w <= L; ++w) D[w] = 0;
    if (i < p.P2) {
        const uint32_t* s = p.c + (i * p.m + t) * L;
#pragma unroll
        for (int w = 0; w < L; ++w) D[w] = s[w];
    }
    if (i >= 1 && i - 1 < p.P2) {
        const uint32_t* s = p.c + ((i - 1) * p.m + t + p.h) * L;
        uint32_t carry = 0;
#pragma unroll
        for (int w = 0; w < L; ++w) {
            uint64_t x = (uint64_t)D[w] + s[w] + carry;
            D[w] = (uint32_t)x;
            carry = (uint32_t)(x >> 32);
        }
        D[L] += carry;
    }
}

// S_j: sum of the 32-bit pieces of all D_k overlapping window j.
template <int L>
__device__ uint64_t window_sum(const DecodeParams& p, uint64_t j) {
    const int64_t lo_bit = (int64_t)32 * (int64_t)j;
    // D_k overlaps the window iff u*k + db > lo_bit and u*k < lo_bit + 32
    const int64_t x = lo_bit - (int64_t)p.db;
    const uint64_t k_lo = x < 0 ? 0 : (uint64_t)(x / p.u) + 1;
    uint64_t k_hi = (uint64_t)(lo_bit + 31) / p.u;
    if (k_hi >= p.k_max) k_hi = p.k_max - 1;
    uint64_t S = 0;
    for (uint64_t k = k_lo; k <= k_hi && k < p.k_max; ++k) {
        uint32_t D[L + 1];
        load_digit<L>(D, p, k);
        int64_t off = lo_bit - (int64_t)p.u * (int64_t)k;   // bit of D at the window start
        uint32_t piece;
        if (off < 0) {
            piece = D[0] << (uint32_t)(-off);
        } else {
            int w = (int)(off >> 5), s = (int)(off & 31);
            uint32_t a = w <= L ? D[w] : 0u;
            uint32_t b = w + 1 <= L ? D[w + 1] : 0u;
            piece = s ? ((a >> s) | (b << (32 - s))) : a;
        }
        S += piece;
    }
    return S;
}

struct GP {
    uint32_t g, p;
};

__device__ __forceinline__ GP gp_combine(GP a, GP b) {  // a then b
    return GP{b.g | (b.p & a.g), a.p & b.p};
}

// Block-wide exclusive scan of (g, p); returns the thread's exclusive prefix
// and writes the block total.
template <int THREADS>
__device__ GP gp_block_scan(GP x, GP& total) {
    __shared__ uint32_t warp_g[THREADS / 32], warp_p[THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    GP incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t g = __shfl_up_sync(0xffffffffu, incl.g, d);
        uint32_t pp = __shfl_up_sync(0xffffffffu, incl.p, d);
        if (lane >= d) incl = gp_combine(GP{g, pp}, incl);
    }
    if (lane == 31) {
        warp_g[warp] = incl.g;
        warp_p[warp] = incl.p;
    }
    __syncthreads();
    GP wpre{0u, 1u};
    for (int w = 0; w < warp; ++w) wpre = gp_combine(wpre, GP{warp_g[w], warp_p[w]});
    GP tot{0u, 1u};
    for (int w = 0; w < THREADS / 32; ++w) tot = gp_combine(tot, GP{warp_g[w], warp_p[w]});
    total = tot;
    uint32_t eg = __shfl_up_sync(0xffffffffu, incl.g, 1);
    uint32_t ep = __shfl_up_sync(0xffffffffu, incl.p, 1);
    GP excl_in_warp = lane == 0 ? GP{0u, 1u} : GP{eg, ep};
    __syncthreads();
    return gp_combine(wpre, excl_in_warp);
}

// Carry resolution inside a tile and the tile aggregate: wv are the thread's
// window values, gbit/pbit its generate/propagate bits (bit w = window j0+w).
__device__ __forceinline__ void decode_tile_finish(const DecodeParams& p, uint64_t j0, const uint32_t (&wv)[kDecWPT],
                                                   uint32_t gbit, uint32_t pbit, uint64_t tile) {
    // thread aggregate: carry out with carry-in 0, and whether a carry-in passes through
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kDecWPT; ++w) c = ((gbit >> w) & 1) | (((pbit >> w) & 1) & c);
    GP mine{c, pbit == (1u << kDecWPT) - 1 ? 1u : 0u};
    GP total;
    GP pre = gp_block_scan<kDecThreads>(mine, total);
    c = pre.g;   // carry into this thread with the tile's carry-in taken as 0
    uint32_t o[kDecWPT];
#pragma unroll
    for (int w = 0; w < kDecWPT; ++w) {
        o[w] = wv[w] + c;
        c = ((gbit >> w) & 1) | (((pbit >> w) & 1) & c);
    }
    if (p.out_aligned16 && j0 + kDecWPT <= p.n_windows) {
        uint4* dst = reinterpret_cast<uint4*>(p.out + j0);
        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
    } else {
        for (int w = 0; w < kDecWPT; ++w)
            if (j0 + w < p.n_windows) p.out[j0 + w] = o[w];
    }
    if (threadIdx.x == 0) p.agg[tile] = total.g | (total.p << 1);
}

template <int L>
__device__ __forceinline__ void decode_tile(const DecodeParams& p, uint64_t tile) {
    const uint64_t j0 = tile * kDecTile + (uint64_t)threadIdx.x * kDecWPT;
    uint64_t S_prev = j0 >= 1 && j0 - 1 < p.n_windows ? window_sum<L>(p, j0 - 1) : 0;
    uint32_t wv[kDecWPT], gbit = 0, pbit = 0;
#pragma unroll
    for (int w = 0; w < kDecWPT; ++w) {
        uint64_t j = j0 + w;
        uint64_t S = j < p.n_windows ? window_sum<L>(p, j) : 0;
        uint64_t T = (S & 0xffffffffull) + (S_prev >> 32);
        wv[w] = (uint32_t)T;
        gbit |= (uint32_t)(T >> 32) << w;
        pbit |= (uint32_t)(wv[w] == 0xffffffffu) << w;
        S_prev = S;
    }
    decode_tile_finish(p, j0, wv, gbit, pbit, tile);
}

template <int L>
__global__ void __launch_bounds__(kDecThreads) k_decode_tiles(DecodeParams p) {
    decode_tile<L>(p, blockIdx.x);
}

// Same tile for u = 32/R (R = 1, 2): digit k sits at bit u*k, so the digits
// R j .. R j + R - 1 start in window j and reach windows j .. j + T - 1.
// Lane x of a warp owns window j = chunk + x: it loads its R digits (lanes
// read consecutive residues, so a warp's loads are contiguous), cuts them into
// the pieces P_t landing in windows j + t, and takes the pieces of window j
// from lanes x - t with shuffles (from the previous chunk across the warp's
// edge).  Window values go through shared memory (sbuf: kDecSmemWords words)
// to the layout of decode_tile_finish, 8 consecutive windows per thread.
constexpr int kDecSmemWords = kDecTile + kDecTile / 4;

template <int L, int R>
__device__ __forceinline__ void decode_tile_aligned(const DecodeParams& p, uint64_t tile, uint32_t* sbuf) {
    constexpr int U = 32 / R;
    constexpr int T = L + 2;                               // windows a digit reaches
    constexpr int PER_WARP = kDecTile / (kDecThreads / 32);
    uint32_t* s_wv = sbuf;
    uint8_t* s_gp = reinterpret_cast<uint8_t*>(sbuf + kDecTile);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t jt = (int64_t)tile * kDecTile;
    const int64_t jw = jt + (int64_t)warp * PER_WARP;
    const uint32_t hshift = 31 - __clz(p.h);
    uint64_t Pprev[T], Sprev = 0;
#pragma unroll
    for (int t = 0; t < T; ++t) Pprev[t] = 0;
    for (int it = -1; it < PER_WARP / 32; ++it) {
        const int64_t j = jw + 32 * it + lane;
        uint64_t P[T];
#pragma unroll
        for (int t = 0; t < T; ++t) P[t] = 0;
#pragma unroll
        for (int s = 0; s < R; ++s) {
            const int64_t k = (int64_t)R * j + s;
            uint32_t D[L + 1];
#pragma unroll
            for (int w = 0; w <= L; ++w) D[w] = 0;
            if (k >= 0 && (uint64_t)k < p.k_max) {
                const uint64_t i = (uint64_t)k >> hshift;
                const uint32_t t = (uint32_t)k & (p.h - 1);
                uint32_t y[L];
                if (i < p.P2) {
                    ld_res<L>(y, p.c + (i * p.m + t) * L);
#pragma unroll
                    for (int w = 0; w < L; ++w) D[w] = y[w];
                }
                if (i >= 1 && i - 1 < p.P2) {
                    ld_res<L>(y, p.c + ((i - 1) * p.m + t + p.h) * L);
                    uint32_t carry = 0;
#pragma unroll
                    for (int w = 0; w < L; ++w) {
                        const uint64_t x = (uint64_t)D[w] + y[w] + carry;
                        D[w] = (uint32_t)x;
                        carry = (uint32_t)(x >> 32);
                    }
                    D[L] = carry;
                }
            }
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const int sh = 32 * t - U * s;   // bit of the digit at the start of window j + t
                uint32_t piece;
                if (sh < 0) {
                    piece = D[0] << (-sh);
                } else {
                    const int lw = sh >> 5, bs = sh & 31;
                    const uint32_t a = lw <= L ? D[lw] : 0u;
                    const uint32_t b = lw + 1 <= L ? D[lw + 1] : 0u;
                    piece = bs ? ((a >> bs) | (b << (32 - bs))) : a;
                }
                P[t] += piece;
            }
        }
        // window j's pieces: P_t of lane x - t (lane y sends to lane y + t, or
        // across the edge its previous chunk's piece)
        uint64_t S = P[0];
#pragma unroll
        for (int t = 1; t < T; ++t) {
            const uint64_t send = lane + t < 32 ? P[t] : Pprev[t];
            const int src = (lane - t) & 31;
            const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)send, src);
            const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(send >> 32), src);
            S += ((uint64_t)hi << 32) | lo;
        }
        if (j < 0 || (uint64_t)j >= p.n_windows) S = 0;
        // T_j = (S_j mod 2^32) + (S_(j-1) div 2^32)
        const uint64_t sendS = lane == 31 ? Sprev : S;
        const uint32_t phi = __shfl_sync(0xffffffffu, (uint32_t)(sendS >> 32), (lane - 1) & 31);
        if (it >= 0) {
            const uint64_t T2 = (S & 0xffffffffull) + phi;
            const uint32_t v = (uint32_t)T2;
            s_wv[j - jt] = v;
            s_gp[j - jt] = (uint8_t)((uint32_t)(T2 >> 32) | ((v == 0xffffffffu) ? 2u : 0u));
        }
#pragma unroll
        for (int t = 0; t < T; ++t) Pprev[t] = P[t];
        Sprev = S;
    }
    __syncthreads();
    uint32_t wv[kDecWPT], gbit = 0, pbit = 0;
#pragma unroll
    for (int w = 0; w < kDecWPT; ++w) {
        const int idx = threadIdx.x * kDecWPT + w;
        wv[w] = s_wv[idx];
        const uint32_t gp = s_gp[idx];
        gbit |= (gp & 1u) << w;
        pbit |= ((gp >> 1) & 1u) << w;
    }
    decode_tile_finish(p, (uint64_t)(jt + threadIdx.x * kDecWPT), wv, gbit, pbit, tile);
}

template <int L, int R>
__global__ void __launch_bounds__(kDecThreads) k_decode_tiles_aligned(DecodeParams p) {
    __shared__ uint32_t sbuf[kDecSmemWords];
    decode_tile_aligned<L, R>(p, blockIdx.x, sbuf);
}

// One CTA of THREADS threads: exclusive scan of the tile aggregates into
// per-tile carry-ins.
template <int THREADS>
__device__ __forceinline__ void decode_scan_block(const DecodeParams& p) {
    uint32_t carry = 0;
    for (uint64_t base = 0; base < p.n_tiles; base += THREADS) {
        uint64_t t = base + threadIdx.x;
        uint32_t a = t < p.n_tiles ? p.agg[t] : 2u;
        GP total;
        GP pre = gp_block_scan<THREADS>(GP{a & 1u, (a >> 1) & 1u}, total);
        if (t < p.n_tiles) p.agg[t] = pre.g | (pre.p & carry);
        carry = total.g | (total.p & carry);
    }
    if (threadIdx.x == 0 && carry) atomicOr(p.status, kStatusCarryOut);
}

static __global__ void __launch_bounds__(kScanThreads) k_decode_scan(DecodeParams p) {
    decode_scan_block<kScanThreads>(p);
}

// Add tile t's carry-in at its first window and ripple it while windows wrap.
__device__ __forceinline__ void decode_fix_tile(const DecodeParams& p, uint64_t t) {
    if (t >= p.n_tiles || !p.agg[t]) return;
    uint64_t end = (t + 1) * kDecTile;
    if (end > p.n_windows) end = p.n_windows;
    for (uint64_t j = t * kDecTile; j < end; ++j) {
        uint32_t v = p.out[j] + 1u;
        p.out[j] = v;
        if (v != 0u) break;
    }
}

static __global__ void k_decode_fix(DecodeParams p) {
    decode_fix_tile(p, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

}  // namespace dkss
