// R-multiplication as exact INT8 tensor-core products (mma.sync u8).
//
// The negacyclic product c_k = sum_i x_i E[(k - r - i) mod 2m] (thesis
// Section 2.9.2, eq. ncycconv; E[t] = y_t, E[t+m] = -y_t) is computed on
// integers first: each residue is split into S bytes (S = bytes of p^z),
// x_i = sum_s x_is 256^s and E_j = sum_t E_jt 256^t, so
//     c_k = sum_{t,s} 256^(t+s) C[t][k][s],  C[t][k][s] = sum_i E_(k-r-i),t x_is.
// For every byte t of E the m x m Toeplitz matrix E_(k-r-i),t times the m x S
// matrix of x bytes is one tensor-core product with M = (t, k), K = i,
// N = s: mma.m16n8k32 with u8 inputs and s32 accumulators.  A partial sum C
// is below m 255^2 < 2^22, so nothing overflows.  The diagonal sums
// D[d][k] = sum_{t+s=d} C[t][k][s] (< S 2^22 < 2^26) are gathered in shared
// memory, recombined exactly into the integer c_k < m (p^z)^2 and reduced with
// the Montgomery reduction of the direct form (26-bit limbs, R' = 2^(26 LR)).
//
// One warp owns an element.  tcgen05.mma has no .kind::i8 on sm_103a, so the
// warp-level mma.sync form is the tensor path that exists here.
#pragma once
#include <cstdint>

#include "rr_arith.cuh"

namespace dkss {

// Shared-memory bytes one warp needs for an R-multiplication with S byte slices.
template <int m>
__host__ __device__ constexpr int i8_warp_bytes(int S) {
    // x bytes: S planes of m; E bytes: S planes of 2m + 4 (wrap copy); D: (S + 16) rows of m words
    return ((S * m + 3) / 4) * 4 + ((S * (2 * m + 4) + 3) / 4) * 4 + (S + 16) * m * 4;
}

__device__ __forceinline__ void mma_u8_16832(int (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 4 consecutive bytes starting at byte offset off of a word-aligned buffer
__device__ __forceinline__ uint32_t ld_bytes4(const uint8_t* base, int off) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(base + (off & ~3));
    const uint32_t lo = w[0], hi = w[1];
    return __byte_perm(lo, hi, 0x3210 + 0x1111 * (off & 3));
}

// Byte planes of one element in a warp's buffer.
//   xb[s*m + i]          byte s of x_i
//   fb[t*(2m+4) + n]     byte t of E[(m - 1 - n) mod 2m] for n < 2m + 4
// With F_t[n] = E_t[(m - 1 - n) mod 2m], E_t[(k - r - i) mod 2m] is
// F_t[(m - 1 - k + r + i) mod 2m], so the 4 bytes of consecutive i an A
// register needs are consecutive in F_t.
template <int m, int LR>
__device__ __forceinline__ void i8_stage(uint8_t* xb, uint8_t* fb, int S, const uint32_t* x26, const uint32_t* E26,
                                         int lane) {
    // x: lane handles coefficients lane (+32)
    for (int i = lane; i < m; i += 32) {
        uint32_t v[LR];
        ld_rr<LR>(v, x26 + i * LR);
        uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < LR; ++j) {
            const int bit = 26 * j, wi = bit >> 5, sh = bit & 31;
            if (wi < 4) w[wi] |= v[j] << sh;
            if (sh > 6 && wi + 1 < 4) w[wi + 1] |= v[j] >> (32 - sh);
        }
        for (int s = 0; s < S; ++s) xb[s * m + i] = (uint8_t)(w[s >> 2] >> (8 * (s & 3)));
    }
    const int FW = 2 * m + 4;
    for (int n = lane; n < FW; n += 32) {
        const int j = ((m - 1 - n) % (2 * m) + 2 * m) % (2 * m);
        uint32_t v[LR];
        ld_rr<LR>(v, E26 + j * LR);
        uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
        for (int jj = 0; jj < LR; ++jj) {
            const int bit = 26 * jj, wi = bit >> 5, sh = bit & 31;
            if (wi < 4) w[wi] |= v[jj] << sh;
            if (sh > 6 && wi + 1 < 4) w[wi + 1] |= v[jj] >> (32 - sh);
        }
        for (int t = 0; t < S; ++t) fb[t * FW + n] = (uint8_t)(w[t >> 2] >> (8 * (t & 3)));
    }
}

// out[c] (c < m/32) = REDC of c_k for k = lane + 32c, canonical 26-bit limbs.
template <int m, int LR>
__device__ void i8_rmul_warp(uint32_t (&out)[m / 32][LR], const uint8_t* xb, const uint8_t* fb, uint32_t* D, int S,
                             int r, const ModRR<LR>& md, int lane) {
    const int g = lane >> 2, tig = lane & 3;
    const int FW = 2 * m + 4;
    const int rows = S + 16;
    for (int i = lane; i < rows * m; i += 32) D[i] = 0;
    __syncwarp();
    for (int ns = 0; ns < 2; ++ns) {
        // B fragments: rows i = 32 kt + 4 tig + {0..3} (+16), column s = 8 ns + g
        uint32_t bf[m / 32][2];
        const int s_col = 8 * ns + g;
#pragma unroll
        for (int kt = 0; kt < m / 32; ++kt) {
            if (s_col < S) {
                bf[kt][0] = *reinterpret_cast<const uint32_t*>(xb + s_col * m + 32 * kt + 4 * tig);
                bf[kt][1] = *reinterpret_cast<const uint32_t*>(xb + s_col * m + 32 * kt + 4 * tig + 16);
            } else {
                bf[kt][0] = bf[kt][1] = 0;
            }
        }
        for (int t = 0; t < S; ++t) {
            const uint8_t* ft = fb + t * FW;
#pragma unroll
            for (int h = 0; h < m / 16; ++h) {
                int c[4] = {0, 0, 0, 0};
                const int k0 = 16 * h + g, k1 = k0 + 8;
#pragma unroll
                for (int kt = 0; kt < m / 32; ++kt) {
                    const int i0 = 32 * kt + 4 * tig;
                    // byte offset of E_t[(k - r - i) mod 2m] in F_t for the first of 4 consecutive i
                    const int o0 = ((m - 1 - k0 + r + i0) % (2 * m) + 2 * m) % (2 * m);
                    const int o1 = ((m - 1 - k1 + r + i0) % (2 * m) + 2 * m) % (2 * m);
                    const int o2 = ((m - 1 - k0 + r + i0 + 16) % (2 * m) + 2 * m) % (2 * m);
                    const int o3 = ((m - 1 - k1 + r + i0 + 16) % (2 * m) + 2 * m) % (2 * m);
                    uint32_t a[4];
                    a[0] = ld_bytes4(ft, o0);
                    a[1] = ld_bytes4(ft, o1);
                    a[2] = ld_bytes4(ft, o2);
                    a[3] = ld_bytes4(ft, o3);
                    mma_u8_16832(c, a, bf[kt]);
                }
                // fold into diagonals d = t + s
                const int s0 = 8 * ns + 2 * tig;
                D[(t + s0) * m + k0] += (uint32_t)c[0];
                D[(t + s0 + 1) * m + k0] += (uint32_t)c[1];
                D[(t + s0) * m + k1] += (uint32_t)c[2];
                D[(t + s0 + 1) * m + k1] += (uint32_t)c[3];
                __syncwarp();
            }
        }
    }
    // recombine c_k = sum_d 256^d D[d][k] and reduce
#pragma unroll
    for (int cc = 0; cc < m / 32; ++cc) {
        const int k = lane + 32 * cc;
        constexpr int TW = 2 * LR + 1;            // 32-bit words of the integer c_k (< 2^(52 LR))
        uint32_t T[TW];
        uint64_t carry = 0;
        const int nd = 2 * S - 1;
#pragma unroll
        for (int w = 0; w < TW; ++w) {
            uint64_t acc = carry;
            for (int j = 0; j < 4; ++j) {
                const int d = 4 * w + j;
                if (d < nd) acc += (uint64_t)D[d * m + k] << (8 * j);
            }
            T[w] = (uint32_t)acc;
            carry = acc >> 32;
        }
        // 26-bit columns of T, then Montgomery reduction
        uint64_t col[2 * LR];
#pragma unroll
        for (int i = 0; i < 2 * LR; ++i) {
            const int bit = 26 * i, w = bit >> 5, sh = bit & 31;
            uint64_t v = T[w] >> sh;
            if (w + 1 < TW) v |= (uint64_t)T[w + 1] << (32 - sh);
            col[i] = v & kM26;
        }
        redc_cols<LR>(out[cc], col, md);
    }
}

}  // namespace dkss
