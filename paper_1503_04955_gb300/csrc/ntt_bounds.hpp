// Limits of the lazy arithmetic in the NTT form of the R-multiplication
// (ntt_rmul.cuh), checked on the host for one ring before a plan uses it.
//
// The transform keeps residues mod p^z unreduced between Montgomery products:
// sums are limbwise additions of 26-bit limb vectors (limbs may grow past 26
// bits) and a difference x - y is x + B - y for a bias B = K p^z whose limbs
// are each at least y's (so no limb goes negative).  ntt_lazy_bounds follows
// the worst case of every limb and of the value through the forward
// transform, the componentwise products and the backwards transform, and
// accepts the ring only if
//   * no 64-bit column of a product or of its Montgomery reduction overflows,
//   * every limb stays below 2^32,
//   * every reduction result fits its limbs, and
//   * the backwards transform ends below 2 p^z (one subtraction makes it
//     canonical).
// It also picks the smallest K for every bias.
#pragma once
#include <cstdint>

#include "host_math.hpp"

namespace dkss_planning {

struct NttBiases {
    uint32_t fwd[5];      // forward butterflies: K p^z, limbs >= those of a reduced product
    uint32_t neg[5];      // negated input coefficients: K p^z, limbs >= those of a canonical residue
    uint32_t bwd[7][5];   // backwards stage b: K_b p^z, limbs >= those of any stage input
    bool prescale;        // componentwise products scale one factor first (keeps the product in range)
    uint32_t evl[8][5];   // DFTs in evaluation coordinates, stage s: K_s p^z, limbs >= those of t
    uint32_t eval_skip;   // bit s: stage s takes t = b unreduced where its twiddle is 1
    uint32_t eval_noscale;  // bit k: after 2^k-point DFTs the product of two lazy factors
                            // fits, so the last level scales at its final reduction instead
    bool eval_ok;         // the limits of those DFTs (log2(2m) lazy stages) hold
};

// true when the lazy transform of R = (Z/qZ)[alpha]/(alpha^m + 1) with LR
// limbs of 26 bits stays within every limit above; fills *out.
bool ntt_lazy_bounds(uint32_t m, uint32_t LR, dkss_host::u128 q, NttBiases* out);

// Bias multiples of the p-adic digit form (padic.cuh): a difference x - y
// adds K (p, p-1, p-1, p-1), K p^4 = 0 mod p^4, with K (p-1) at least y's
// digits.  kf: forward stages and negated inputs; kb[b]: backwards stage b.
struct PdBiases {
    uint32_t kf = 0;
    uint32_t kb[7] = {0, 0, 0, 0, 0, 0, 0};
    bool ok = false;
    bool fast = false;   // the fast carries of ModPD<Z, true> stay within their limits too
    bool dft_ok = false; // DFTs of up to 2^7 points on digits (dft_dit_pd) stay within their limits
};

// true when the p-adic digit form with z = 4 digits (p < 2^30, residues
// stored in L <= 4 words, transforms of length m) keeps every digit below
// 2^32 and every product column below 2^64 (pd_lazy_bounds in
// ntt_bounds.cpp); fills *out.
bool pd_lazy_bounds(uint64_t p, uint32_t m, uint32_t L, PdBiases* out);

}  // namespace dkss_planning
