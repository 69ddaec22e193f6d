// Host launchers of the DKSS_MUL kernels for one (m, L) pair.
#pragma once
#include <algorithm>
#include "debug_checks.cuh"
#include "decode.cuh"
#include "dkss_kernels.cuh"
#include "eval_levels.cuh"
#include "plan.hpp"

namespace dkss {

template <int L>
static Mod<L> make_mod(const dkss_plan_s* pl) {
    Mod<L> md;
    for (int i = 0; i < L; ++i) md.q[i] = pl->q_limbs[i];
    md.nprime = pl->nprime;
    md.nsub = pl->nsub;
    return md;
}

template <int LR, class MR = ModRR<LR>>
static MR make_modrr(const dkss_plan_s* pl) {
    MR md;
    for (int i = 0; i < LR; ++i) md.q[i] = pl->q_rr[i];
    md.nprime = pl->nprime26;
    md.qtop_inv = qtop_reciprocal(pl->q_rr[LR - 1], pl->q_rr[LR - 2]);
    return md;
}

// Modulus constants of the NTT-form kernels: 26-bit-limb Montgomery
// (ModRR, ModRRSparse) or p-adic digits (ModPD, padic.cuh).
template <int LR, class MR>
static MR make_mr(const dkss_plan_s* pl) {
    if constexpr (IsPD<MR>::value) {
        MR md;
        md.p = (uint32_t)pl->p;
        md.nmu = pl->pd_nmu;
        md.nsh = pl->pd_s + 1;
        md.mu_lo = pl->pd_mu_lo;
        md.lg_nmu = pl->pd_lg_nmu;
        md.s = pl->pd_s;
        md.mu = pl->pd_mu;
        return md;
    } else {
        return make_modrr<LR, MR>(pl);
    }
}

static LevelParams make_level(const dkss_plan_s* pl) {
    LevelParams lp{};
    lp.data = pl->d_work;
    lp.table = pl->d_table;
    lp.poly_words = pl->poly_words;
    lp.P2 = pl->P2;
    lp.mu_top = pl->mu_top;
    lp.M = pl->M;
    lp.n_bits = pl->n_bits;
    lp.raw_words = (pl->n_bits + 63) / 64;
    lp.u = pl->u;
    lp.log2_mu_top = pl->log2_mu_top;
    for (int i = 0; i < 5; ++i) lp.kscale[i] = pl->kscale[i];
    lp.table_eval = pl->d_table;
    lp.ntt_cst = pl->d_ntt;
    lp.i8_S = pl->i8_S;
    lp.ntt_prescale = pl->ntt_bias.prescale ? 1u : 0u;
    lp.eval_skip = pl->ntt_bias.eval_skip;
    lp.dft_lazy = pl->dft_lazy ? 1u : 0u;
    lp.red_rcp = pl->red_rcp;
    lp.pd_io = pl->pd_io ? 1u : 0u;
    lp.pd_fast = pl->pd_fast ? 1u : 0u;
    if (pl->pd_io) {
        lp.pd = make_mr<kPdDigits, ModPD<kPdDigits>>(pl);
        lp.pd_pw = pl->d_ntt + pl->pd_pw_off;
    }
    {
        uint32_t k = 0;
        while ((1ull << k) < pl->r_last) ++k;
        lp.eval_noscale = (pl->ntt_bias.eval_noscale >> k) & 1;
    }
    return lp;
}

// Last forward level alone (root alpha^(2m/len)), for stage output.
template <int m, int L>
__global__ void __launch_bounds__(kThreads) k_final_dft(LevelParams prm, Mod<L> md) {
    using G = Geo<m, L>;
    extern __shared__ __align__(16) uint32_t smem[];
    const int n = (int)prm.len;
    const int log2n = 31 - __clz(n);
    const uint64_t base = (uint64_t)blockIdx.x * n;
    for (int idx = threadIdx.x; idx < n * m; idx += kThreads) {
        int j = idx / m, t = idx % m;
        uint32_t x[L];
        ld_res<L>(x, prm.data + ((base + j) * m + t) * L);
        if constexpr (L == kPdDigits) {
            if (prm.pd_io) {   // the forward levels left canonical p-adic digits
                uint32_t w[L];
                pd_to_words<L, L>(w, x, prm.pd);
#pragma unroll
                for (int k = 0; k < L; ++k) x[k] = w[k];
            }
        }
        st_res<L>(smem + bitrev(j, log2n) * G::ES + t * L, x);
    }
    __syncthreads();
    dft_dit<m, L>(smem, 1, n, G::TWO_M / n, md);
    for (int idx = threadIdx.x; idx < n * m; idx += kThreads) {
        int j = idx / m, t = idx % m;
        uint32_t x[L];
        ld_res<L>(x, smem + j * G::ES + t * L);
        st_res<L>(prm.data + ((base + j) * m + t) * L, x);
    }
}

// Natural-order copy of a transformed polynomial: frequency i sits at the
// digit-reversed position sum_d v_d * (2M/(2m)^d) + f, where
// i = v_1 + 2m v_2 + ... + (2m)^levels f.
template <int m, int L>
__global__ void k_unpermute(const uint32_t* src, uint64_t* dst, uint64_t P2, uint32_t levels) {
    uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P2 * m) return;
    uint64_t i = idx / m;
    uint32_t t = (uint32_t)(idx % m);
    uint64_t rest = i, pos = 0, mu = P2;
    for (uint32_t d = 0; d < levels; ++d) {
        mu /= 2 * m;
        pos += (rest % (2 * m)) * mu;
        rest /= 2 * m;
    }
    pos += rest;
    const uint32_t* s = src + (pos * m + t) * L;
    uint64_t lo = s[0] | (L > 1 ? (uint64_t)s[1] << 32 : 0);
    uint64_t hi = (L > 2 ? s[2] : 0) | (L > 3 ? (uint64_t)s[3] << 32 : 0);
    dst[2 * idx] = lo;
    dst[2 * idx + 1] = hi;
}

#define DKSS_CHECK_LAUNCH()                          \
    do {                                             \
        if (cudaGetLastError() != cudaSuccess) return DKSS_ECUDA; \
    } while (0)

// DKSS_DEBUG_CHECKS: every residue of n_res residues at poly is below p^z
// (debug_checks.cuh); a failure sets kStatusRange in the plan's status word.
template <int L>
static dkss_status range_check(dkss_plan_s* pl, const uint32_t* poly, uint64_t n_res, cudaStream_t st,
                               bool digits = false) {
    if (!(pl->flags & DKSS_DEBUG_CHECKS)) return DKSS_OK;
    RangeParams rp{};
    rp.poly = poly;
    rp.n_res = n_res;
    for (int i = 0; i < 4; ++i) rp.q[i] = pl->q_limbs[i];
    rp.digit_p = digits ? (uint32_t)pl->p : 0u;
    rp.status = pl->d_status;
    const uint64_t blocks = std::min<uint64_t>((n_res + 255) / 256, (uint64_t)pl->sm_count * 8);
    k_check_range<L><<<(unsigned)std::max<uint64_t>(1, blocks), 256, 0, st>>>(rp);
    DKSS_CHECK_LAUNCH();
    return DKSS_OK;
}

// Test hook (DKSS_FAULT_RANGE, host side): overwrite residue 0 of the first
// polynomial with 2^(32L) - 1, which is above p^z, by a host-to-device copy
// queued on the stream.  The range check that follows must report it.
template <int L>
static dkss_status inject_range_fault(dkss_plan_s* pl, cudaStream_t st) {
    if (!(dkss_planning::fault_mask() & DKSS_FAULT_RANGE)) return DKSS_OK;
    static const uint32_t bad[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
    if (cudaMemcpyAsync(pl->d_work, bad, L * sizeof(uint32_t), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return DKSS_ECUDA;
    return DKSS_OK;
}

// Columns of more than 64 KiB (m = 64, L >= 3) run their DFTs in halves
// (k_dft_fwd_half, k_dft_inv_half): three or four CTAs per SM instead of one
// or two.
template <int m, int L>
constexpr bool half_columns() {
    return column_smem_bytes<m, L>() > 64 * 1024;
}

// The NTT form's kernels take the sparse-modulus Montgomery product when the
// plan's p^z allows it (Proth primes, dkss_plan_proth; ntt_rmul.cuh).
template <int LR>
static bool sparse_ntt(const dkss_plan_s* pl) {
    return LR >= 3 && pl->q_sparse && !(pl->flags & (DKSS_RMUL_DIRECT | DKSS_FORM_INT8TC));
}

// The NTT form runs each radix-2m level as one fused kernel (column DFT and
// its R-multiplications) when a column and the exchange buffers fit three or
// more CTAs per SM; bigger columns (m = 64 with 4-word residues) keep the
// separate DFT and element-parallel twiddle kernels.
template <int m, int L, int LR>
static bool fused_levels(const dkss_plan_s* pl) {
    return !(pl->flags & (DKSS_RMUL_DIRECT | DKSS_FORM_INT8TC)) && level_ntt_smem_bytes<m, L, LR>() <= 64 * 1024;
}

template <int m, int L, int LR>
dkss_status prepare(dkss_plan_s* pl) {
    using G = Geo<m, L>;
    const int colb = (int)column_smem_bytes<m, L>();
    const int twb = (int)twiddle_smem_bytes<m, L, LR>();
    const bool direct = (pl->flags & (DKSS_RMUL_DIRECT | DKSS_FORM_INT8TC)) != 0;
    const int fin = (int)final_smem_bytes<m, L, LR>((int)pl->r_last, direct ? kFormDirect : kFormNtt);
    const int twn = (int)twiddle_ntt_smem_bytes<m, L, LR>();
    const int lvl = (int)level_ntt_smem_bytes<m, L, LR>();
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device) != cudaSuccess)
        return DKSS_ECUDA;
    if (colb > optin || twb > optin || twn > optin || fin > optin || lvl > optin) return DKSS_EUNSUPPORTED;
    if (pl->flags & DKSS_FORM_INT8TC) {
        if constexpr (m >= 32) {
            // INT8 form: sized for the largest byte count (16), shared by all plans of this kind
            const int i8tw = (int)twiddle_i8_smem_bytes<m, L, LR>(16);
            const int i8fin = (int)final_smem_bytes<m, L, LR>((int)pl->r_last, kFormI8, (int)pl->i8_S);
            const int i8fin_max = (int)std::min<size_t>(final_smem_bytes<m, L, LR>(G::TWO_M, kFormI8, 16), (size_t)optin);
            if (i8tw > optin || i8fin > optin) return DKSS_EUNSUPPORTED;
            if (cudaFuncSetAttribute(k_twiddle_i8<m, L, LR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, i8tw) ||
                cudaFuncSetAttribute(k_twiddle_i8<m, L, LR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, i8tw) ||
                cudaFuncSetAttribute(k_final_pointwise<m, L, LR, kFormI8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     i8fin_max))
                return DKSS_ECUDA;
        } else {
            return DKSS_EUNSUPPORTED;   // the INT8 form needs a warp per element (m >= 32)
        }
    }
    // The limit is a property of the kernel, shared by every plan of this
    // (m, L, LR): set it to the most any plan can ask for (last level of
    // length 2m), capped by the device, so that no plan lowers another's.
    const int fin_max = (int)std::min<size_t>(final_smem_bytes<m, L, LR>(G::TWO_M), (size_t)optin);
    const int fin_ntt_max = (int)std::min<size_t>(final_smem_bytes<m, L, LR>(G::TWO_M, kFormNtt), (size_t)optin);
    const int fdft_max = (int)std::min<size_t>(sizeof(uint32_t) * G::TWO_M * G::ES, (size_t)optin);
    if (cudaFuncSetAttribute(k_dft_fwd<m, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, colb) ||
        cudaFuncSetAttribute(k_dft_fwd<m, L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, colb) ||
        cudaFuncSetAttribute(k_dft_inv<m, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, colb) ||
        cudaFuncSetAttribute(k_twiddle<m, L, LR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, twb) ||
        cudaFuncSetAttribute(k_twiddle<m, L, LR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, twb) ||
        cudaFuncSetAttribute(k_final_pointwise<m, L, LR, kFormDirect>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             fin_max) ||
        cudaFuncSetAttribute(k_final_pointwise<m, L, LR, kFormNtt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             fin_ntt_max) ||
        cudaFuncSetAttribute(k_level_fwd_ntt<m, L, LR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lvl) ||
        cudaFuncSetAttribute(k_level_fwd_ntt<m, L, LR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lvl) ||
        cudaFuncSetAttribute(k_level_inv_ntt<m, L, LR>, cudaFuncAttributeMaxDynamicSharedMemorySize, lvl) ||
        cudaFuncSetAttribute(k_twiddle_ntt<m, L, LR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, twn) ||
        cudaFuncSetAttribute(k_twiddle_ntt<m, L, LR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, twn) ||
        cudaFuncSetAttribute(k_final_dft<m, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, fdft_max))
        return DKSS_ECUDA;
    if constexpr (half_columns<m, L>()) {
        // persistent grids of the half-column DFTs and one scratch slice per CTA
        const int hb = (int)half_column_smem_bytes<m, L>();
        int occ_f = 0, occ_i = 0;
        if (cudaFuncSetAttribute(k_dft_fwd_half<m, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hb) ||
            cudaFuncSetAttribute(k_dft_fwd_half<m, L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, hb) ||
            cudaFuncSetAttribute(k_dft_inv_half<m, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, hb) ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, k_dft_fwd_half<m, L, true>, kThreads, hb) ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_i, k_dft_inv_half<m, L>, kThreads, hb) || occ_f < 1 ||
            occ_i < 1)
            return DKSS_ECUDA;
        pl->half_grid_fwd = occ_f * pl->sm_count;
        pl->half_grid_inv = occ_i * pl->sm_count;
        if (!pl->d_half) {
            const size_t words = (size_t)std::max(pl->half_grid_fwd, pl->half_grid_inv) * m * G::EW;
            if (cudaMalloc(&pl->d_half, words * sizeof(uint32_t)) != cudaSuccess) {
                cudaGetLastError();
                return DKSS_ENOMEM;
            }
            pl->dev_bytes += words * sizeof(uint32_t);
        }
    }
    if constexpr (LR >= 3) {
        using MS = ModRRSparse<LR>;
        if (sparse_ntt<LR>(pl) &&
            (cudaFuncSetAttribute(k_final_pointwise<m, L, LR, kFormNtt, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  fin_ntt_max) ||
             cudaFuncSetAttribute(k_level_fwd_ntt<m, L, LR, true, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize, lvl) ||
             cudaFuncSetAttribute(k_level_fwd_ntt<m, L, LR, false, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize, lvl) ||
             cudaFuncSetAttribute(k_level_inv_ntt<m, L, LR, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize, lvl) ||
             cudaFuncSetAttribute(k_twiddle_ntt<m, L, LR, false, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize, twn) ||
             cudaFuncSetAttribute(k_twiddle_ntt<m, L, LR, true, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize, twn)))
            return DKSS_ECUDA;
    }
    if constexpr (m == 64) {
        if (pl->padic) {
            constexpr int Z = kPdDigits;
            const int twp = (int)twiddle_ntt_smem_bytes<m, L, Z>();
            const int finp = (int)std::min<size_t>(final_smem_bytes<m, L, Z>(G::TWO_M, kFormNtt), (size_t)optin);
            if ((int)final_smem_bytes<m, L, Z>((int)pl->r_last, kFormNtt) > optin || twp > optin)
                return DKSS_EUNSUPPORTED;
            auto set = [&](auto pd) {
                using PD = decltype(pd);
                return cudaFuncSetAttribute(k_twiddle_ntt<m, L, Z, false, PD>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, twp) ||
                       cudaFuncSetAttribute(k_twiddle_ntt<m, L, Z, true, PD>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, twp) ||
                       cudaFuncSetAttribute(k_final_pointwise<m, L, Z, kFormNtt, PD>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, finp);
            };
            if (pl->pd_fast ? set(ModPD<Z, true>{}) : set(ModPD<Z, false>{})) return DKSS_ECUDA;
        }
    }
    if constexpr (m <= 32) {
        if (pl->eval_levels) {
            const int fe = (int)std::min<size_t>(final_eval_smem_bytes<m, L, LR>(G::TWO_M), (size_t)optin);
            if ((int)final_eval_smem_bytes<m, L, LR>((int)pl->r_last) > optin) return DKSS_EUNSUPPORTED;
            if (cudaFuncSetAttribute(k_level0_fwd_eval<m, L, LR>, cudaFuncAttributeMaxDynamicSharedMemorySize, lvl) ||
                cudaFuncSetAttribute(k_level0_inv_eval<m, L, LR>, cudaFuncAttributeMaxDynamicSharedMemorySize, lvl) ||
                cudaFuncSetAttribute(k_final_eval<m, L, LR>, cudaFuncAttributeMaxDynamicSharedMemorySize, fe))
                return DKSS_ECUDA;
        }
    }
    // launches per dkss_mul: per radix-2m level a DFT and a twiddle launch forward
    // and backwards, the fused last level, three decode kernels
    // (the NTT form fuses each level's DFT and R-multiplications into one launch)
    // (DKSS_DEBUG_CHECKS adds three range checks, one before decoding with
    // the levels in evaluation coordinates)
    pl->launches = (fused_levels<m, L, LR>(pl) ? 2 : 4) * pl->col_levels + 1 + 3 +
                   ((pl->flags & DKSS_DEBUG_CHECKS) ? (pl->eval_levels ? 1 : 3) : 0);
    return DKSS_OK;
}

// Block length and twiddle base power of radix-2m level d (0-based).
static inline void level_geometry(const dkss_plan_s* pl, uint32_t d, uint64_t* len, uint64_t* bp) {
    uint64_t b = 1;
    for (uint32_t i = 0; i < d; ++i) b *= 2 * pl->m;
    *bp = b;
    *len = pl->P2 / b;
}

template <int m, int L, int LR, bool INV, class MR = ModRR<LR>>
static dkss_status launch_twiddle(dkss_plan_s* pl, LevelParams lp, int operands, cudaStream_t st) {
    using G = Geo<m, L>;
    const MR mr = make_mr<LR, MR>(pl);
    const uint64_t mu_d = lp.len / G::TWO_M;
    const uint64_t total = (uint64_t)(G::TWO_M - 1) * (mu_d - 1) * (pl->P2 / lp.len);
    if (total == 0) return DKSS_OK;
    dim3 grid((unsigned)((total + G::NTEAMS - 1) / G::NTEAMS), operands);
    if constexpr (IsPD<MR>::value) {
        dim3 gn((unsigned)((pl->P2 + NttTeam<m>::NTEAMS - 1) / NttTeam<m>::NTEAMS), operands);
        k_twiddle_ntt<m, L, LR, INV, MR><<<gn, kThreads, twiddle_ntt_smem_bytes<m, L, LR>(), st>>>(lp, mr);
    } else if (pl->flags & DKSS_FORM_INT8TC) {
        if constexpr (m >= 32) {
            dim3 g8((unsigned)((total + kWarps - 1) / kWarps), operands);
            k_twiddle_i8<m, L, LR, INV><<<g8, kThreads, twiddle_i8_smem_bytes<m, L, LR>((int)pl->i8_S), st>>>(lp, mr);
        }
    } else if (pl->flags & DKSS_RMUL_DIRECT)
        k_twiddle<m, L, LR, INV><<<grid, kThreads, twiddle_smem_bytes<m, L, LR>(), st>>>(lp, mr);
    else {
        // one team per element of the level (those with twiddle 1 return at once)
        dim3 gn((unsigned)((pl->P2 + NttTeam<m>::NTEAMS - 1) / NttTeam<m>::NTEAMS), operands);
        k_twiddle_ntt<m, L, LR, INV, MR><<<gn, kThreads, twiddle_ntt_smem_bytes<m, L, LR>(), st>>>(lp, mr);
    }
    DKSS_CHECK_LAUNCH();
    return DKSS_OK;
}

template <int m, int L, int LR, class MR = ModRR<LR>>
static dkss_status launch_forward_levels(dkss_plan_s* pl, LevelParams lp, int operands, cudaStream_t st) {
    using G = Geo<m, L>;
    const Mod<L> md = make_mod<L>(pl);
    dim3 grid((unsigned)(pl->P2 / G::TWO_M), operands);
    const bool fused = !IsPD<MR>::value && fused_levels<m, L, LR>(pl);
    for (uint32_t d = 0; d < pl->col_levels; ++d) {
        level_geometry(pl, d, &lp.len, &lp.bp);
        if constexpr (!IsPD<MR>::value) {
            if (fused) {   // inner DFT and R-multiplications of a column in one kernel (NTT form)
                ProfScope ps(pl, st, kProfFwdTwiddle);
                const MR mr = make_modrr<LR, MR>(pl);
                if (d == 0)
                    k_level_fwd_ntt<m, L, LR, true, MR><<<grid, kThreads, level_ntt_smem_bytes<m, L, LR>(), st>>>(lp, md, mr);
                else
                    k_level_fwd_ntt<m, L, LR, false, MR><<<grid, kThreads, level_ntt_smem_bytes<m, L, LR>(), st>>>(lp, md,
                                                                                                                 mr);
                DKSS_CHECK_LAUNCH();
                continue;
            }
        }
        {
            ProfScope ps(pl, st, kProfFwdDft);
            if constexpr (half_columns<m, L>()) {
                const size_t hb = half_column_smem_bytes<m, L>();
                const unsigned hg = (unsigned)std::min<uint64_t>(pl->half_grid_fwd, (pl->P2 / G::TWO_M) * operands);
                if (d == 0) k_dft_fwd_half<m, L, true><<<hg, kThreads, hb, st>>>(lp, md, pl->d_half, operands);
                else k_dft_fwd_half<m, L, false><<<hg, kThreads, hb, st>>>(lp, md, pl->d_half, operands);
            } else {
                if (d == 0) k_dft_fwd<m, L, true><<<grid, kThreads, column_smem_bytes<m, L>(), st>>>(lp, md);
                else k_dft_fwd<m, L, false><<<grid, kThreads, column_smem_bytes<m, L>(), st>>>(lp, md);
            }
            DKSS_CHECK_LAUNCH();
        }
        ProfScope ps(pl, st, kProfFwdTwiddle);
        dkss_status s = launch_twiddle<m, L, LR, false, MR>(pl, lp, operands, st);
        if (s != DKSS_OK) return s;
    }
    return DKSS_OK;
}

// Decoding and carry propagation of the product polynomial in the plan's workspace.
template <int m, int L, int LR>
static dkss_status launch_decode(dkss_plan_s* pl, uint64_t* out, cudaStream_t st) {
    DecodeParams dp{};
    dp.c = pl->d_work;
    dp.out = reinterpret_cast<uint32_t*>(out);
    dp.agg = pl->d_agg;
    dp.status = pl->d_status;
    dp.P2 = pl->P2;
    dp.n_windows = 4 * ((pl->n_bits + 63) / 64);
    dp.n_tiles = pl->n_tiles;
    dp.k_max = pl->P2 * (m / 2) + m / 2;
    dp.m = m;
    dp.h = m / 2;
    dp.u = pl->u;
    dp.db = 0;
    for (dkss_host::u128 t = pl->q; t; t >>= 1) dp.db++;
    dp.db += 1;
    dp.out_aligned16 = ((uintptr_t)out & 15) == 0;
    ProfScope ps(pl, st, kProfDecode);
    if (pl->u == 32) k_decode_tiles_aligned<L, 1><<<(unsigned)pl->n_tiles, kDecThreads, 0, st>>>(dp);
    else if (pl->u == 16) k_decode_tiles_aligned<L, 2><<<(unsigned)pl->n_tiles, kDecThreads, 0, st>>>(dp);
    else k_decode_tiles<L><<<(unsigned)pl->n_tiles, kDecThreads, 0, st>>>(dp);
    DKSS_CHECK_LAUNCH();
    k_decode_scan<<<1, kScanThreads, 0, st>>>(dp);
    DKSS_CHECK_LAUNCH();
    k_decode_fix<<<(unsigned)((pl->n_tiles + 255) / 256), 256, 0, st>>>(dp);
    DKSS_CHECK_LAUNCH();
    return DKSS_OK;
}

// Inner levels in evaluation coordinates: level 0 forward, levels >= 1 and the last level in
// evaluation coordinates, level 0 backwards (eval_levels.cuh).
template <int m, int L, int LR>
static dkss_status run_eval_levels(dkss_plan_s* pl, LevelParams lp, cudaStream_t st) {
    using G = Geo<m, L>;
    const Mod<L> md = make_mod<L>(pl);
    const ModRR<LR> mr = make_modrr<LR>(pl);
    const unsigned cols = (unsigned)(pl->P2 / G::TWO_M);
    const unsigned slices = (unsigned)(m / EvalKC<m>::value);
    for (uint32_t d = 0; d < pl->col_levels; ++d) {
        {
            ProfScope ps(pl, st, kProfFwdTwiddle);
            level_geometry(pl, d, &lp.len, &lp.bp);
            if (d == 0) {
                k_level0_fwd_eval<m, L, LR><<<dim3(cols, 2), kThreads, level_ntt_smem_bytes<m, L, LR>(), st>>>(lp, md, mr);
            } else {
                lp.tw_lvl = pl->d_evtw + pl->evtw_offs[d];
                k_level_eval_fwd<m, L, LR><<<dim3(cols, slices, 2), kThreads, level_eval_smem_bytes<m, L, LR>(), st>>>(
                    lp, mr);
            }
            DKSS_CHECK_LAUNCH();
        }
    }
    lp.len = pl->r_last;
    {
        ProfScope ps(pl, st, kProfFinal);
        const unsigned blocks = (unsigned)(pl->P2 / final_eval_elems<m>((int)pl->r_last));
        k_final_eval<m, L, LR><<<dim3(blocks, slices), kThreads, final_eval_smem_bytes<m, L, LR>((int)pl->r_last), st>>>(
            lp, mr);
        DKSS_CHECK_LAUNCH();
    }
    for (int d = (int)pl->col_levels - 1; d >= 0; --d) {
        ProfScope ps(pl, st, kProfInvTwiddle);
        level_geometry(pl, (uint32_t)d, &lp.len, &lp.bp);
        if (d == 0) {
            k_level0_inv_eval<m, L, LR><<<cols, kThreads, level_ntt_smem_bytes<m, L, LR>(), st>>>(lp, md, mr);
        } else {
            lp.tw_lvl = pl->d_evtw + pl->evtw_offs[d];
            k_level_eval_inv<m, L, LR><<<dim3(cols, slices), kThreads, level_eval_smem_bytes<m, L, LR>(), st>>>(lp, mr);
        }
        DKSS_CHECK_LAUNCH();
    }
    return DKSS_OK;
}

// A product with every radix-2m level on coefficients (the thesis's
// structure); MR is the modulus type of the NTT-form kernels (ModRRSparse for
// a sparse Proth modulus, ntt_rmul.cuh).
template <int m, int L, int LR, class MR>
static dkss_status run_mul_coef(dkss_plan_s* pl, const uint64_t* a, const uint64_t* b, uint64_t* out, cudaStream_t st) {
    using G = Geo<m, L>;
    const Mod<L> md = make_mod<L>(pl);
    const MR mr = make_mr<LR, MR>(pl);
    LevelParams lp = make_level(pl);
    lp.raw_a = a;
    lp.raw_b = b;
    dkss_status s = DKSS_OK;
    // a square (a == b) transforms one polynomial; the last level reads it as both factors
    const bool square = a == b;
    s = launch_forward_levels<m, L, LR, MR>(pl, lp, square ? 1 : 2, st);
    if (s != DKSS_OK) return s;
    if ((s = inject_range_fault<L>(pl, st)) != DKSS_OK) return s;
    // both transformed operands (b directly follows a); p-adic digits where the forward levels keep them
    if ((s = range_check<L>(pl, pl->d_work, (square ? 1 : 2) * pl->P2 * m, st, pl->pd_io)) != DKSS_OK) return s;
    lp.len = pl->r_last;
    if (square) {
        lp.poly_words = 0;
        lp.square = 1;
    }
    {
        ProfScope ps(pl, st, kProfFinal);
        const unsigned blocks = (unsigned)(pl->P2 / pl->r_last);
        const unsigned nblocks = blocks / (unsigned)final_blocks_per_cta<m>((int)pl->r_last);
        if constexpr (IsPD<MR>::value) {
            k_final_pointwise<m, L, LR, kFormNtt, MR>
                <<<nblocks, kThreads, final_smem_bytes<m, L, LR>((int)pl->r_last, kFormNtt), st>>>(lp, md, mr);
        } else if (pl->flags & DKSS_FORM_INT8TC) {
            const ModRR<LR> mr0 = make_modrr<LR>(pl);
            if constexpr (m >= 32)
                k_final_pointwise<m, L, LR, kFormI8>
                    <<<blocks, kThreads, final_smem_bytes<m, L, LR>((int)pl->r_last, kFormI8, (int)pl->i8_S), st>>>(
                        lp, md, mr0);
        } else if (pl->flags & DKSS_RMUL_DIRECT) {
            const ModRR<LR> mr0 = make_modrr<LR>(pl);
            k_final_pointwise<m, L, LR, kFormDirect><<<blocks, kThreads, final_smem_bytes<m, L, LR>((int)pl->r_last), st>>>(
                lp, md, mr0);
        } else {
            k_final_pointwise<m, L, LR, kFormNtt, MR>
                <<<nblocks, kThreads, final_smem_bytes<m, L, LR>((int)pl->r_last, kFormNtt), st>>>(lp, md, mr);
        }
        DKSS_CHECK_LAUNCH();
    }
    lp.poly_words = pl->poly_words;
    lp.square = 0;
    if ((s = range_check<L>(pl, pl->d_work, pl->P2 * m, st)) != DKSS_OK) return s;
    const bool fused = !IsPD<MR>::value && fused_levels<m, L, LR>(pl);
    for (int d = (int)pl->col_levels - 1; d >= 0; --d) {
        level_geometry(pl, (uint32_t)d, &lp.len, &lp.bp);
        if constexpr (!IsPD<MR>::value) {
            if (fused) {   // R-multiplications and inner DFT of a column in one kernel (NTT form)
                ProfScope ps(pl, st, kProfInvTwiddle);
                k_level_inv_ntt<m, L, LR, MR><<<(unsigned)(pl->P2 / G::TWO_M), kThreads,
                                               level_ntt_smem_bytes<m, L, LR>(), st>>>(lp, md, mr);
                DKSS_CHECK_LAUNCH();
                continue;
            }
        }
        {
            ProfScope ps(pl, st, kProfInvTwiddle);
            s = launch_twiddle<m, L, LR, true, MR>(pl, lp, 1, st);
            if (s != DKSS_OK) return s;
        }
        ProfScope ps(pl, st, kProfInvDft);
        if constexpr (half_columns<m, L>()) {
            const unsigned hg = (unsigned)std::min<uint64_t>(pl->half_grid_inv, pl->P2 / G::TWO_M);
            k_dft_inv_half<m, L><<<hg, kThreads, half_column_smem_bytes<m, L>(), st>>>(lp, md, pl->d_half);
        } else {
            k_dft_inv<m, L><<<(unsigned)(pl->P2 / G::TWO_M), kThreads, column_smem_bytes<m, L>(), st>>>(lp, md);
        }
        DKSS_CHECK_LAUNCH();
    }
    // the product polynomial's coefficients, before decoding
    if ((s = range_check<L>(pl, pl->d_work, pl->P2 * m, st)) != DKSS_OK) return s;
    return launch_decode<m, L, LR>(pl, out, st);
}

template <int m, int L, int LR>
dkss_status run_mul(dkss_plan_s* pl, const uint64_t* a, const uint64_t* b, uint64_t* out, cudaStream_t st) {
    if constexpr (m <= 32) {
        if (pl->eval_levels) {
            LevelParams lp = make_level(pl);
            lp.raw_a = a;
            lp.raw_b = b;
            dkss_status s = run_eval_levels<m, L, LR>(pl, lp, st);
            if (s != DKSS_OK) return s;
            s = range_check<L>(pl, pl->d_work, pl->P2 * m, st);
            if (s != DKSS_OK) return s;
            return launch_decode<m, L, LR>(pl, out, st);
        }
    }
    if constexpr (m == 64) {
        if (pl->padic && pl->pd_fast) return run_mul_coef<m, L, kPdDigits, ModPD<kPdDigits, true>>(pl, a, b, out, st);
        if (pl->padic) return run_mul_coef<m, L, kPdDigits, ModPD<kPdDigits>>(pl, a, b, out, st);
    }
    if constexpr (LR >= 3) {
        if (sparse_ntt<LR>(pl)) return run_mul_coef<m, L, LR, ModRRSparse<LR>>(pl, a, b, out, st);
    }
    return run_mul_coef<m, L, LR, ModRR<LR>>(pl, a, b, out, st);
}

template <int m, int L, int LR>
dkss_status run_forward(dkss_plan_s* pl, const uint64_t* a, uint64_t* out, cudaStream_t st) {
    using G = Geo<m, L>;
    const Mod<L> md = make_mod<L>(pl);
    LevelParams lp = make_level(pl);
    lp.raw_a = a;
    lp.raw_b = a;
    if (pl->d_table_minv) lp.table_eval = pl->d_table_minv;   // coefficient levels for a plan in evaluation coordinates
    dkss_status s = DKSS_OK;
    if constexpr (m == 64) {
        if (pl->padic && pl->pd_fast) s = launch_forward_levels<m, L, kPdDigits, ModPD<kPdDigits, true>>(pl, lp, 1, st);
        else if (pl->padic) s = launch_forward_levels<m, L, kPdDigits, ModPD<kPdDigits>>(pl, lp, 1, st);
        else s = launch_forward_levels<m, L, LR>(pl, lp, 1, st);
    } else {
        s = launch_forward_levels<m, L, LR>(pl, lp, 1, st);
    }
    if (s != DKSS_OK) return s;
    lp.len = pl->r_last;
    k_final_dft<m, L><<<(unsigned)(pl->P2 / pl->r_last), kThreads, sizeof(uint32_t) * pl->r_last * G::ES, st>>>(lp, md);
    DKSS_CHECK_LAUNCH();
    uint64_t total = pl->P2 * m;
    k_unpermute<m, L><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(pl->d_work, out, pl->P2, pl->col_levels);
    DKSS_CHECK_LAUNCH();
    return DKSS_OK;
}

}  // namespace dkss

#define DKSS_INSTANTIATE(M_, L_, LR_)                                                                        \
    template dkss_status dkss::run_mul<M_, L_, LR_>(dkss_plan_s*, const uint64_t*, const uint64_t*, uint64_t*, \
                                                   cudaStream_t);                                               \
    template dkss_status dkss::run_forward<M_, L_, LR_>(dkss_plan_s*, const uint64_t*, uint64_t*, cudaStream_t); \
    template dkss_status dkss::prepare<M_, L_, LR_>(dkss_plan_s*);
