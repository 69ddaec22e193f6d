// Many products of uneven sizes in one persistent kernel launch.
//
// A batch groups its jobs into size classes that share the limb layout (m,
// L, LR) and each have their own ring (p, z), M and u; the ring's constants
// travel with every job.  The persistent kernel walks a
// host-built list of stages (per level the fused column DFT and its
// R-multiplications, forward; the fused last level with the componentwise
// products; per level backwards the fused R-multiplications and column DFT;
// decode tiles, carry scan, carry fix-up).  In each stage
// every CTA takes work items -- a column, a group of elements, a block, a
// tile -- from all jobs at once, then the grid synchronises (a cooperative
// launch keeps every CTA resident, so the grid barrier cannot wait on a CTA
// that is not running).  Each job's stages keep the order of a single
// product; a job with fewer levels simply has no items in the others.
#pragma once
#include <cooperative_groups.h>

#include <cstdint>

#include "decode.cuh"
#include "dkss_kernels.cuh"

namespace dkss {

enum BatchStageType : uint32_t {
    kStFwdDft = 0,
    kStFwdTwiddle = 1,
    kStFinal = 2,
    kStInvTwiddle = 3,
    kStInvDft = 4,
    kStDecTiles = 5,
    kStDecScan = 6,
    kStDecFix = 7,
    kStFwdLevel = 8,    // column DFT and its R-multiplications fused (level_fwd_ntt)
    kStInvLevel = 9     // R-multiplications and column DFT fused (level_inv_ntt)
};

// Per-job parameters (device copy).  lp.len / lp.bp are set per stage.
struct BatchJob {
    LevelParams lp;
    DecodeParams dp;
    uint32_t col_levels;
    uint32_t r_last;
    // the job's ring Z/p^zZ: p^z in 32-bit limbs (Mod) and 26-bit limbs (ModRR)
    uint32_t q32[4];
    uint32_t nprime32, nsub;
    uint32_t q26[5];
    uint32_t nprime26;
    uint64_t qtop_inv26;
};

struct BatchStage {
    uint32_t type;
    uint32_t level;          // radix-2m level for DFT / twiddle stages
    uint64_t total;          // work items over all jobs
    const uint64_t* offs;    // count + 1 exclusive prefix sums of per-job items
};

// Work items of one job in one stage (host and device agree on this count).
template <int m>
__host__ __device__ inline uint64_t batch_items(uint32_t type, uint32_t level, uint64_t P2, uint32_t col_levels,
                                                uint64_t r_last, uint64_t n_tiles, int nteams) {
    const uint64_t cols = P2 / (2 * m);
    uint64_t len = P2;
    for (uint32_t i = 0; i < level; ++i) len /= 2 * m;
    const uint64_t mu_d = len / (2 * m);
    // NTT-form twiddle stages: one team per element of the level
    const uint64_t groups = mu_d > 1 ? (P2 + nteams - 1) / nteams : 0;
    switch (type) {
        case kStFwdDft: return level < col_levels ? 2 * cols : 0;
        case kStFwdTwiddle: return level < col_levels ? 2 * groups : 0;
        case kStFinal: return P2 / (r_last * final_blocks_per_cta<m>((int)r_last));
        case kStInvTwiddle: return level < col_levels ? groups : 0;
        case kStInvDft: return level < col_levels ? cols : 0;
        case kStDecTiles: return n_tiles;
        case kStDecScan: return 1;
        case kStDecFix: return (n_tiles + kThreads - 1) / kThreads;
        case kStFwdLevel: return level < col_levels ? 2 * cols : 0;
        case kStInvLevel: return level < col_levels ? cols : 0;
    }
    return 0;
}

template <int m, int L, int LR, class MR>
__global__ void __launch_bounds__(kThreads, 2) k_batch(const BatchJob* __restrict__ jobs, const BatchStage* __restrict__ stages,
                                                    uint32_t n_stages, uint32_t count) {
    using G = Geo<m, L>;
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) uint32_t smem[];
    cg::grid_group grid = cg::this_grid();
    for (uint32_t s = 0; s < n_stages; ++s) {
        const BatchStage st = stages[s];
        for (uint64_t item = blockIdx.x; item < st.total; item += gridDim.x) {
            uint32_t lo = 0, hi = count;   // last job with offs[job] <= item
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) / 2;
                if (st.offs[mid] <= item) lo = mid;
                else hi = mid;
            }
            const BatchJob& jb = jobs[lo];
            const uint64_t local = item - st.offs[lo];
            Mod<L> md;
#pragma unroll
            for (int i = 0; i < L; ++i) md.q[i] = jb.q32[i];
            md.nprime = jb.nprime32;
            md.nsub = jb.nsub;
            MR mr;
#pragma unroll
            for (int i = 0; i < LR; ++i) mr.q[i] = jb.q26[i];
            mr.nprime = jb.nprime26;
            mr.qtop_inv = jb.qtop_inv26;
            LevelParams lp = jb.lp;
            uint64_t bp = 1;
            for (uint32_t i = 0; i < st.level; ++i) bp *= G::TWO_M;
            lp.bp = bp;
            lp.len = lp.P2 / bp;
            const uint64_t cols = lp.P2 / G::TWO_M;
            switch (st.type) {
                case kStFwdLevel:
                    if (st.level == 0) level_fwd_ntt<m, L, LR, true, MR>(lp, md, mr, smem, local % cols, (int)(local / cols));
                    else level_fwd_ntt<m, L, LR, false, MR>(lp, md, mr, smem, local % cols, (int)(local / cols));
                    break;
                case kStInvLevel:
                    level_inv_ntt<m, L, LR, MR>(lp, md, mr, smem, local);
                    break;
                case kStFwdDft:
                    if (st.level == 0) dft_fwd_column<m, L, true>(lp, md, smem, local % cols, (int)(local / cols));
                    else dft_fwd_column<m, L, false>(lp, md, smem, local % cols, (int)(local / cols));
                    break;
                case kStFwdTwiddle:
                case kStInvTwiddle: {
                    const uint64_t groups = (lp.P2 + NttTeam<m>::NTEAMS - 1) / NttTeam<m>::NTEAMS;
                    if (st.type == kStFwdTwiddle)
                        twiddle_ntt_group<m, L, LR, false, MR>(lp, mr, local % groups, (int)(local / groups), smem);
                    else
                        twiddle_ntt_group<m, L, LR, true, MR>(lp, mr, local, 0, smem);
                    break;
                }
                case kStFinal:
                    lp.len = jb.r_last;
                    final_block<m, L, LR, kFormNtt, MR>(lp, md, mr, smem, local);
                    break;
                case kStInvDft:
                    dft_inv_column<m, L>(lp, md, smem, local);
                    break;
                case kStDecTiles:
                    if (jb.dp.u == 32) decode_tile_aligned<L, 1>(jb.dp, local, smem);
                    else if (jb.dp.u == 16) decode_tile_aligned<L, 2>(jb.dp, local, smem);
                    else decode_tile<L>(jb.dp, local);
                    break;
                case kStDecScan:
                    decode_scan_block<kThreads>(jb.dp);
                    break;
                case kStDecFix:
                    decode_fix_tile(jb.dp, local * kThreads + threadIdx.x);
                    break;
            }
            __syncthreads();   // shared memory is reused by the next item
        }
        grid.sync();
    }
}

}  // namespace dkss
