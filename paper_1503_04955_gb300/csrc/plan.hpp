// Internal plan object behind dkss_plan_t (include/dkss.h).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/dkss.h"
#include "host_math.hpp"
#include "ntt_bounds.hpp"
#include "status_bits.hpp"

struct dkss_plan_s {
    // parameters (thesis Section 3.2 steps 1-2)
    uint64_t n_bits = 0, M = 0, P2 = 0, mu_top = 0;
    dkss_host::u128 p = 0;        // the prime (above 2^64 only for Proth primes, dkss_plan_proth)
    uint32_t m = 0, u = 0, z = 0, flags = 0;
    uint32_t L = 0;               // 32-bit limbs per residue
    uint32_t log2_mu_top = 0;
    uint32_t col_levels = 0;      // radix-2m levels of the transform
    uint64_t r_last = 0;          // length of the last (alpha-power) level
    dkss_host::u128 q = 0;        // p^z
    uint32_t q_limbs[4] = {0, 0, 0, 0};
    uint32_t nprime = 0, nsub = 0;
    uint32_t LR = 0;              // 26-bit limbs of the product arithmetic
    uint32_t i8_S = 0;            // bytes per residue for the INT8 tensor-core form
    uint32_t q_rr[5] = {0, 0, 0, 0, 0};
    uint32_t nprime26 = 0;        // -(p^z)^-1 mod 2^26
    bool q_sparse = false;        // p^z = 1 mod 2^26 and its 26-bit limbs 1 .. LR-2 are zero (Proth
                                  // primes h 2^n + 1, n >= 26 (LR-1)): Montgomery reduction without the
                                  // digit product and with one limb product per digit (rr_arith.cuh)
    uint32_t kscale[5] = {0, 0, 0, 0, 0};  // (2M)^-1 R'^2 mod p^z, 26-bit limbs
    dkss_host::Roots roots;
    bool ntt_ok = false;                  // the lazy NTT form's limits hold for this ring
    dkss_planning::NttBiases ntt_bias{};  // its bias constants
    // p-adic digit form of the m = 64 NTT kernels (padic.cuh): z = 4, p < 2^30, within
    // the limits pd_lazy_bounds checks; tables and constants then hold 4 digits per residue
    bool padic = false;
    dkss_planning::PdBiases pd_bias{};
    uint32_t pd_nmu = 0, pd_s = 0;
    uint64_t pd_mu = 0;
    bool dft_lazy = false;        // m = 64 forward half-column DFTs unreduced between stages: 2^7 p^z < 2^(32L)
    uint32_t red_rcp = 0;         // their reduction: floor(2^40 / (top word of p^z + 1))
    bool pd_io = false;           // the forward levels keep p-adic digits in HBM (padic: 4 words per residue)
    uint64_t pd_pw_off = 0;       // word offset of the digits of 2^(32j) mod p^4 in d_ntt
    bool pd_fast = false;         // fast carries (floor(2^32/p) a power of two; padic.cuh)
    uint32_t pd_mu_lo = 0, pd_lg_nmu = 0;
    // device memory owned by the plan
    int device = 0;
    int sm_count = 1;
    uint32_t* d_table = nullptr;  // rho^s (s < mu_top): coefficients, or evaluations (default)
    uint32_t* d_ntt = nullptr;    // constants of the transform in R
    bool eval_levels = false;     // inner levels in evaluation coordinates (eval_levels.cuh)
    uint32_t* d_evtw = nullptr;   // their bad twiddles of levels d >= 1
    uint32_t* d_table_minv = nullptr;  // their plans: the level-twiddle table with m^-1 (dkss_forward)
    std::vector<uint64_t> evtw_offs;  // word offset of level d's table in d_evtw
    uint32_t* d_work = nullptr;   // two transformed polynomials
    uint64_t poly_words = 0;
    uint32_t* d_agg = nullptr;    // carry-scan tile aggregates
    uint32_t* d_half = nullptr;   // m = 64 column DFTs in halves: one half column per resident CTA
    int half_grid_fwd = 0, half_grid_inv = 0;   // their persistent grids
    uint64_t n_tiles = 0;
    uint32_t* d_status = nullptr;
    uint64_t* d_stage = nullptr;  // dkss_mul_host staging: a, b, out
    uint32_t launches = 0;
    uint64_t dev_bytes = 0;       // device memory the plan holds (workspace, tables, scratch)
    // DKSS_PROFILE: CUDA events around each kernel group, summed by kind on read
    struct ProfRec {
        cudaEvent_t start, stop;
        int kind;
    };
    std::vector<ProfRec> prof;
    double prof_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t prof_count[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace dkss_planning {
// Process-wide host fault-injection mask (dkss_fault_inject; 0 in normal use).
uint32_t fault_mask();
// Host parts of a plan, shared by single plans and batches (capi.cu).
dkss_status plan_host(dkss_plan_s* pl, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t p, uint32_t z);
dkss_status plan_host_proth(dkss_plan_s* pl, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t h,
                            uint32_t n);
bool proth_ring_lr(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint32_t LR, uint64_t* h, uint32_t* n);
// The primes the parameter search draws from (dkss_plan_candidates).
constexpr size_t kNumCandidatePrimes = 10;
extern const uint64_t kCandidatePrimes[kNumCandidatePrimes];
void build_table(const dkss_plan_s* pl, std::vector<uint32_t>& out);
void build_eval_table(const dkss_plan_s* pl, std::vector<uint32_t>& out, bool with_minv);
void build_ntt_consts(const dkss_plan_s* pl, std::vector<uint32_t>& out);
void build_eval_level_tables(const dkss_plan_s* pl, std::vector<uint32_t>& out, std::vector<uint64_t>& offs);
}  // namespace dkss_planning

namespace dkss {
// Kernel-group kinds reported by dkss_profile_read.
enum ProfKind {
    kProfFwdDft = 0,      // forward inner DFTs (first level encodes)
    kProfFwdTwiddle = 1,  // forward bad multiplications
    kProfFinal = 2,       // last forward level + products + first backwards level
    kProfInvTwiddle = 3,  // backwards bad multiplications
    kProfInvDft = 4,      // backwards inner DFTs
    kProfDecode = 5       // decoding and carry scan
};

// Record an event pair around a kernel group when the plan profiles.
struct ProfScope {
    dkss_plan_s* pl;
    cudaStream_t st;
    int kind;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ProfScope(dkss_plan_s* p, cudaStream_t s, int k) : pl(p), st(s), kind(k) {
        if (!(pl->flags & DKSS_PROFILE) || pl->prof.size() >= 65536) return;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            e0 = e1 = nullptr;
            return;
        }
        cudaEventRecord(e0, st);
    }
    ~ProfScope() {
        if (!e0) return;
        cudaEventRecord(e1, st);
        pl->prof.push_back({e0, e1, kind});
    }
};
}  // namespace dkss

namespace dkss {
// Per-(m, L, LR) launchers, explicitly instantiated by inst.cu.
template <int m, int L, int LR>
dkss_status run_mul(dkss_plan_s* pl, const uint64_t* a, const uint64_t* b, uint64_t* out, cudaStream_t st);
template <int m, int L, int LR>
dkss_status run_forward(dkss_plan_s* pl, const uint64_t* a, uint64_t* out, cudaStream_t st);
template <int m, int L, int LR>
dkss_status prepare(dkss_plan_s* pl);
}  // namespace dkss
