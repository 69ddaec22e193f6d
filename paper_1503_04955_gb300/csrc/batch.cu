// Batched products of uneven sizes (dkss_batch_*, dkss_mul_batch): size
// classes, the autotuner that picks each class's parameters, and the graph
// that launches the persistent kernel of batch.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "batch.cuh"
#include "plan.hpp"

using dkss_host::u128;

namespace {

// The limb layout shared by all classes of a batch (one kernel instantiation):
// m = 32, residues of L = 3 32-bit words, products in LR = 4 26-bit limbs.
// Each class has its own M, u and ring Z/p^zZ with that layout.
constexpr uint32_t kBm = 32, kBL = 3, kBLR = 4;

// A class's ring: (p, z) with p from the candidate primes, or a Proth prime
// p = h 2^n + 1 with z = 1 (dkss_plan_proth).
struct Ring {
    uint64_t p = 0, h = 0;
    uint32_t z = 0, n = 0;
    bool proth = false;
};

struct ClassParams {
    uint64_t M = 0;
    uint32_t u = 0;
    Ring ring;
    double ms = -1.0;   // measured device time of one product of the class (autotuned)
};

struct ClassTables {
    dkss_plan_s host;              // plan math only (no device memory)
    uint32_t* d_eval = nullptr;
    uint32_t* d_ntt = nullptr;
};

uint64_t next_pow2(uint64_t x) {
    uint64_t r = 1;
    while (r < x) r <<= 1;
    return r;
}

dkss_status class_host(dkss_plan_s* pl, uint64_t N, uint64_t M, uint32_t u, const Ring& r) {
    return r.proth ? dkss_planning::plan_host_proth(pl, N, M, kBm, u, r.h, r.n)
                   : dkss_planning::plan_host(pl, N, M, kBm, u, r.p, r.z);
}

bool in_layout(const dkss_plan_s& h) { return h.L == kBL && h.LR == kBLR && h.ntt_ok; }

// Smallest M for u: M (m/2) u >= N and 2M > 2m (one radix-2m level at least).
uint64_t class_M(uint64_t N, uint32_t u) {
    uint64_t M = next_pow2((N + (kBm / 2) * u - 1) / ((kBm / 2) * u));
    return M < 2 * kBm ? 2 * kBm : M;
}

// The class's ring in the batch layout: with proth, the Proth prime of
// dkss_proth_ring at LR = 4; otherwise, of the candidate primes with 2M | p-1,
// the smallest p^z above the coefficient bound whose plan has the layout
// (p^z just above the bound, the thesis's choice of Section 4.1).
bool class_ring(uint64_t N, uint64_t M, uint32_t u, bool proth, Ring* out) {
    if (proth) {
        Ring r;
        r.proth = true;
        r.z = 1;
        if (!dkss_planning::proth_ring_lr(N, M, kBm, u, kBLR, &r.h, &r.n)) return false;
        dkss_plan_s pl;
        if (class_host(&pl, N, M, u, r) != DKSS_OK || !in_layout(pl)) return false;
        r.p = (uint64_t)pl.p;
        *out = r;
        return true;
    }
    bool found = false;
    u128 best = 0;
    for (size_t i = 0; i < dkss_planning::kNumCandidatePrimes; ++i) {
        const uint64_t p = dkss_planning::kCandidatePrimes[i];
        if ((p - 1) % (2 * M) != 0) continue;
        for (uint32_t z = 1; z <= 8; ++z) {
            dkss_plan_s pl;
            const dkss_status s = dkss_planning::plan_host(&pl, N, M, kBm, u, p, z);
            if (s != DKSS_OK || !in_layout(pl)) continue;
            if (!found || pl.q < best) {
                best = pl.q;
                out->p = p;
                out->z = z;
                out->proth = false;
                found = true;
            }
            break;
        }
    }
    return found;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, uint64_t, bool>, ClassParams> g_tune_cache;   // (device, class N, proth) -> choice

// Device time of one product of the class with (M, u, ring): plan, 2 warm-up
// calls, median of 5 timed calls.
double time_candidate(uint64_t N, uint64_t M, uint32_t u, const Ring& r) {
    dkss_plan_t pl = nullptr;
    const dkss_status ps = r.proth ? dkss_plan_proth(&pl, N, M, kBm, u, r.h, r.n, 0)
                                   : dkss_plan(&pl, N, M, kBm, u, r.p, r.z, 0);
    if (ps != DKSS_OK) return -1.0;
    const size_t nw = (N + 63) / 64;
    uint64_t* buf = nullptr;
    double result = -1.0;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&buf, 4 * nw * sizeof(uint64_t)) == cudaSuccess && cudaStreamCreate(&st) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
        cudaMemsetAsync(buf, 0xA5, 2 * nw * sizeof(uint64_t), st) == cudaSuccess) {
        // operands with the top bits above N cleared
        const uint64_t top = N - 64 * (nw - 1);
        if (top < 64) {
            uint64_t last = ((uint64_t)1 << top) - 1;
            last &= 0xA5A5A5A5A5A5A5A5ull;
            cudaMemcpyAsync(buf + nw - 1, &last, 8, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(buf + 2 * nw - 1, &last, 8, cudaMemcpyHostToDevice, st);
        }
        bool ok = true;
        for (int i = 0; i < 2 && ok; ++i) ok = dkss_mul(pl, buf, buf + nw, buf + 2 * nw, (dkss_stream_t)st) == DKSS_OK;
        std::vector<float> t;
        for (int i = 0; i < 5 && ok; ++i) {
            float ms = 0.f;
            ok = cudaEventRecord(e0, st) == cudaSuccess &&
                 dkss_mul(pl, buf, buf + nw, buf + 2 * nw, (dkss_stream_t)st) == DKSS_OK &&
                 cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            t.push_back(ms);
        }
        if (ok) {
            std::sort(t.begin(), t.end());
            result = t[t.size() / 2];
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(buf);
    dkss_plan_destroy(pl);
    return result;
}

// Parameters of the class of operands up to N bits, over the configured
// primes or over Proth primes: by the rule (the largest u with a ring in the
// layout, the thesis's "maximise u" of Section 4.1) or by timing u = 32 and
// u = 16, each with its ring.
ClassParams choose_class(int device, uint64_t N, bool proth, bool autotune) {
    ClassParams c;
    const uint32_t us[2] = {32, 16};
    if (!autotune) {
        for (uint32_t u : us) {
            const uint64_t M = class_M(N, u);
            Ring r;
            if (2 * M <= (1u << 16) && class_ring(N, M, u, proth, &r)) {
                c.M = M;
                c.u = u;
                c.ring = r;
                return c;
            }
        }
        return c;
    }
    const auto key = std::make_tuple(device, N, proth);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return it->second;
    }
    for (uint32_t u : us) {
        const uint64_t M = class_M(N, u);
        Ring r;
        if (2 * M > (1u << 16) || !class_ring(N, M, u, proth, &r)) continue;
        const double t = time_candidate(N, M, u, r);
        if (t > 0 && (c.ms < 0 || t < c.ms)) {
            c.ms = t;
            c.M = M;
            c.u = u;
            c.ring = r;
        }
    }
    if (!c.M) return choose_class(device, N, proth, false);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = c;
    return c;
}

const void* batch_kernel(bool proth) {
    if (proth) return (const void*)dkss::k_batch<kBm, kBL, kBLR, dkss::ModRRSparse<kBLR>>;
    return (const void*)dkss::k_batch<kBm, kBL, kBLR, dkss::ModRR<kBLR>>;
}

}  // namespace

struct dkss_batch_s {
    int device = 0;
    uint32_t flags = 0;
    std::vector<uint64_t> n_bits;
    std::vector<uint64_t> class_N;                 // per class: largest operand size
    std::vector<ClassParams> class_params;
    std::vector<std::unique_ptr<ClassTables>> tables;
    std::vector<uint32_t> job_class;
    std::vector<dkss::BatchJob> h_jobs;
    dkss::BatchJob* d_jobs = nullptr;
    dkss::BatchJob* h_jobs_pinned = nullptr;
    dkss::BatchStage* d_stages = nullptr;
    uint64_t* d_offs = nullptr;
    uint32_t n_stages = 0;
    uint32_t* d_work = nullptr;
    uint32_t* d_agg = nullptr;
    uint32_t* d_status = nullptr;
    bool proth = false;                            // every class over a Proth prime (sparse reduction)
    int grid = 0;
    size_t smem = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
};

namespace {

void batch_free(dkss_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (auto& t : b->tables) {
        if (!t) continue;
        cudaFree(t->d_eval);
        cudaFree(t->d_ntt);
    }
    cudaFree(b->d_jobs);
    cudaFreeHost(b->h_jobs_pinned);
    cudaFree(b->d_stages);
    cudaFree(b->d_offs);
    cudaFree(b->d_work);
    cudaFree(b->d_agg);
    cudaFree(b->d_status);
    delete b;
}

dkss_status launch_batch(dkss_batch_s* b, cudaStream_t st) {
    uint32_t count = (uint32_t)b->n_bits.size();
    void* args[] = {&b->d_jobs, &b->d_stages, &b->n_stages, &count};
    cudaError_t e = cudaLaunchCooperativeKernel(batch_kernel(b->proth), dim3(b->grid), dim3(dkss::kThreads), args,
                                                b->smem, st);
    return e == cudaSuccess ? DKSS_OK : DKSS_ECUDA;
}

}  // namespace

extern "C" {

dkss_status dkss_batch_plan(dkss_batch_t* out, const uint64_t* n_bits, size_t count, uint32_t flags) {
    if (!out) return DKSS_EINVAL;
    *out = nullptr;
    if (!n_bits || count == 0 || count > (1u << 20)) return DKSS_EINVAL;
    dkss_batch_s* b = new (std::nothrow) dkss_batch_s;
    if (!b) return DKSS_ENOMEM;
    b->flags = flags;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return DKSS_ECUDA;
    }
    b->n_bits.assign(n_bits, n_bits + count);
    // size classes: operands up to the next power of two (at least 2^12 bits)
    std::map<uint64_t, uint32_t> cls;
    for (uint64_t n : b->n_bits) {
        if (n == 0) {
            delete b;
            return DKSS_EINVAL;
        }
        cls.emplace(std::max<uint64_t>(4096, next_pow2(n)), 0);
    }
    std::map<uint64_t, uint64_t> jobs_per_class;
    for (uint64_t n : b->n_bits) ++jobs_per_class[std::max<uint64_t>(4096, next_pow2(n))];
    // rings: the configured primes or Proth primes for every class (one kernel
    // instantiation per batch); by flag, by the rule (configured primes), or
    // the set with the smaller sum over classes of jobs x measured time
    const bool autotune = !(flags & DKSS_BATCH_RULE);
    bool proth = (flags & DKSS_BATCH_PROTH) != 0;
    if (autotune && !(flags & (DKSS_BATCH_PROTH | DKSS_BATCH_NO_PROTH))) {
        double cost[2] = {0, 0};
        for (int mode = 0; mode < 2; ++mode)
            for (auto& kv : cls) {
                const ClassParams c = choose_class(b->device, kv.first, mode == 1, true);
                cost[mode] += (c.M && c.ms > 0) ? c.ms * (double)jobs_per_class[kv.first] : 1e30;
            }
        proth = cost[1] < cost[0];
    }
    b->proth = proth;
    for (auto& kv : cls) {
        kv.second = (uint32_t)b->class_N.size();
        b->class_N.push_back(kv.first);
        ClassParams c = choose_class(b->device, kv.first, proth, autotune);
        if (!c.M) {
            delete b;
            return DKSS_EUNSUPPORTED;
        }
        b->class_params.push_back(c);
    }
    for (uint64_t n : b->n_bits) b->job_class.push_back(cls[std::max<uint64_t>(4096, next_pow2(n))]);

    // per-class plan math and device tables
    dkss_status s = DKSS_OK;
    for (size_t c = 0; c < b->class_N.size() && s == DKSS_OK; ++c) {
        auto t = std::make_unique<ClassTables>();
        s = class_host(&t->host, b->class_N[c], b->class_params[c].M, b->class_params[c].u, b->class_params[c].ring);
        if (s == DKSS_OK && (!in_layout(t->host) || t->host.q_sparse != b->proth)) s = DKSS_EUNSUPPORTED;
        if (s == DKSS_OK) {
            std::vector<uint32_t> ev, nt;
            dkss_planning::build_eval_table(&t->host, ev, true);
            dkss_planning::build_ntt_consts(&t->host, nt);
            if (cudaMalloc(&t->d_eval, ev.size() * 4) != cudaSuccess || cudaMalloc(&t->d_ntt, nt.size() * 4) != cudaSuccess ||
                cudaMemcpy(t->d_eval, ev.data(), ev.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(t->d_ntt, nt.data(), nt.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                s = DKSS_ENOMEM;
        }
        b->tables.push_back(std::move(t));
    }
    if (s != DKSS_OK) {
        cudaGetLastError();
        batch_free(b);
        return s;
    }

    // workspaces, carry scratch, job table
    uint64_t work_words = 0, agg_words = 0;
    std::vector<uint64_t> work_off(count), agg_off(count), tiles(count);
    for (size_t j = 0; j < count; ++j) {
        const dkss_plan_s& h = b->tables[b->job_class[j]]->host;
        work_off[j] = work_words;
        work_words += 2 * h.P2 * kBm * kBL;
        tiles[j] = (4 * ((b->n_bits[j] + 63) / 64) + dkss::kDecTile - 1) / dkss::kDecTile;
        agg_off[j] = agg_words;
        agg_words += tiles[j];
    }
    if (cudaMalloc(&b->d_work, work_words * 4) != cudaSuccess || cudaMalloc(&b->d_agg, agg_words * 4) != cudaSuccess ||
        cudaMalloc(&b->d_status, 4) != cudaSuccess || cudaMemset(b->d_status, 0, 4) != cudaSuccess ||
        cudaMalloc(&b->d_jobs, count * sizeof(dkss::BatchJob)) != cudaSuccess ||
        cudaMallocHost(&b->h_jobs_pinned, count * sizeof(dkss::BatchJob)) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return DKSS_ENOMEM;
    }
    b->h_jobs.resize(count);
    uint32_t max_levels = 0;
    for (size_t j = 0; j < count; ++j) {
        const ClassTables& t = *b->tables[b->job_class[j]];
        const dkss_plan_s& h = t.host;
        dkss::BatchJob& jb = b->h_jobs[j];
        std::memset(&jb, 0, sizeof(jb));
        dkss::LevelParams& lp = jb.lp;
        lp.data = b->d_work + work_off[j];
        lp.table = t.d_eval;
        lp.table_eval = t.d_eval;
        lp.ntt_cst = t.d_ntt;
        lp.ntt_prescale = h.ntt_bias.prescale ? 1u : 0u;
        lp.poly_words = h.P2 * kBm * kBL;
        lp.P2 = h.P2;
        lp.mu_top = h.mu_top;
        lp.M = h.M;
        lp.n_bits = b->n_bits[j];
        lp.raw_words = (b->n_bits[j] + 63) / 64;
        lp.u = h.u;
        lp.log2_mu_top = h.log2_mu_top;
        for (int i = 0; i < 5; ++i) lp.kscale[i] = h.kscale[i];
        dkss::DecodeParams& dp = jb.dp;
        dp.c = lp.data;
        dp.agg = b->d_agg + agg_off[j];
        dp.status = b->d_status;
        dp.P2 = h.P2;
        dp.n_windows = 4 * lp.raw_words;
        dp.n_tiles = tiles[j];
        dp.k_max = h.P2 * (kBm / 2) + kBm / 2;
        dp.m = kBm;
        dp.h = kBm / 2;
        dp.u = h.u;
        dp.db = 0;
        for (u128 x = h.q; x; x >>= 1) dp.db++;
        dp.db += 1;
        jb.col_levels = h.col_levels;
        jb.r_last = (uint32_t)h.r_last;
        for (int i = 0; i < 4; ++i) jb.q32[i] = h.q_limbs[i];
        jb.nprime32 = h.nprime;
        jb.nsub = h.nsub;
        for (int i = 0; i < 5; ++i) jb.q26[i] = h.q_rr[i];
        jb.nprime26 = h.nprime26;
        jb.qtop_inv26 = dkss::qtop_reciprocal(h.q_rr[kBLR - 1], h.q_rr[kBLR - 2]);
        max_levels = std::max(max_levels, h.col_levels);
    }

    // stage list and per-stage job offsets
    std::vector<std::pair<uint32_t, uint32_t>> st;
    for (uint32_t d = 0; d < max_levels; ++d) {
        st.push_back({dkss::kStFwdLevel, d});
    }
    st.push_back({dkss::kStFinal, 0});
    for (int d = (int)max_levels - 1; d >= 0; --d) {
        st.push_back({dkss::kStInvLevel, (uint32_t)d});
    }
    st.push_back({dkss::kStDecTiles, 0});
    st.push_back({dkss::kStDecScan, 0});
    st.push_back({dkss::kStDecFix, 0});
    b->n_stages = (uint32_t)st.size();
    std::vector<uint64_t> offs(st.size() * (count + 1));
    std::vector<dkss::BatchStage> stages(st.size());
    if (cudaMalloc(&b->d_offs, offs.size() * 8) != cudaSuccess ||
        cudaMalloc(&b->d_stages, stages.size() * sizeof(dkss::BatchStage)) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return DKSS_ENOMEM;
    }
    using G = dkss::Geo<kBm, kBL>;
    for (size_t k = 0; k < st.size(); ++k) {
        uint64_t acc = 0;
        for (size_t j = 0; j < count; ++j) {
            offs[k * (count + 1) + j] = acc;
            const dkss_plan_s& h = b->tables[b->job_class[j]]->host;
            acc += dkss::batch_items<kBm>(st[k].first, st[k].second, h.P2, h.col_levels, h.r_last, tiles[j],
                                          dkss::NttTeam<kBm>::NTEAMS);
        }
        offs[k * (count + 1) + count] = acc;
        stages[k].type = st[k].first;
        stages[k].level = st[k].second;
        stages[k].total = acc;
        stages[k].offs = b->d_offs + k * (count + 1);
    }
    std::memcpy(b->h_jobs_pinned, b->h_jobs.data(), count * sizeof(dkss::BatchJob));
    if (cudaMemcpy(b->d_offs, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_stages, stages.data(), stages.size() * sizeof(dkss::BatchStage), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->d_jobs, b->h_jobs.data(), count * sizeof(dkss::BatchJob), cudaMemcpyHostToDevice) != cudaSuccess) {
        batch_free(b);
        return DKSS_ECUDA;
    }

    // persistent grid: as many CTAs as can be resident
    // column DFTs; the fused last level with the NTT exchange buffers after its
    // two blocks; twiddle exchange buffers; fused levels (column + exchange
    // buffers); decode tiles
    const size_t xbuf = sizeof(uint32_t) * (size_t)dkss::NttTeam<kBm>::NTEAMS * kBm * kBLR;
    size_t fin = 0;
    for (const auto& t : b->tables)
        fin = std::max(fin, dkss::final_smem_bytes<kBm, kBL, kBLR>((int)t->host.r_last, dkss::kFormNtt));
    b->smem = std::max({sizeof(uint32_t) * (size_t)G::TWO_M * G::ES, fin, xbuf,
                        dkss::level_ntt_smem_bytes<kBm, kBL, kBLR>(), sizeof(uint32_t) * (size_t)dkss::kDecSmemWords});
    int per_sm = 0, sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) != cudaSuccess ||
        (int)b->smem > optin ||
        cudaFuncSetAttribute(batch_kernel(b->proth), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(b->proth), dkss::kThreads, b->smem) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        batch_free(b);
        return DKSS_ECUDA;
    }
    b->grid = per_sm * sms;

    // capture the launch in a graph (plain cooperative launches when DKSS_BATCH_NO_GRAPH)
    if (!(flags & DKSS_BATCH_NO_GRAPH)) {
        if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            batch_free(b);
            return DKSS_ECUDA;
        }
        dkss_status ls = launch_batch(b, b->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &b->graph);
        if (ls != DKSS_OK || ce != cudaSuccess || cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
            // a runtime that cannot capture cooperative launches: launch directly
            cudaGetLastError();
            if (b->exec) cudaGraphExecDestroy(b->exec);
            if (b->graph) cudaGraphDestroy(b->graph);
            b->exec = nullptr;
            b->graph = nullptr;
        }
    }
    *out = b;
    return DKSS_OK;
}

dkss_status dkss_batch_run(dkss_batch_t b, const dkss_job* jobs, dkss_stream_t stream) {
    if (!b || !jobs) return DKSS_EINVAL;
    const size_t count = b->n_bits.size();
    for (size_t j = 0; j < count; ++j) {
        if (!jobs[j].a || !jobs[j].b || !jobs[j].out || jobs[j].n_bits != b->n_bits[j]) return DKSS_EINVAL;
        dkss::BatchJob& jb = b->h_jobs_pinned[j];
        jb.lp.raw_a = jobs[j].a;
        jb.lp.raw_b = jobs[j].b;
        jb.dp.out = reinterpret_cast<uint32_t*>(jobs[j].out);
        jb.dp.out_aligned16 = ((uintptr_t)jobs[j].out & 15) == 0;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(b->d_jobs, b->h_jobs_pinned, count * sizeof(dkss::BatchJob), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return DKSS_ECUDA;
    if (b->exec) return cudaGraphLaunch(b->exec, st) == cudaSuccess ? DKSS_OK : DKSS_ECUDA;
    return launch_batch(b, st);
}

dkss_status dkss_batch_job_params(dkss_batch_t b, size_t job, uint64_t* params, size_t n) {
    if (!b || job >= b->n_bits.size() || !params) return DKSS_EINVAL;
    const ClassParams& c = b->class_params[b->job_class[job]];
    const ClassTables& t = *b->tables[b->job_class[job]];
    const uint64_t v[13] = {c.M, kBm, c.u, (uint64_t)t.host.p, c.ring.z, b->class_N[b->job_class[job]],
                            (uint64_t)(t.host.col_levels + 1), (uint64_t)b->grid, (uint64_t)(b->exec != nullptr),
                            (uint64_t)(t.host.p >> 64), (uint64_t)c.ring.proth, c.ring.h, c.ring.n};
    for (size_t i = 0; i < n && i < 13; ++i) params[i] = v[i];
    return DKSS_OK;
}

dkss_status dkss_batch_destroy(dkss_batch_t b) {
    if (!b) return DKSS_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    return DKSS_OK;
}

dkss_status dkss_mul_batch(const dkss_job* jobs, size_t count, uint32_t flags, dkss_stream_t stream) {
    // The batch plan of the most recent call is kept and reused while the
    // lengths stay the same.
    static std::mutex mu;
    static dkss_batch_t cached = nullptr;
    static std::vector<uint64_t> cached_bits;
    static uint32_t cached_flags = 0;
    static int cached_dev = -1;
    if (!jobs || count == 0) return DKSS_EINVAL;
    std::lock_guard<std::mutex> g(mu);
    std::vector<uint64_t> bits(count);
    for (size_t j = 0; j < count; ++j) bits[j] = jobs[j].n_bits;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return DKSS_ECUDA;
    if (!cached || bits != cached_bits || flags != cached_flags || dev != cached_dev) {
        dkss_batch_destroy(cached);
        cached = nullptr;
        dkss_status s = dkss_batch_plan(&cached, bits.data(), count, flags);
        if (s != DKSS_OK) return s;
        cached_bits = bits;
        cached_flags = flags;
        cached_dev = dev;
    }
    return dkss_batch_run(cached, jobs, stream);
}

}  // extern "C"
