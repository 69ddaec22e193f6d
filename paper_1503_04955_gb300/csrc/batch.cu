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
#include <vector>

#include "batch.cuh"
#include "plan.hpp"

using dkss_host::u128;

namespace {

// The residue ring shared by all classes of a batch: m = 32, p = 65537 = 2^16 + 1
// (2M | p - 1 for every 2M <= 2^16), z = 5, so p^z ~ 2^80 exceeds the largest
// coefficient M (m/2) (2^u - 1)^2 for M <= 4096 with u = 32; L = 3, LR = 4.
constexpr uint32_t kBm = 32, kBL = 3, kBLR = 4, kBz = 5;
constexpr uint64_t kBp = 65537;

struct ClassParams {
    uint64_t M = 0;
    uint32_t u = 0;
    double ms[2] = {-1.0, -1.0};   // measured time per product for u = 32, 16 (autotuned)
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

u128 ring_q() {
    u128 q = 1;
    for (uint32_t i = 0; i < kBz; ++i) q *= kBp;
    return q;
}

// Smallest valid M for u, or 0: M (m/2) u >= N, 2M > 2m (one radix-2m level at
// least), and the coefficient bound below p^z.
uint64_t class_M(uint64_t N, uint32_t u) {
    uint64_t M = next_pow2((N + (kBm / 2) * u - 1) / ((kBm / 2) * u));
    if (M < 2 * kBm) M = 2 * kBm;
    const u128 umax = ((u128)1 << u) - 1;
    if ((u128)M * (kBm / 2) * umax * umax >= ring_q() || 2 * M > (1u << 16)) return 0;
    return M;
}

std::mutex g_tune_mu;
std::map<std::pair<int, uint64_t>, ClassParams> g_tune_cache;   // (device, class N) -> choice

// Device time of one product of the class with (M, u): plan, 2 warm-up calls,
// median of 5 timed calls.
double time_candidate(uint64_t N, uint64_t M, uint32_t u) {
    dkss_plan_t pl = nullptr;
    if (dkss_plan(&pl, N, M, kBm, u, kBp, kBz, 0) != DKSS_OK) return -1.0;
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

// Parameters of the class of operands up to N bits: by the rule (largest valid
// u, the thesis's "maximise u" heuristic of Section 4.1) or by measurement.
ClassParams choose_class(int device, uint64_t N, bool autotune) {
    ClassParams c;
    const uint32_t us[2] = {32, 16};
    if (!autotune) {
        for (uint32_t u : us)
            if ((c.M = class_M(N, u))) {
                c.u = u;
                return c;
            }
        return c;
    }
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find({device, N});
        if (it != g_tune_cache.end()) return it->second;
    }
    double best = -1.0;
    for (int i = 0; i < 2; ++i) {
        const uint64_t M = class_M(N, us[i]);
        if (!M) continue;
        const double t = time_candidate(N, M, us[i]);
        c.ms[i] = t;
        if (t > 0 && (best < 0 || t < best)) {
            best = t;
            c.M = M;
            c.u = us[i];
        }
    }
    if (!c.M) return choose_class(device, N, false);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[{device, N}] = c;
    return c;
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
    dkss::Mod<kBL> md{};
    dkss::ModRR<kBLR> mr{};
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
    void* args[] = {&b->d_jobs, &b->d_stages, &b->n_stages, &count, &b->md, &b->mr};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)dkss::k_batch<kBm, kBL, kBLR>, dim3(b->grid),
                                                dim3(dkss::kThreads), args, b->smem, st);
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
    for (auto& kv : cls) {
        kv.second = (uint32_t)b->class_N.size();
        b->class_N.push_back(kv.first);
        ClassParams c = choose_class(b->device, kv.first, !(flags & DKSS_BATCH_RULE));
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
        s = dkss_planning::plan_host(&t->host, b->class_N[c], b->class_params[c].M, kBm, b->class_params[c].u, kBp,
                                     kBz);
        if (s == DKSS_OK && (t->host.L != kBL || t->host.LR != kBLR || !t->host.ntt_ok)) s = DKSS_EUNSUPPORTED;
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
    const dkss_plan_s& h0 = b->tables[0]->host;
    for (int i = 0; i < (int)kBL; ++i) b->md.q[i] = h0.q_limbs[i];
    b->md.nprime = h0.nprime;
    b->md.nsub = h0.nsub;
    for (int i = 0; i < (int)kBLR; ++i) b->mr.q[i] = h0.q_rr[i];
    b->mr.nprime = h0.nprime26;

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
    b->smem = std::max({sizeof(uint32_t) * (size_t)G::TWO_M * G::EW, fin, xbuf,
                        dkss::level_ntt_smem_bytes<kBm, kBL, kBLR>(), sizeof(uint32_t) * (size_t)dkss::kDecSmemWords});
    int per_sm = 0, sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) != cudaSuccess ||
        (int)b->smem > optin ||
        cudaFuncSetAttribute(dkss::k_batch<kBm, kBL, kBLR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dkss::k_batch<kBm, kBL, kBLR>, dkss::kThreads, b->smem) !=
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
    const uint64_t v[9] = {c.M, kBm, c.u, kBp, kBz, b->class_N[b->job_class[job]], (uint64_t)(t.host.col_levels + 1),
                           (uint64_t)b->grid, (uint64_t)(b->exec != nullptr)};
    for (size_t i = 0; i < n && i < 9; ++i) params[i] = v[i];
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
