// Autotuning of the resident path's lane mappings for one query size.
//
// The resident path is one cost launch (the dense Q^T-vs-vocabulary distance
// block and K = exp(-lambda M), the M and K steps of Algorithm 1) followed by
// one solver launch that runs every Sinkhorn iteration (Algorithms 2 and 3 fused
// per document, Section III-C).  Which solver and lane mapping is fastest depends
// on the corpus's length mix and on v_r, so it is measured here on the corpus
// itself instead of fixed by hand (the paper picks its mappings by hand for each
// machine, Sections IV-V).
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <set>
#include <tuple>
#include <vector>

#include "corpus.h"

using namespace swmd;

namespace {

constexpr float kTuneLambda = 10.0f;
constexpr int kTuneIters = 15;

// splitmix64: a fixed, platform-independent generator for the timing query
uint64_t splitmix(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Median time in ms of `reps` whole queries (prep, cost, solver) after one
// untimed run; a negative value when the configuration cannot launch.
float time_query(swmd_corpus *c, Slot &s, int vr, int reps, cudaStream_t st, cudaEvent_t e0,
                 cudaEvent_t e1) {
    if (enqueue_query(c, s, s.q_in, s.r_in, vr, kTuneLambda, kTuneIters, s.out, s.status, st, false))
        return -1.0f;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1.0f;
    std::vector<float> ms;
    for (int i = 0; i < reps; ++i) {
        cudaEventRecord(e0, st);
        if (enqueue_query(c, s, s.q_in, s.r_in, vr, kTuneLambda, kTuneIters, s.out, s.status, st,
                          false))
            return -1.0f;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        ms.push_back(t);
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
}

}  // namespace

int swmd_autotune(swmd_corpus *c, int32_t v_r, int32_t reps, swmd_tune_result *out) {
    if (!c || !out) return set_error(SWMD_EINVAL, "swmd_autotune: NULL argument");
    if (reps < 1) return set_error(SWMD_EINVAL, "swmd_autotune: reps must be >= 1");
    if (c->opt.path != SWMD_PATH_RESIDENT && c->opt.path != SWMD_PATH_AUTO)
        return set_error(SWMD_EINVAL, "swmd_autotune tunes the resident path and the automatic choice; "
                         "the corpus uses path %d", c->opt.path);
    if (v_r < 1 || v_r > c->opt.max_vr || v_r > c->V)
        return set_error(SWMD_EINVAL, "swmd_autotune: v_r %d outside [1, min(max_vr %d, V %d)]", v_r,
                         c->opt.max_vr, c->V);
    std::memset(out, 0, sizeof(*out));
    if (c->Nl == 0) return SWMD_OK;

    std::lock_guard<std::mutex> lk(c->mu);
    if (c->servers > 0)
        return set_error(SWMD_EINVAL, "swmd_autotune: a server is attached to the corpus; tune before serving");
    DeviceGuard guard(c->device);
    Slot &s = c->main;
    cudaStream_t st = c->stream;

    // the timing query: v_r distinct ids, uniform weights
    std::vector<int32_t> ids;
    std::vector<float> r((size_t)v_r, 1.0f / (float)v_r);
    if ((int64_t)v_r * 2 > c->V) {
        for (int i = 0; i < v_r; ++i) ids.push_back(i);
    } else {
        std::set<int32_t> seen;
        uint64_t x = 0x2107064330ull + (uint64_t)v_r;
        while ((int)ids.size() < v_r) {
            const int32_t w = (int32_t)(splitmix(x) % (uint64_t)c->V);
            if (seen.insert(w).second) ids.push_back(w);
        }
    }
    SWMD_CK(cudaMemcpyAsync(s.q_in, ids.data(), sizeof(int32_t) * v_r, cudaMemcpyHostToDevice, st));
    SWMD_CK(cudaMemcpyAsync(s.r_in, r.data(), sizeof(float) * v_r, cudaMemcpyHostToDevice, st));

    const int kprec = c->opt.k_precision;
    const auto key = std::make_pair(v_r, kprec);
    const int tight = tight_vrp(v_r);   // the layout of the solvers other than the column-split one

    // time with every tunable field free and the resident path forced; the caller's
    // fields are put back after
    const int fix_solver = c->opt.solver, fix_npl = c->opt.nnz_per_lane, fix_split = c->opt.cost_split;
    const int fix_path = c->opt.path;
    c->opt.solver = c->opt.nnz_per_lane = c->opt.cost_split = 0;
    c->opt.path = SWMD_PATH_RESIDENT;
    c->tuned_resident.erase(key);

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);

    auto timed = [&](std::tuple<int, int, int> cfg) {
        c->tuned_resident[key] = cfg;
        const float ms = time_query(c, s, v_r, reps, st, e0, e1);
        cudaGetLastError();   // a configuration that cannot launch leaves no sticky error
        ++out->candidates;
        return ms;
    };

    std::tuple<int, int, int> best{0, 0, 0};
    float best_ms = timed(best);
    out->default_ms = best_ms;
    std::vector<std::tuple<int, int, int>> cands;
    if (c->col_tasks_dev) cands.emplace_back(kSolverCols, 0, 0);
    if (regs_rows_per_lane(tight, 0) > 0)
        for (int npl : {1, 2, 3, 4, 8})
            if (regs_rows_per_lane(tight, npl) == npl) cands.emplace_back(kSolverRegs, npl, 0);
    if (tiled_supported(tight, kprec)) cands.emplace_back(kSolverTiled, 0, 0);
    for (auto &cfg : cands) {
        const float ms = timed(cfg);
        if (ms > 0.0f && (best_ms <= 0.0f || ms < best_ms)) best_ms = ms, best = cfg;
    }
    if (v_r <= 32) {   // threads per word of the row-wise cost kernel (layouts up to 32)
        for (int split : {1, 2, 4}) {
            auto cfg = std::make_tuple(std::get<0>(best), std::get<1>(best), split);
            const float ms = timed(cfg);
            if (ms > 0.0f && (best_ms <= 0.0f || ms < best_ms)) best_ms = ms, best = cfg;
        }
    }
    c->tuned_resident[key] = best;
    // under SWMD_PATH_AUTO, the per-iteration fused path for the same query
    int chosen = SWMD_PATH_RESIDENT;
    float fused_ms = -1.0f;
    if (fix_path == SWMD_PATH_AUTO) {
        c->opt.path = SWMD_PATH_FUSED;
        fused_ms = time_query(c, s, v_r, reps, st, e0, e1);
        cudaGetLastError();
        ++out->candidates;
        if (fused_ms > 0.0f && (best_ms <= 0.0f || fused_ms < best_ms)) chosen = SWMD_PATH_FUSED;
        c->tuned_path[std::make_pair(v_r, kprec)] = chosen;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->opt.path = fix_path;

    c->opt.solver = fix_solver;
    c->opt.nnz_per_lane = fix_npl;
    c->opt.cost_split = fix_split;
    // captured graphs hold the kernels of the settings they were captured with
    clear_graphs(c);

    if (best_ms <= 0.0f && fused_ms <= 0.0f)
        return set_error(SWMD_ECUDA, "swmd_autotune: no configuration ran for v_r %d", v_r);
    out->vrp = layout_vrp(c, v_r, SWMD_PATH_RESIDENT);
    out->solver = std::get<0>(best);
    out->nnz_per_lane = std::get<1>(best);
    out->cost_split = std::get<2>(best);
    out->best_ms = chosen == SWMD_PATH_FUSED ? fused_ms : best_ms;
    out->path = chosen;
    return SWMD_OK;
}

int swmd_autotune_batch(swmd_corpus *c, int32_t n_queries, const int64_t *q_ptr, const int32_t *h_word_ids,
                        const float *h_weights, const float *h_lambdas, int32_t max_iter, int32_t reps,
                        swmd_batch_tune_result *out) {
    if (!c || !out || n_queries < 1 || !q_ptr || !h_word_ids || !h_weights || !h_lambdas)
        return set_error(SWMD_EINVAL, "swmd_autotune_batch: bad arguments");
    if (reps < 1) return set_error(SWMD_EINVAL, "swmd_autotune_batch: reps must be >= 1");
    std::memset(out, 0, sizeof(*out));
    const int kprec = c->opt.k_precision;
    // the column-split layouts the batch holds
    std::set<int> layouts;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (c->servers > 0)
            return set_error(SWMD_EINVAL, "swmd_autotune_batch: a server is attached to the corpus");
        for (int32_t i = 0; i < n_queries; ++i) {
            const int64_t n = q_ptr[i + 1] - q_ptr[i];
            if (n < 1 || n > INT32_MAX) return set_error(SWMD_EINVAL, "swmd_autotune_batch: bad q_ptr");
            std::vector<int32_t> ids((size_t)n);
            std::vector<float> r((size_t)n);
            int32_t vr = 0;
            int rc = swmd_select(c->V, (int32_t)n, h_word_ids + q_ptr[i], h_weights + q_ptr[i], ids.data(),
                                 r.data(), &vr);
            if (rc) return rc;
            if (vr > c->opt.max_vr) continue;   // swmd_query_batch reports it
            if (resolve_path(c, vr) == SWMD_PATH_RESIDENT && resident_solver(c, vr, kprec) == kSolverCols)
                layouts.insert(cols_vrp(vr));
        }
        for (int v : layouts) c->tuned_qpt.erase(std::make_pair(v, kprec));
    }
    std::vector<double> sink((size_t)n_queries * std::max(c->Nl, 1));
    auto time_batch = [&]() -> float {
        // the first call of a shape captures its graph: untimed
        int rc = swmd_query_batch(c, n_queries, q_ptr, h_word_ids, h_weights, h_lambdas, max_iter, sink.data());
        if (rc && rc != SWMD_ENUMERIC) return -1.0f;
        std::vector<float> ms;
        for (int k = 0; k < reps; ++k) {
            const auto t0 = std::chrono::steady_clock::now();
            rc = swmd_query_batch(c, n_queries, q_ptr, h_word_ids, h_weights, h_lambdas, max_iter, sink.data());
            if (rc && rc != SWMD_ENUMERIC) return -1.0f;
            ms.push_back(std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count());
        }
        std::sort(ms.begin(), ms.end());
        return ms[ms.size() / 2];
    };
    auto set_tile = [&](int v, int qpt) {
        std::lock_guard<std::mutex> lk(c->mu);
        if (qpt > 0) c->tuned_qpt[std::make_pair(v, kprec)] = qpt;
        else c->tuned_qpt.erase(std::make_pair(v, kprec));
        clear_graphs(c);   // captured batches hold the tile size they were captured with
    };
    out->default_ms = time_batch();
    ++out->candidates;
    if (out->default_ms < 0.0f) return set_error(SWMD_ECUDA, "swmd_autotune_batch: %s", swmd_last_error());
    float best_all = out->default_ms;
    int li = 0;
    for (int v : layouts) {
        int best = 0;
        float best_ms = best_all;
        for (int qpt : {1, 2, 4, 8}) {
            set_tile(v, qpt);
            const float ms = time_batch();
            ++out->candidates;
            if (ms > 0.0f && ms < best_ms) best_ms = ms, best = qpt;
        }
        const int chosen = best > 0 ? best : 0;
        set_tile(v, chosen);
        {
            std::lock_guard<std::mutex> lk(c->mu);
            if (chosen == 0) {   // the default stood: record the size it resolved to
                const int d = cols_queries_per_group(c, v, kprec);
                c->tuned_qpt[std::make_pair(v, kprec)] = d;
            }
            if (li < 4) {
                out->vrp[li] = v;
                out->queries_per_tile[li] = cols_queries_per_group(c, v, kprec);
            }
        }
        best_all = best_ms;
        ++li;
    }
    out->layouts = li;
    out->best_ms = best_all;
    return SWMD_OK;
}
