// C ABI of libswmd: corpus construction, the single query and its steps.
//
// The problem statement is the paper's sinkhorn_wmd(r, c, vecs, lambda, max_iter)
// (Section III-B1): a query histogram r over the vocabulary, a V x N CSR c whose
// columns are target documents, the V x d embeddings vecs; the answer is the
// Sinkhorn distance of r to every column of c (Algorithm 1).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "corpus.h"

namespace swmd {

static thread_local std::string g_error;

int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return set_error(e == cudaErrorMemoryAllocation ? SWMD_ENOMEM : SWMD_ECUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

namespace {

template <class T>
int dev_alloc(swmd_corpus *c, T **p, size_t count, int64_t *bytes) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = corpus_malloc(c, reinterpret_cast<void **>(p), count * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "device allocation");
    if (bytes) *bytes += (int64_t)(count * sizeof(T));
    return SWMD_OK;
}

void dev_free(swmd_corpus *c, void *p) { corpus_free(c, p); }

std::mutex g_alloc_mu;
Allocator g_allocator;   // the allocator corpora created from now on take

}  // namespace

// Every layout a query of up to max_vr words may take: the resident solvers' tight
// padding, the per-iteration walks' power of two >= 4 and the column-split
// solver's power of two >= 16 all fit.
int max_vrp_of(int max_vr) { return std::max(vrp_for(max_vr, 8), cols_vrp(max_vr)); }

cudaError_t corpus_malloc(swmd_corpus *c, void **p, size_t bytes) {
    *p = nullptr;
    if (!c->allocator.alloc) return cudaMalloc(p, bytes);
    void *q = c->allocator.alloc(bytes, c->device, c->stream, c->allocator.user);
    if (!q) return cudaErrorMemoryAllocation;
    {
        std::lock_guard<std::mutex> lk(c->alloc_mu);
        c->alloc_sizes[q] = bytes;
    }
    *p = q;
    return cudaSuccess;
}

void corpus_free(swmd_corpus *c, void *p) {
    if (!p) return;
    if (!c->allocator.release) {
        cudaFree(p);
        return;
    }
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(c->alloc_mu);
        auto it = c->alloc_sizes.find(p);
        if (it != c->alloc_sizes.end()) {
            bytes = it->second;
            c->alloc_sizes.erase(it);
        }
    }
    c->allocator.release(p, bytes, c->device, c->stream, c->allocator.user);
}

void clear_graphs(swmd_corpus *c) {
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    for (auto &kv : c->batch_graphs) cudaGraphExecDestroy(kv.second);
    c->batch_graphs.clear();
    c->batch_seen.clear();
}

int status_to_code(int st) {
    if (st & ST_BOUNDS)
        return set_error(SWMD_EINVAL, "a device bounds check failed: a corpus index lies outside its array");
    if (st & (ST_BAD_ID | ST_BAD_R))
        return set_error(SWMD_EINVAL, "query id outside [0, V) or weight not finite and > 0");
    if (st & ST_BAD_SIZE)
        return set_error(SWMD_EINVAL, "a pair side is empty or above its declared size bound");
    if (st & ST_NUMERIC)
        return set_error(SWMD_ENUMERIC, "a NaN, an infinity or a vanished K^T u appeared");
    return SWMD_OK;
}

int alloc_slot(swmd_corpus *c, Slot &s, int max_vr, int kprec, bool with_v) {
    free_slot(c, s);
    const int vrp = max_vrp_of(max_vr);
    const size_t kb = kprec_bytes(kprec);
    int rc;
    unsigned char *kt = nullptr, *kmt = nullptr;
    if ((rc = dev_alloc(c, &kt, (size_t)std::max(c->Vu, 1) * vrp * kb, &s.bytes))) return rc;
    s.KT = kt;
    if ((rc = dev_alloc(c, &kmt, (size_t)std::max(c->Vu, 1) * vrp * kb, &s.bytes))) return rc;
    s.KMT = kmt;
    if ((rc = dev_alloc(c, &s.u, (size_t)std::max(c->Nl, 1) * vrp, &s.bytes))) return rc;
    if (with_v) {
        s.v_elems = std::max<int64_t>(std::max(c->nnz, c->slice_total), 1);
        if ((rc = dev_alloc(c, &s.v, (size_t)s.v_elems, &s.bytes))) return rc;
    }
    if ((rc = dev_alloc(c, &s.q_ids, vrp, &s.bytes))) return rc;
    if ((rc = dev_alloc(c, &s.r, vrp, &s.bytes))) return rc;
    if ((rc = dev_alloc(c, &s.qp, 1, &s.bytes))) return rc;
    // the distances and, right after them, the status word: one device-to-host copy
    if ((rc = dev_alloc(c, &s.out, (size_t)std::max(c->Nl, 1) + 1, &s.bytes))) return rc;
    s.status = reinterpret_cast<int *>(s.out + std::max(c->Nl, 1));
    if ((rc = dev_alloc(c, &s.conv, 1 + kMaxConvIters, &s.bytes))) return rc;
    SWMD_CK(cudaMemset(s.conv, 0, sizeof(unsigned) * (1 + kMaxConvIters)));
    // the staged query ids and, right after them, its weights: one host-to-device copy
    if ((rc = dev_alloc(c, &s.q_in, 2 * (size_t)vrp, &s.bytes))) return rc;
    s.r_in = reinterpret_cast<float *>(s.q_in + vrp);
    s.carved_io = true;
    SWMD_CK(cudaMemset(s.u, 0, (size_t)std::max(c->Nl, 1) * vrp * sizeof(float)));
    s.vrp_cap = vrp;
    s.kprec = kprec;
    return SWMD_OK;
}

void free_slot(swmd_corpus *c, Slot &s) {
    dev_free(c, s.KT); dev_free(c, s.KMT); dev_free(c, s.u); dev_free(c, s.v); dev_free(c, s.q_ids);
    dev_free(c, s.r); dev_free(c, s.qp); dev_free(c, s.out); dev_free(c, s.q_in);
    dev_free(c, s.conv);
    if (!s.carved_io) {   // else they live inside out / q_in
        dev_free(c, s.status);
        dev_free(c, s.r_in);
    }
    s = Slot{};
}

int tight_vrp(int vr) { return vrp_for(vr, vr <= 32 ? 1 : (vr <= 64 ? 2 : 4)); }

static bool pow2_times4(int v) { return v >= 4 && v <= 128 && ((v / 4) & (v / 4 - 1)) == 0 && v % 4 == 0; }

// Padding VRP of the K^T / KM^T / u layout for a query of vr words on `path`:
// the per-iteration paths use a power of two >= 4 (the sliced walk gives each lane
// of a power-of-two team a 32-byte slice of every row); the resident solvers keep
// the tight padding.
int layout_vrp(swmd_corpus *c, int vr, int path) {
    const int tl = c->opt.team_lanes, lq = c->opt.lanes_per_nz;
    if (tl > 0 && lq > 0 && tl % lq == 0) {
        Mapping m{vrp_for(vr, lq), lq, tl / lq};
        if (mapping_supported(m)) return m.vrp;
    }
    if (path == SWMD_PATH_FUSED || path == SWMD_PATH_PLAIN) {
        int v = 4;
        while (v < vr) v *= 2;
        return v;
    }
    // the column-split register solver takes power-of-two layouts of 16 to 128
    if (resident_solver(c, vr, c->opt.k_precision) == kSolverCols) return cols_vrp(vr);
    return tight_vrp(vr);
}

// Kernel mapping for walking a layout of padding vrp: p = 0 selects the sliced
// walk (k_walk3; its team size follows from VRP and the K precision); otherwise
// the general walk with P sub-teams of Q lanes (swmd_options team_lanes /
// lanes_per_nz).
Mapping walk_mapping(swmd_corpus *c, int vrp, int path) {
    const int tl = c->opt.team_lanes, lq = c->opt.lanes_per_nz;
    if (tl > 0 && lq > 0 && tl % lq == 0) {
        Mapping m{vrp, lq, tl / lq};
        if (mapping_supported(m)) return m;
    }
    (void)path;
    if (pow2_times4(vrp)) return Mapping{vrp, vrp / 4, 0};
    const int p = c->mean_len >= 24.0 ? 8 : 4;
    for (int q = 1; q <= 8; q *= 2) {
        Mapping m{vrp, q, p};
        if (mapping_supported(m)) return m;
        m.p = 4;
        if (mapping_supported(m)) return m;
    }
    return Mapping{vrp, 1, 4};
}

int resolve_path(swmd_corpus *c, int vr) {
    if (c->opt.path != SWMD_PATH_AUTO) return c->opt.path;
    if (c->opt.tol > 0.f) return SWMD_PATH_FUSED;   // the convergence mode's path
    auto it = c->tuned_path.find(std::make_pair(vr, c->opt.k_precision));
    if (it != c->tuned_path.end()) return it->second;
    // the column-split register solver keeps every document's rows on chip for all
    // iterations: faster than the per-iteration walk at every width it takes, where
    // it holds every document
    bool whole = false;
    if (resident_solver(c, vr, c->opt.k_precision) == kSolverCols && cols_takes(c, vr, &whole) && whole)
        return SWMD_PATH_RESIDENT;
    return (c->Nl < kAutoResidentDocs || vr <= kAutoResidentVr) ? SWMD_PATH_RESIDENT : SWMD_PATH_FUSED;
}

Mapping choose_mapping(swmd_corpus *c, int vr, int path) {
    return walk_mapping(c, layout_vrp(c, vr, path), path);
}

// per-iteration launches of one mapping (the sliced walk when m.p == 0)
static cudaError_t iter_fused(const IterArgs &ia, Mapping m, int kprec, int sms, cudaStream_t st) {
    return m.p == 0 ? launch_fused3(ia, m.vrp, kprec, sms, st) : launch_fused(ia, m, kprec, sms, st);
}
static cudaError_t iter_sddmm(const IterArgs &ia, Mapping m, int kprec, int sms, cudaStream_t st) {
    return m.p == 0 ? launch_sddmm3(ia, m.vrp, kprec, sms, st) : launch_sddmm(ia, m, kprec, sms, st);
}
static cudaError_t iter_spmm(const IterArgs &ia, Mapping m, int kprec, int sms, cudaStream_t st) {
    return m.p == 0 ? launch_spmm3(ia, m.vrp, kprec, sms, st) : launch_spmm(ia, m, kprec, sms, st);
}
static cudaError_t iter_final(const IterArgs &ia, Mapping m, int kprec, int sms, cudaStream_t st) {
    return m.p == 0 ? launch_final3(ia, m.vrp, kprec, sms, st) : launch_final(ia, m, kprec, sms, st);
}

int build_tiles(swmd_corpus *c) {
    const int threads = c->opt.tile_threads > 0 ? c->opt.tile_threads : 128;
    const int npl = c->opt.nnz_per_lane > 0 ? c->opt.nnz_per_lane : 4;
    if (threads != 64 && threads != 128 && threads != 256)
        return set_error(SWMD_EINVAL, "tile_threads must be 64, 128 or 256");
    if (c->tiles_dev && threads == c->tile_threads && npl == c->tile_npl) return SWMD_OK;
    // tiles: consecutive documents (decreasing length) of one team size, at most
    // threads / team size of them and at most `budget` nonzeros
    std::vector<int> all;
    std::vector<int> off, count;
    for (int bi = 0; bi < kNumTileBudgets; ++bi) {
        const int budget = kTileBudgets[bi];
        off.push_back((int)all.size());
        int n = 0, d = 0;
        all.push_back(0);
        while (d < c->Nl) {
            int sum = 0, k = 0;
            const int g = team_lanes_for(c->len_sorted[d], npl);
            while (d + k < c->Nl && k < threads / g && team_lanes_for(c->len_sorted[d + k], npl) == g &&
                   (k == 0 || sum + c->len_sorted[d + k] <= budget)) {
                sum += c->len_sorted[d + k];
                ++k;
            }
            d += k;
            all.push_back(d);
            ++n;
        }
        count.push_back(n);
    }
    int *dev = nullptr;
    int64_t bytes = 0;
    int rc = dev_alloc(c, &dev, all.size(), &bytes);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(dev, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dev_free(c, dev);
        return cuda_fail(e, "copy tiles");
    }
    if (c->tiles_dev) {
        cudaDeviceSynchronize();   // no launch may still read the old sets
        dev_free(c, c->tiles_dev);
    }
    c->tiles_dev = dev;
    c->tile_off = off;
    c->tile_count = count;
    c->tile_threads = threads;
    c->tile_npl = npl;
    return SWMD_OK;
}

int build_tasks(swmd_corpus *c) {
    // the documents each column-split layout does not hold: documents are in
    // decreasing length, so they are the first col_first
    for (int li = 0; li < kColLayouts; ++li) {
        const int maxl = cols_max_len(16 << li);
        int f = 0;
        while (f < c->Nl && c->len_sorted[f] > maxl) ++f;
        c->col_first[li] = f;
    }
    std::vector<int4> all;
    for (int npl = 1; npl <= 8; ++npl) {
        c->task_off[npl] = (int)all.size();
        c->task_prefix[npl][0] = c->task_prefix[npl][1] = 0;
        int d = 0, n = 0;
        while (d < c->Nl) {
            // no task straddles the first column-split document of the 16- and
            // 32-column layouts: a prefix of the list covers exactly the documents
            // before it (a document's team, and so its result, does not depend on
            // the task it is in)
            int end = c->Nl;
            for (int li = 0; li < 2; ++li)
                if (c->col_first[li] > d) end = std::min(end, c->col_first[li]);
            const int g = reg_team_lanes(c->len_sorted[d], npl);
            int k = 0;
            while (d + k < end && k < 32 / g && reg_team_lanes(c->len_sorted[d + k], npl) == g) ++k;
            all.push_back(make_int4(d, g, k, 0));
            d += k;
            ++n;
            for (int li = 0; li < 2; ++li)
                if (d == c->col_first[li]) c->task_prefix[npl][li] = n;
        }
        c->task_count[npl] = n;
    }
    int64_t bytes = 0;
    int rc = dev_alloc(c, &c->tasks_dev, std::max<size_t>(all.size(), 1), &bytes);
    if (rc) return rc;
    c->base_bytes += bytes;
    if (!all.empty()) {
        cudaError_t e = cudaMemcpy(c->tasks_dev, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "copy tasks");
    }
    // Column-split solver: per layout, runs of up to 32 / (lanes per document)
    // consecutive documents of one bucket (documents are in decreasing length, so a bucket's
    // documents are contiguous), over the documents the layout's buckets hold.
    std::vector<int4> cols;
    for (int li = 0; li < kColLayouts; ++li) {
        const int vrp = 16 << li;
        c->col_off[li] = (int)cols.size();
        c->col_long[li] = 0;
        int d = c->col_first[li];
        while (d < c->Nl) {
            const int b = cols_bucket(c->len_sorted[d], vrp);
            if (b > 32) c->col_long[li] = 1;
            const int per_warp = cols_docs_per_task(b, vrp);
            int k = 0;
            while (d + k < c->Nl && k < per_warp && cols_bucket(c->len_sorted[d + k], vrp) == b) ++k;
            cols.push_back(make_int4(d, k, b, 0));
            d += k;
        }
        c->col_count[li] = (int)cols.size() - c->col_off[li];
    }
    if (cols.empty()) return SWMD_OK;
    bytes = 0;
    if ((rc = dev_alloc(c, &c->col_tasks_dev, cols.size(), &bytes))) return rc;
    c->base_bytes += bytes;
    cudaError_t e = cudaMemcpy(c->col_tasks_dev, cols.data(), sizeof(int4) * cols.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "copy column-split tasks");
    return SWMD_OK;
}

void resident_settings(swmd_corpus *c, int vr, int kprec, int *solver, int *npl_want, int *split) {
    int s = 0, n = 0, cs = 0;
    auto it = c->tuned_resident.find(std::make_pair(vr, kprec));
    if (it != c->tuned_resident.end()) std::tie(s, n, cs) = it->second;
    *solver = c->opt.solver ? c->opt.solver : s;
    *npl_want = c->opt.nnz_per_lane ? c->opt.nnz_per_lane : n;
    *split = c->opt.cost_split ? c->opt.cost_split : cs;
}

bool cols_takes(swmd_corpus *c, int vr, bool *whole) {
    if (whole) *whole = false;
    const int vrp = cols_vrp(vr);
    if (!c->col_tasks_dev || !cols_supported(vrp)) return false;
    const int li = cols_index(vrp);
    if (c->col_count[li] == 0) return false;
    if (c->col_first[li] == 0) {
        if (whole) *whole = true;
        return true;
    }
    return li < 2 && c->tasks_dev && regs_rows_per_lane(vrp, 0) > 0;
}

int resident_solver(swmd_corpus *c, int vr, int kprec) {
    int s = 0, n = 0, cs = 0;
    resident_settings(c, vr, kprec, &s, &n, &cs);
    bool whole = false;
    const bool takes = cols_takes(c, vr, &whole);
    // automatic: the column-split solver where it holds every document in buckets of
    // up to 32 rows.  The longer buckets and the launch that hands the longest
    // documents to the register solver run when asked for or tuned: on the
    // paper-shaped corpus (documents of 10-300 words) that pair of launches took
    // 0.239 ms per query against 0.106 ms for the register solver alone.
    if (s == kSolverAuto && takes && whole && !c->col_long[cols_index(cols_vrp(vr))]) s = kSolverCols;
    if (s == kSolverCols && !takes) s = kSolverAuto;
    return s;
}

int cols_queries_per_group(swmd_corpus *c, int vrp, int kprec) {
    if (c->opt.queries_per_tile > 0) return std::min(c->opt.queries_per_tile, 64);
    auto it = c->tuned_qpt.find(std::make_pair(vrp, kprec));
    if (it != c->tuned_qpt.end()) return it->second;
    const size_t per_query = 2 * (size_t)std::max(c->Vu, 1) * vrp * kprec_bytes(kprec);
    const size_t fit = (c->l2_bytes / 4) / per_query;
    return (int)std::max<size_t>(1, std::min<size_t>(8, fit));
}

int run_resident_batch(swmd_corpus *c, const ResidentArgs &ra, Mapping m, int kprec, int vr, int nq,
                       const ResidentArgs *d_batch, cudaStream_t st) {
    int solver = 0, npl_want = 0, split = 0;
    resident_settings(c, vr, kprec, &solver, &npl_want, &split);
    solver = resident_solver(c, vr, kprec);
    if (solver == kSolverCols && m.vrp == cols_vrp(vr) && cols_supported(m.vrp)) {
        const int li = cols_index(m.vrp);
        if (c->col_first[li] > 0) {
            // the documents too long for the layout's buckets (the first col_first of
            // the sorted order) on the register solver, in a launch before the rest
            int npl = regs_rows_per_lane(m.vrp, npl_want);
            if (npl <= 0) npl = regs_rows_per_lane(m.vrp, 0);
            if (li > 1 || !c->tasks_dev || npl <= 0)
                return set_error(SWMD_EINVAL, "column-split solver (VRP %d): no register solver for its %d "
                                 "longest documents", m.vrp, c->col_first[li]);
            TaskSet ts{c->tasks_dev + c->task_off[npl], c->task_prefix[npl][li], npl, c->len_sorted[0]};
            cudaError_t e = launch_resident_regs(ra, m.vrp, kprec, ts, c->sms, st, nq, d_batch);
            if (e != cudaSuccess)
                return set_error(e == cudaErrorMemoryAllocation ? SWMD_ENOMEM : SWMD_ECUDA,
                                 "register-resident solver for the %d longest documents (VRP %d): %s",
                                 c->col_first[li], m.vrp, cudaGetErrorString(e));
        }
        if (c->col_count[li] == 0) return SWMD_OK;
        ColArgs ca{};
        ca.doc_ptr = c->doc_ptr;
        ca.nz = c->nz;
        ca.doc_orig = c->doc_orig;
        ca.tasks = c->col_tasks_dev + c->col_off[li];
        ca.n_tasks = c->col_count[li];
        ca.long_docs = c->col_long[li];
        ca.Vu = c->Vu;
        ca.nnz = c->nnz;
        ca.kprec = kprec;
        ca.q0 = ra;
        ca.queries = d_batch;
        ca.nq = d_batch ? nq : 1;
        ca.q_per_group = cols_queries_per_group(c, m.vrp, kprec);
        cudaError_t e = launch_resident_cols(ca, m.vrp, c->sms, st, nq);
        if (e != cudaSuccess)
            return set_error(e == cudaErrorMemoryAllocation ? SWMD_ENOMEM : SWMD_ECUDA,
                             "column-split resident solver (VRP %d): %s", m.vrp, cudaGetErrorString(e));
        return SWMD_OK;
    }
    if (solver == kSolverCols) solver = kSolverAuto;   // another layout (explicit lane mapping)
    const int npl = regs_rows_per_lane(m.vrp, npl_want);
    if (c->tasks_dev && npl > 0 && (solver == 0 || solver == 1)) {
        TaskSet ts{c->tasks_dev + c->task_off[npl], c->task_count[npl], npl,
                   c->Nl > 0 ? c->len_sorted[0] : 0};
        cudaError_t e = launch_resident_regs(ra, m.vrp, kprec, ts, c->sms, st, nq, d_batch);
        if (e != cudaSuccess)
            return set_error(e == cudaErrorMemoryAllocation ? SWMD_ENOMEM : SWMD_ECUDA,
                             "register-resident solver (VRP %d, %d rows per lane, longest document %d): %s",
                             m.vrp, npl, ts.max_len, cudaGetErrorString(e));
        return SWMD_OK;
    }
    if (c->tiles_dev && tiled_supported(m.vrp, kprec) && solver != 3) {
        // the largest nonzero budget that fits the requested size, or ~110 KB of
        // shared memory (two blocks per SM) when none is requested
        const int kb = (int)kprec_bytes(kprec);
        int pick = 0;
        for (int i = 0; i < kNumTileBudgets; ++i) {
            const bool fits = c->opt.tile_nnz > 0
                                  ? kTileBudgets[i] <= c->opt.tile_nnz
                                  : tiled_smem_bytes(m.vrp, kb, kTileBudgets[i]) <= 110 * 1024;
            if (fits && tiled_smem_bytes(m.vrp, kb, kTileBudgets[i]) <= 220 * 1024) pick = i;
        }
        TileSet ts{c->tiles_dev + c->tile_off[pick], c->tile_count[pick], kTileBudgets[pick],
                   c->tile_threads, c->tile_npl};
        SWMD_CK(launch_resident_tiled(ra, m.vrp, kprec, ts, c->sms, st, nq, d_batch));
        return SWMD_OK;
    }
    if (nq != 1 || d_batch)
        return set_error(SWMD_EINVAL, "no batched resident solver for VRP %d with these options", m.vrp);
    SWMD_CK(launch_resident(ra, m, kprec, c->sms, st));
    return SWMD_OK;
}

int run_resident(swmd_corpus *c, const ResidentArgs &ra, Mapping m, int kprec, int vr, cudaStream_t st) {
    return run_resident_batch(c, ra, m, kprec, vr, 1, nullptr, st);
}

static int launch_sequence(swmd_corpus *c, Slot &s, Mapping m, int vr, int t, int path, int kprec,
                           int shift, cudaStream_t st) {
    CostArgs ca{};
    ca.E = c->E;
    ca.d4 = c->d4;
    ca.used = c->used;
    ca.Vu = c->Vu;
    ca.q_ids = s.q_ids;
    ca.qp = s.qp;
    ca.V = c->V;
    ca.shift = shift;
    {
        int s_ = 0, n_ = 0, cs_ = 0;
        resident_settings(c, vr, kprec, &s_, &n_, &cs_);
        ca.split = cs_;
    }
    ca.KT = s.KT;
    ca.KMT = s.KMT;
    SWMD_CK(launch_cost(ca, m.vrp, kprec, st));

    IterArgs ia{};
    ia.doc_ptr = c->doc_ptr;
    ia.nz = c->nz;
    ia.KT = s.KT;
    ia.KMT = s.KMT;
    ia.u = s.u;
    ia.r = s.r;
    ia.v = s.v;
    ia.doc_orig = c->doc_orig;
    ia.qp = s.qp;
    ia.doc0 = 0;
    ia.N = c->Nl;
    ia.Vu = c->Vu;
    ia.slice_ptr = c->slice_ptr;
    ia.slice_nz = c->slice_nz;
    ia.n_slices = c->n_slices;
    if (path == SWMD_PATH_RESIDENT) {
        ResidentArgs ra{ia, t};
        ra.it.first = 1;
        return run_resident(c, ra, m, kprec, vr, st);
    }
    ia.conv = s.conv;   // the final step records the x-updates applied
    if (c->opt.tol > 0.f) {
        if (!s.conv) return set_error(SWMD_EINVAL, "convergence mode: this slot has no record");
        ia.tol = c->opt.tol;
        SWMD_CK(cudaMemsetAsync(s.conv, 0, sizeof(unsigned) * (1 + (size_t)t), st));
    }
    if (path == SWMD_PATH_PLAIN && (!s.v || s.v_elems < std::max(c->nnz, c->slice_total)))
        return set_error(SWMD_EINVAL, "plain path: SDDMM output buffer missing or too small");
    for (int it = 0; it < t; ++it) {
        ia.first = it == 0;
        ia.it = it;
        if (path == SWMD_PATH_PLAIN) {
            SWMD_CK(iter_sddmm(ia, m, kprec, c->sms, st));
            ia.first = 0;
            SWMD_CK(iter_spmm(ia, m, kprec, c->sms, st));
        } else {
            SWMD_CK(iter_fused(ia, m, kprec, c->sms, st));
        }
    }
    ia.first = t == 0;
    ia.it = t;
    SWMD_CK(iter_final(ia, m, kprec, c->sms, st));
    return SWMD_OK;
}

int enqueue_query(swmd_corpus *c, Slot &s, const int *d_ids, const float *d_r, int vr,
                  float lambda, int t, double *d_out, int *d_status, cudaStream_t st,
                  bool allow_graph, int path) {
    if (path < 0) path = resolve_path(c, vr);
    const int kprec = c->opt.k_precision;
    if (c->opt.tol > 0.f && path != SWMD_PATH_FUSED)
        return set_error(SWMD_EINVAL, "tol > 0 (convergence mode) needs the fused per-iteration path");
    if (c->opt.tol > 0.f && t > kMaxConvIters)
        return set_error(SWMD_EINVAL, "convergence mode: max_iter %d above %d", t, kMaxConvIters);
    if (!s.external && (s.kprec != kprec || (path == SWMD_PATH_PLAIN && !s.v))) {
        // buffers move: every captured graph of this corpus is stale
        clear_graphs(c);
        int rc = alloc_slot(c, s, c->opt.max_vr, kprec, path == SWMD_PATH_PLAIN);
        if (rc) return rc;
    }
    const Mapping m = choose_mapping(c, vr, path);
    s.cur_vrp = m.vrp;
    s.cur_vr = vr;
    s.last_t = t;
    s.last_path = path;
    SWMD_CK(launch_prep(s.qp, lambda, vr, c->V, d_ids, d_r, s.q_ids, s.r, s.vrp_cap, d_out,
                        d_status ? d_status : s.status, st));
    const int shift = c->opt.column_shift ? 1 : 0;
    if (!(allow_graph && c->opt.use_graph)) return launch_sequence(c, s, m, vr, t, path, kprec, shift, st);

    int solver_ = 0, npl_ = 0, split_ = 0;
    resident_settings(c, vr, kprec, &solver_, &npl_, &split_);
    if (path == SWMD_PATH_RESIDENT) solver_ = resident_solver(c, vr, kprec);
    GraphKey key{m.vrp, m.q, m.p, t, path, kprec, shift, solver_, npl_, split_, (const void *)&s};
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        // The launch sequence of a new shape is captured once on the corpus's own
        // stream and replayed on the caller's stream from then on.
        cudaGraph_t g = nullptr;
        SWMD_CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
        int rc = launch_sequence(c, s, m, vr, t, path, kprec, shift, c->stream);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        SWMD_CK(e);
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        SWMD_CK(e);
        it = c->graphs.emplace(key, ge).first;
    }
    SWMD_CK(cudaGraphLaunch(it->second, st));
    return SWMD_OK;
}

}  // namespace swmd

using namespace swmd;

extern "C" {

void swmd_default_options(swmd_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->k_precision = SWMD_K_FP32;
    opt->path = SWMD_PATH_AUTO;
    opt->use_graph = 1;
    opt->column_shift = 1;
    opt->max_vr = 128;
    opt->device = -1;
    opt->doc_begin = -1;
    opt->doc_end = -1;
}

const char *swmd_last_error(void) { return g_error.c_str(); }

int swmd_set_allocator(swmd_alloc_fn alloc, swmd_free_fn release, void *user) {
    if ((alloc == nullptr) != (release == nullptr))
        return set_error(SWMD_EINVAL, "swmd_set_allocator: give both functions or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_allocator.alloc = alloc;
    g_allocator.release = release;
    g_allocator.user = alloc ? user : nullptr;
    return SWMD_OK;
}

int swmd_select(int32_t V, int32_t n, const int32_t *h_ids, const float *h_weights,
                int32_t *h_out_ids, float *h_out_r, int32_t *out_vr) {
    if (V <= 0 || n < 0 || (n > 0 && (!h_ids || !h_weights || !h_out_ids || !h_out_r)) ||
        !out_vr)
        return set_error(SWMD_EINVAL, "swmd_select: bad arguments");
    // merge repeated ids (sum of weights), keep positive totals, ascending ids
    std::vector<std::pair<int32_t, double>> e;
    e.reserve(n);
    for (int32_t i = 0; i < n; ++i) {
        const double w = h_weights[i];
        if (h_ids[i] < 0 || h_ids[i] >= V)
            return set_error(SWMD_EINVAL, "swmd_select: word id %d outside [0, %d)", h_ids[i], V);
        if (!(w >= 0.0) || std::isinf(w))
            return set_error(SWMD_EINVAL, "swmd_select: weight %g of word %d is not finite and >= 0",
                             w, h_ids[i]);
        e.emplace_back(h_ids[i], w);
    }
    std::sort(e.begin(), e.end(),
              [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                  return a.first < b.first;
              });
    std::vector<std::pair<int32_t, double>> m;
    for (auto &x : e) {
        if (!m.empty() && m.back().first == x.first) m.back().second += x.second;
        else m.push_back(x);
    }
    double total = 0.0;
    int32_t k = 0;
    for (auto &x : m)
        if (x.second > 0.0) total += x.second;
    for (auto &x : m)
        if (x.second > 0.0) {
            h_out_ids[k] = x.first;
            h_out_r[k] = (float)(x.second / total);
            ++k;
        }
    if (k == 0) return set_error(SWMD_EINVAL, "swmd_select: no word has a positive weight");
    *out_vr = k;
    return SWMD_OK;
}

int swmd_partition_documents(int32_t N, const int64_t *doc_nnz, int32_t parts,
                             int32_t *out_bounds) {
    if (N < 0 || parts < 1 || !out_bounds || (N > 0 && !doc_nnz))
        return set_error(SWMD_EINVAL, "swmd_partition_documents: bad arguments");
    std::vector<int64_t> pre((size_t)N + 1, 0);
    for (int32_t j = 0; j < N; ++j) {
        if (doc_nnz[j] < 0) return set_error(SWMD_EINVAL, "swmd_partition_documents: negative count");
        pre[j + 1] = pre[j] + doc_nnz[j];
    }
    // boundary g: the first document whose prefix reaches g/parts of the nonzeros
    out_bounds[0] = 0;
    for (int32_t g = 1; g < parts; ++g) {
        const long double target = (long double)pre[N] * g / parts;
        int32_t j = (int32_t)(std::lower_bound(pre.begin(), pre.end(), (int64_t)(target + 0.5L)) - pre.begin());
        if (j < out_bounds[g - 1]) j = out_bounds[g - 1];
        if (j > N) j = N;
        out_bounds[g] = j;
    }
    out_bounds[parts] = N;
    return SWMD_OK;
}

int swmd_create_corpus(int32_t V, int32_t N, int64_t nnz, const int64_t *row_ptr,
                       const int32_t *doc_idx, const float *val, const float *emb, int32_t d,
                       const swmd_options *opt_in, swmd_corpus **out) {
    if (!out) return set_error(SWMD_EINVAL, "swmd_create_corpus: out is NULL");
    *out = nullptr;
    swmd_options opt;
    if (opt_in) opt = *opt_in;
    else swmd_default_options(&opt);
    if (V <= 0 || N < 0 || d <= 0 || nnz < 0 || nnz >= ((int64_t)1 << 31))
        return set_error(SWMD_EINVAL, "swmd_create_corpus: need V > 0, N >= 0, d > 0, 0 <= nnz < 2^31");
    if (!row_ptr || !emb || (nnz > 0 && (!doc_idx || !val)))
        return set_error(SWMD_EINVAL, "swmd_create_corpus: NULL input array");
    if (opt.max_vr <= 0) opt.max_vr = 128;
    if (opt.max_vr > 128) return set_error(SWMD_EINVAL, "swmd_create_corpus: max_vr above 128");
    if (opt.k_precision < 0 || opt.k_precision > 2 || opt.path < 0 || opt.path > 3 || !(opt.tol >= 0.f) ||
        std::isinf(opt.tol) || opt.queries_per_tile < 0)
        return set_error(SWMD_EINVAL, "swmd_create_corpus: bad k_precision or path");
    int b = opt.doc_begin < 0 ? 0 : opt.doc_begin;
    int e = opt.doc_end < 0 ? N : opt.doc_end;
    if (b > e || e > N) return set_error(SWMD_EINVAL, "swmd_create_corpus: bad document range");

    // ---- validate the CSR (Section III-B1: c is V x N, passed as CSR)
    if (row_ptr[0] != 0 || row_ptr[V] != nnz)
        return set_error(SWMD_EINVAL, "swmd_create_corpus: row_ptr[0] must be 0 and row_ptr[V] = nnz");
    const int Nl = e - b;
    std::vector<int64_t> cnt((size_t)Nl + 1, 0);
    std::vector<double> colsum((size_t)std::max(Nl, 1), 0.0);
    std::vector<char> word_used((size_t)V, 0);
    for (int32_t w = 0; w < V; ++w) {
        if (row_ptr[w + 1] < row_ptr[w])
            return set_error(SWMD_EINVAL, "swmd_create_corpus: row_ptr decreases at row %d", w);
        for (int64_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p) {
            const int32_t j = doc_idx[p];
            const float x = val[p];
            if (j < 0 || j >= N)
                return set_error(SWMD_EINVAL, "swmd_create_corpus: doc_idx[%lld] = %d outside [0, %d)",
                                 (long long)p, j, N);
            if (!(x > 0.f) || std::isinf(x))
                return set_error(SWMD_EINVAL, "swmd_create_corpus: val[%lld] = %g is not finite and > 0",
                                 (long long)p, (double)x);
            if (j >= b && j < e) {
                cnt[j - b + 1]++;
                colsum[j - b] += (double)x;
                word_used[w] = 1;
            }
        }
    }
    for (int j = 0; j < Nl; ++j)
        if (cnt[j + 1] == 0)
            return set_error(SWMD_EINVAL, "swmd_create_corpus: document %d has no words", j + b);

    // ---- compact vocabulary: the words that occur in the loaded documents
    std::vector<int32_t> compact((size_t)V, -1), used;
    for (int32_t w = 0; w < V; ++w)
        if (word_used[w]) {
            compact[w] = (int32_t)used.size();
            used.push_back(w);
        }

    // ---- document-major copy, documents in decreasing length (stable)
    std::vector<int32_t> order((size_t)Nl);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return cnt[x + 1] > cnt[y + 1]; });
    std::vector<int32_t> pos_of((size_t)Nl);
    for (int i = 0; i < Nl; ++i) pos_of[order[i]] = i;
    std::vector<int32_t> dptr((size_t)Nl + 1, 0);
    for (int i = 0; i < Nl; ++i) dptr[i + 1] = dptr[i] + (int32_t)cnt[order[i] + 1];
    const int64_t nnz_l = dptr[Nl];
    std::vector<int2> nzh((size_t)std::max<int64_t>(nnz_l, 1));
    std::vector<int32_t> fill((size_t)Nl, 0);
    for (int32_t w = 0; w < V; ++w)   // rows ascending: each document lists its words ascending
        for (int64_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p) {
            const int32_t j = doc_idx[p];
            if (j < b || j >= e) continue;
            const int32_t i = pos_of[j - b];
            const float cv = (float)((double)val[p] / colsum[j - b]);
            int2 t;
            t.x = compact[w];
            std::memcpy(&t.y, &cv, sizeof cv);
            nzh[(size_t)dptr[i] + fill[i]++] = t;
        }

    // ---- the sliced copy: slices of 32 consecutive documents, entry (i, t) at
    // slice_ptr[s] + 32 i + t, padded with (0, c = 0) to the slice's longest document
    // rounded up to a multiple of kSliceRows rows
    const int n_slices = (Nl + kSliceDocs - 1) / kSliceDocs;
    std::vector<int32_t> sptr((size_t)n_slices + 1, 0);
    for (int s = 0; s < n_slices; ++s) {
        const int64_t rows = (dptr[s * kSliceDocs + 1] - dptr[s * kSliceDocs] + kSliceRows - 1) / kSliceRows * kSliceRows;
        const int64_t next = (int64_t)sptr[s] + (int64_t)kSliceDocs * rows;
        if (next > INT32_MAX) return set_error(SWMD_EINVAL, "swmd_create_corpus: too many nonzeros");
        sptr[s + 1] = (int32_t)next;
    }
    const int64_t slice_total = sptr[n_slices];
    std::vector<int2> snz((size_t)std::max<int64_t>(slice_total, 1), make_int2(0, 0));
    for (int i = 0; i < Nl; ++i) {
        const int s = i / kSliceDocs, t = i % kSliceDocs;
        for (int32_t k = 0; k < dptr[i + 1] - dptr[i]; ++k)
            snz[(size_t)sptr[s] + (size_t)k * kSliceDocs + t] = nzh[(size_t)dptr[i] + k];
    }

    auto *c = new swmd_corpus();
    c->V = V;
    c->n_slices = n_slices;
    c->slice_total = slice_total;
    c->N = N;
    c->d = d;
    c->d4 = (d + 3) / 4 * 4;
    c->Vu = (int)used.size();
    c->nnz = nnz_l;
    c->doc_begin = b;
    c->doc_end = e;
    c->Nl = Nl;
    c->opt = opt;
    c->mean_len = Nl ? (double)nnz_l / Nl : 0.0;
    c->len_sorted.resize((size_t)Nl);
    for (int i = 0; i < Nl; ++i) c->len_sorted[i] = dptr[i + 1] - dptr[i];

    int dev = opt.device;
    if (dev < 0) {
        cudaError_t ce = cudaGetDevice(&dev);
        if (ce != cudaSuccess) {
            delete c;
            return cuda_fail(ce, "cudaGetDevice");
        }
    }
    c->device = dev;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        c->allocator = g_allocator;
    }
    DeviceGuard guard(dev);
    int rc = SWMD_OK;
    auto bail = [&](int code) {
        swmd_destroy_corpus(c);
        return code;
    };
    {
        cudaError_t ce = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
        if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaDeviceGetAttribute"));
        int l2 = 0;
        ce = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaDeviceGetAttribute"));
        c->l2_bytes = (size_t)l2;
        ce = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamCreateWithFlags"));
    }
    if ((rc = dev_alloc(c, &c->E, (size_t)V * c->d4, &c->base_bytes))) return bail(rc);
    if ((rc = dev_alloc(c, &c->used, (size_t)std::max(c->Vu, 1), &c->base_bytes))) return bail(rc);
    if ((rc = dev_alloc(c, &c->doc_ptr, (size_t)Nl + 1, &c->base_bytes))) return bail(rc);
    if ((rc = dev_alloc(c, &c->nz, (size_t)std::max<int64_t>(nnz_l, 1), &c->base_bytes))) return bail(rc);
    if ((rc = dev_alloc(c, &c->doc_orig, (size_t)std::max(Nl, 1), &c->base_bytes))) return bail(rc);
    if ((rc = dev_alloc(c, &c->slice_ptr, (size_t)n_slices + 1, &c->base_bytes))) return bail(rc);
    if ((rc = dev_alloc(c, &c->slice_nz, (size_t)std::max<int64_t>(slice_total, 1), &c->base_bytes)))
        return bail(rc);
    cudaError_t ce;
    if (c->d4 == d) {
        ce = cudaMemcpy(c->E, emb, sizeof(float) * (size_t)V * d, cudaMemcpyHostToDevice);
    } else {
        ce = cudaMemset(c->E, 0, sizeof(float) * (size_t)V * c->d4);
        if (ce == cudaSuccess)
            ce = cudaMemcpy2D(c->E, sizeof(float) * c->d4, emb, sizeof(float) * d, sizeof(float) * d,
                              V, cudaMemcpyHostToDevice);
    }
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "copy embeddings"));
    if (!used.empty() &&
        (ce = cudaMemcpy(c->used, used.data(), sizeof(int32_t) * used.size(),
                         cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(ce, "copy used words"));
    if ((ce = cudaMemcpy(c->doc_ptr, dptr.data(), sizeof(int32_t) * dptr.size(),
                         cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(ce, "copy doc_ptr"));
    if (nnz_l > 0 && (ce = cudaMemcpy(c->nz, nzh.data(), sizeof(int2) * (size_t)nnz_l,
                                      cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(ce, "copy nonzeros"));
    if ((ce = cudaMemcpy(c->slice_ptr, sptr.data(), sizeof(int32_t) * sptr.size(),
                         cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(ce, "copy slice offsets"));
    if (slice_total > 0 && (ce = cudaMemcpy(c->slice_nz, snz.data(), sizeof(int2) * (size_t)slice_total,
                                            cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(ce, "copy sliced nonzeros"));
    if (Nl > 0 && (ce = cudaMemcpy(c->doc_orig, order.data(), sizeof(int32_t) * (size_t)Nl,
                                   cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(ce, "copy document order"));
    if ((rc = build_tiles(c))) return bail(rc);
    if ((rc = build_tasks(c))) return bail(rc);
    if ((rc = alloc_slot(c, c->main, opt.max_vr, opt.k_precision, opt.path == SWMD_PATH_PLAIN)))
        return bail(rc);
    // pinned staging of swmd_query: the query (ids, weights) in, the status word out
    c->h_io_in_bytes = sizeof(int32_t) * 2 * (size_t)c->main.vrp_cap;
    if ((ce = cudaMallocHost(&c->h_io, c->h_io_in_bytes + sizeof(double))) != cudaSuccess)
        return bail(cuda_fail(ce, "pinned staging buffer"));
    *out = c;
    return SWMD_OK;
}

void swmd_destroy_corpus(swmd_corpus *c) {
    if (!c) return;
    {
        DeviceGuard guard(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        clear_graphs(c);
        free_slot(c, c->main);
        dev_free(c, c->batch_ws);
        dev_free(c, c->pair_ws);
        dev_free(c, c->pair_kws);
        dev_free(c, c->E);
        dev_free(c, c->used);
        dev_free(c, c->doc_ptr);
        dev_free(c, c->nz);
        dev_free(c, c->slice_ptr);
        dev_free(c, c->slice_nz);
        dev_free(c, c->doc_orig);
        dev_free(c, c->tiles_dev);
        dev_free(c, c->tasks_dev);
        dev_free(c, c->col_tasks_dev);
        if (c->h_io) cudaFreeHost(c->h_io);
        if (c->stream) cudaStreamDestroy(c->stream);
    }
    delete c;
}

int swmd_corpus_get_info(const swmd_corpus *c, swmd_corpus_info *out) {
    if (!c || !out) return set_error(SWMD_EINVAL, "swmd_corpus_get_info: NULL argument");
    out->V = c->V;
    out->N = c->N;
    out->d = c->d;
    out->V_used = c->Vu;
    out->nnz = c->nnz;
    out->doc_begin = c->doc_begin;
    out->doc_end = c->doc_end;
    out->device = c->device;
    out->device_bytes = c->base_bytes + c->main.bytes;
    return SWMD_OK;
}

int swmd_corpus_get_options(const swmd_corpus *c, swmd_options *out) {
    if (!c || !out) return set_error(SWMD_EINVAL, "swmd_corpus_get_options: NULL argument");
    *out = c->opt;
    return SWMD_OK;
}

int swmd_corpus_set_options(swmd_corpus *c, const swmd_options *opt) {
    if (!c || !opt) return set_error(SWMD_EINVAL, "swmd_corpus_set_options: NULL argument");
    if (opt->k_precision < 0 || opt->k_precision > 2 || opt->path < 0 || opt->path > 3 ||
        !(opt->tol >= 0.f) || std::isinf(opt->tol))
        return set_error(SWMD_EINVAL, "swmd_corpus_set_options: bad k_precision or path");
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->servers > 0)
        return set_error(SWMD_EINVAL, "swmd_corpus_set_options: a server is attached to the corpus");
    c->opt.k_precision = opt->k_precision;
    c->opt.path = opt->path;
    c->opt.use_graph = opt->use_graph;
    c->opt.column_shift = opt->column_shift;
    c->opt.team_lanes = opt->team_lanes;
    c->opt.lanes_per_nz = opt->lanes_per_nz;
    c->opt.tile_threads = opt->tile_threads;
    c->opt.nnz_per_lane = opt->nnz_per_lane;
    c->opt.tile_nnz = opt->tile_nnz;
    c->opt.cost_split = opt->cost_split;
    c->opt.solver = opt->solver;
    c->opt.tol = opt->tol;
    c->opt.queries_per_tile = opt->queries_per_tile;
    clear_graphs(c);
    DeviceGuard guard(c->device);
    return build_tiles(c);
}

static int check_query_args(swmd_corpus *c, int vr, float lambda, int t) {
    if (!c) return set_error(SWMD_EINVAL, "NULL corpus");
    if (vr < 1 || vr > c->opt.max_vr)
        return set_error(SWMD_EINVAL, "query has %d distinct words; allowed 1..%d", vr, c->opt.max_vr);
    if (!(lambda > 0.f) || std::isinf(lambda))
        return set_error(SWMD_EINVAL, "lambda must be finite and > 0");
    if (t < 0) return set_error(SWMD_EINVAL, "max_iter must be >= 0");
    return SWMD_OK;
}

int swmd_query(swmd_corpus *c, const int32_t *h_word_ids, const float *h_weights, int32_t n_words,
               float lambda, int32_t max_iter, double *h_out_dist) {
    if (!c || (c->Nl > 0 && !h_out_dist)) return set_error(SWMD_EINVAL, "swmd_query: NULL argument");
    std::vector<int32_t> ids((size_t)std::max(n_words, 1));
    std::vector<float> r((size_t)std::max(n_words, 1));
    int32_t vr = 0;
    int rc = swmd_select(c->V, n_words, h_word_ids, h_weights, ids.data(), r.data(), &vr);
    if (rc) return rc;
    if ((rc = check_query_args(c, vr, lambda, max_iter))) return rc;
    if (c->Nl == 0) return SWMD_OK;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    Slot &s = c->main;
    cudaStream_t st = c->stream;
    // one pinned copy in (ids at 0, weights at vrp_cap: the slot's q_in / r_in are laid
    // out the same way)
    int32_t *h_in = static_cast<int32_t *>(c->h_io);
    std::memcpy(h_in, ids.data(), sizeof(int32_t) * vr);
    std::memcpy(h_in + s.vrp_cap, r.data(), sizeof(float) * vr);
    SWMD_CK(cudaMemcpyAsync(s.q_in, h_in, sizeof(int32_t) * (size_t)(s.vrp_cap + vr),
                            cudaMemcpyHostToDevice, st));
    if ((rc = enqueue_query(c, s, s.q_in, s.r_in, vr, lambda, max_iter, s.out, s.status, st, true)))
        return rc;
    // the distances straight into the caller's buffer (a copy through the pinned
    // staging plus a host memcpy took 10x as long for 8 MB on a GB300 host); the
    // status word into the staging
    int *h_res = reinterpret_cast<int *>(static_cast<char *>(c->h_io) + c->h_io_in_bytes);
    SWMD_CK(cudaMemcpyAsync(h_out_dist, s.out, sizeof(double) * c->Nl, cudaMemcpyDeviceToHost, st));
    SWMD_CK(cudaMemcpyAsync(h_res, s.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SWMD_CK(cudaStreamSynchronize(st));
    int h_status = 0;
    std::memcpy(&h_status, h_res, sizeof(int));
    return status_to_code(h_status);
}

int swmd_query_device(swmd_corpus *c, const int32_t *d_ids, const float *d_r, int32_t v_r,
                      float lambda, int32_t max_iter, double *d_out, int32_t *d_status,
                      void *stream) {
    int rc = check_query_args(c, v_r, lambda, max_iter);
    if (rc) return rc;
    if (!d_ids || !d_r || (c->Nl > 0 && !d_out))
        return set_error(SWMD_EINVAL, "swmd_query_device: NULL device pointer");
    if (c->Nl == 0) return SWMD_OK;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    return enqueue_query(c, c->main, d_ids, d_r, v_r, lambda, max_iter, d_out, d_status, st, true);
}

// ---------------------------------------------------------------- the steps
// VRP of the K^T layout the last swmd_step_cost / query wrote (v_r's default
// layout for the corpus's path if none yet)
static int slot_vrp(swmd_corpus *c, Slot &s, int v_r) {
    return (s.cur_vrp > 0 && s.cur_vr == v_r) ? s.cur_vrp : layout_vrp(c, v_r, resolve_path(c, v_r));
}

static IterArgs iter_args(swmd_corpus *c, Slot &s) {
    IterArgs ia{};
    ia.doc_ptr = c->doc_ptr;
    ia.nz = c->nz;
    ia.KT = s.KT;
    ia.KMT = s.KMT;
    ia.u = s.u;
    ia.r = s.r;
    ia.v = s.v;
    ia.doc_orig = c->doc_orig;
    ia.qp = s.qp;
    ia.doc0 = 0;
    ia.N = c->Nl;
    ia.Vu = c->Vu;
    ia.slice_ptr = c->slice_ptr;
    ia.slice_nz = c->slice_nz;
    ia.n_slices = c->n_slices;
    return ia;
}

int swmd_step_cost(swmd_corpus *c, const int32_t *d_ids, const float *d_r, int32_t v_r,
                   float lambda, int32_t *d_status, void *stream) {
    int rc = check_query_args(c, v_r, lambda, 0);
    if (rc) return rc;
    if (!d_ids) return set_error(SWMD_EINVAL, "swmd_step_cost: NULL ids");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    Slot &s = c->main;
    if (s.kprec != c->opt.k_precision) {
        clear_graphs(c);
        if ((rc = alloc_slot(c, s, c->opt.max_vr, c->opt.k_precision, c->opt.path == SWMD_PATH_PLAIN)))
            return rc;
    }
    const Mapping m = choose_mapping(c, v_r, resolve_path(c, v_r));
    s.cur_vrp = m.vrp;
    s.cur_vr = v_r;
    SWMD_CK(launch_prep(s.qp, lambda, v_r, c->V, d_ids, d_r, s.q_ids, s.r, s.vrp_cap, s.out,
                        d_status ? d_status : s.status, st));
    CostArgs ca{};
    ca.E = c->E;
    ca.d4 = c->d4;
    ca.used = c->used;
    ca.Vu = c->Vu;
    ca.q_ids = s.q_ids;
    ca.qp = s.qp;
    ca.V = c->V;
    ca.shift = c->opt.column_shift ? 1 : 0;
    {
        int s_ = 0, n_ = 0, cs_ = 0;
        resident_settings(c, v_r, c->opt.k_precision, &s_, &n_, &cs_);
        ca.split = cs_;
    }
    ca.KT = s.KT;
    ca.KMT = s.KMT;
    SWMD_CK(launch_cost(ca, m.vrp, c->opt.k_precision, st));
    return SWMD_OK;
}

int swmd_step_iterate(swmd_corpus *c, int32_t v_r, int32_t n_iter, int32_t first, int32_t path,
                      void *stream) {
    int rc = check_query_args(c, v_r, 1.f, n_iter);
    if (rc) return rc;
    if (path != SWMD_PATH_FUSED && path != SWMD_PATH_PLAIN)
        return set_error(SWMD_EINVAL, "swmd_step_iterate: path must be FUSED or PLAIN");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    Slot &s = c->main;
    if (path == SWMD_PATH_PLAIN && !s.v) {
        int64_t extra = 0;
        s.v_elems = std::max<int64_t>(std::max(c->nnz, c->slice_total), 1);
        if ((rc = dev_alloc(c, &s.v, (size_t)s.v_elems, &extra))) return rc;
        s.bytes += extra;
        clear_graphs(c);
    }
    if (path == SWMD_PATH_PLAIN && s.v_elems < std::max(c->nnz, c->slice_total))
        return set_error(SWMD_EINVAL, "swmd_step_iterate: SDDMM output buffer too small");
    const Mapping m = walk_mapping(c, slot_vrp(c, s, v_r), path);
    IterArgs ia = iter_args(c, s);
    for (int it = 0; it < n_iter; ++it) {
        ia.first = (first && it == 0) ? 1 : 0;
        if (path == SWMD_PATH_PLAIN) {
            SWMD_CK(iter_sddmm(ia, m, c->opt.k_precision, c->sms, st));
            ia.first = 0;
            SWMD_CK(iter_spmm(ia, m, c->opt.k_precision, c->sms, st));
        } else {
            SWMD_CK(iter_fused(ia, m, c->opt.k_precision, c->sms, st));
        }
    }
    return SWMD_OK;
}

int swmd_step_final(swmd_corpus *c, int32_t v_r, int32_t t0, double *d_out, void *stream) {
    int rc = check_query_args(c, v_r, 1.f, 0);
    if (rc) return rc;
    if (!d_out && c->Nl > 0) return set_error(SWMD_EINVAL, "swmd_step_final: NULL output");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    Slot &s = c->main;
    const Mapping m = walk_mapping(c, slot_vrp(c, s, v_r), SWMD_PATH_FUSED);
    IterArgs ia = iter_args(c, s);
    ia.first = t0 ? 1 : 0;
    ia.out = d_out;
    SWMD_CK(iter_final(ia, m, c->opt.k_precision, c->sms, st));
    return SWMD_OK;
}

int swmd_step_resident(swmd_corpus *c, int32_t v_r, int32_t max_iter, double *d_out,
                       void *stream) {
    int rc = check_query_args(c, v_r, 1.f, max_iter);
    if (rc) return rc;
    if (!d_out && c->Nl > 0) return set_error(SWMD_EINVAL, "swmd_step_resident: NULL output");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    Slot &s = c->main;
    const int vrp = slot_vrp(c, s, v_r);
    const Mapping m = walk_mapping(c, vrp, SWMD_PATH_RESIDENT);
    ResidentArgs ra{iter_args(c, s), max_iter};
    ra.it.out = d_out;
    return run_resident(c, ra, m, c->opt.k_precision, v_r, st);
}

int swmd_get_mapping(swmd_corpus *c, int32_t v_r, int32_t path, int32_t *out3) {
    if (!c || !out3) return set_error(SWMD_EINVAL, "swmd_get_mapping: NULL argument");
    if (v_r < 1 || v_r > c->opt.max_vr) return set_error(SWMD_EINVAL, "swmd_get_mapping: bad v_r");
    std::lock_guard<std::mutex> lk(c->mu);
    if (path == SWMD_PATH_AUTO) path = resolve_path(c, v_r);
    const Mapping m = choose_mapping(c, v_r, path);
    out3[0] = m.vrp;
    out3[1] = m.q;
    out3[2] = m.p;
    if (m.p == 0 && path != SWMD_PATH_RESIDENT) {
        // the sliced walk's team: a 32-byte slice of every row per lane
        const int eb = (int)kprec_bytes(c->opt.k_precision);
        const int per_lane = m.vrp * eb >= 32 ? 32 / eb : m.vrp;
        out3[1] = m.vrp / per_lane;
    }
    return SWMD_OK;
}

int swmd_last_iterations(swmd_corpus *c, int32_t *out_iterations) {
    if (!c || !out_iterations) return set_error(SWMD_EINVAL, "swmd_last_iterations: NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    // only the per-iteration walks stop early; the resident path always applies all
    unsigned v = (unsigned)c->main.last_t;
    if (c->main.conv && c->main.last_path == SWMD_PATH_FUSED) {
        SWMD_CK(cudaMemcpyAsync(&v, c->main.conv, sizeof v, cudaMemcpyDeviceToHost, c->stream));
        SWMD_CK(cudaStreamSynchronize(c->stream));
    }
    *out_iterations = (int32_t)v;
    return SWMD_OK;
}

int swmd_resolve_path(swmd_corpus *c, int32_t v_r, int32_t *out_path) {
    if (!c || !out_path) return set_error(SWMD_EINVAL, "swmd_resolve_path: NULL argument");
    if (v_r < 1 || v_r > c->opt.max_vr) return set_error(SWMD_EINVAL, "swmd_resolve_path: bad v_r");
    std::lock_guard<std::mutex> lk(c->mu);
    *out_path = resolve_path(c, v_r);
    return SWMD_OK;
}

int swmd_debug_plant(swmd_corpus *c, int32_t what, int64_t index, int32_t value) {
#if SWMD_DEBUG_CHECKS
    if (!c || (what != 0 && what != 1)) return set_error(SWMD_EINVAL, "swmd_debug_plant: bad arguments");
    const int64_t n = what == 0 ? c->nnz : c->slice_total;
    if (index < 0 || index >= n) return set_error(SWMD_EINVAL, "swmd_debug_plant: index outside [0, %lld)", (long long)n);
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    SWMD_CK(cudaStreamSynchronize(c->stream));
    int2 *dst = (what == 0 ? c->nz : c->slice_nz) + index;
    SWMD_CK(cudaMemcpy(&dst->x, &value, sizeof value, cudaMemcpyHostToDevice));
    return SWMD_OK;
#else
    (void)c;
    (void)what;
    (void)index;
    (void)value;
    return set_error(SWMD_EINVAL, "swmd_debug_plant: available in debug builds only (build(debug=True))");
#endif
}

int swmd_debug_read(swmd_corpus *c, int32_t what, int32_t v_r, void *h_dst) {
    if (!c || !h_dst) return set_error(SWMD_EINVAL, "swmd_debug_read: NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    SWMD_CK(cudaStreamSynchronize(c->stream));
    SWMD_CK(cudaDeviceSynchronize());
    Slot &s = c->main;
    if (what == 3) {
        SWMD_CK(cudaMemcpy(h_dst, c->used, sizeof(int32_t) * c->Vu, cudaMemcpyDeviceToHost));
        return SWMD_OK;
    }
    if (v_r < 1 || v_r > c->opt.max_vr) return set_error(SWMD_EINVAL, "swmd_debug_read: bad v_r");
    const int vrp = slot_vrp(c, s, v_r);
    float *dst = static_cast<float *>(h_dst);
    if (what == 0 || what == 1) {
        const size_t kb = kprec_bytes(s.kprec);
        std::vector<unsigned char> raw((size_t)c->Vu * vrp * kb);
        SWMD_CK(cudaMemcpy(raw.data(), what == 0 ? s.KT : s.KMT, raw.size(), cudaMemcpyDeviceToHost));
        for (size_t w = 0; w < (size_t)c->Vu; ++w)
            for (int k = 0; k < v_r; ++k) {
                const size_t i = w * vrp + k;
                float x;
                if (s.kprec == 0) std::memcpy(&x, raw.data() + 4 * i, 4);
                else if (s.kprec == 1) x = __bfloat162float(*reinterpret_cast<__nv_bfloat16 *>(raw.data() + 2 * i));
                else x = __half2float(*reinterpret_cast<__half *>(raw.data() + 2 * i));
                dst[w * v_r + k] = x;
            }
        return SWMD_OK;
    }
    if (what == 2) {
        std::vector<float> uu((size_t)c->Nl * vrp);
        std::vector<int32_t> orig((size_t)c->Nl);
        SWMD_CK(cudaMemcpy(uu.data(), s.u, sizeof(float) * uu.size(), cudaMemcpyDeviceToHost));
        SWMD_CK(cudaMemcpy(orig.data(), c->doc_orig, sizeof(int32_t) * orig.size(), cudaMemcpyDeviceToHost));
        for (int i = 0; i < c->Nl; ++i)
            for (int k = 0; k < v_r; ++k) dst[(size_t)orig[i] * v_r + k] = uu[(size_t)i * vrp + k];
        return SWMD_OK;
    }
    return set_error(SWMD_EINVAL, "swmd_debug_read: unknown array %d", what);
}

}  // extern "C"
