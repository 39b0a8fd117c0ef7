// Multi-query batches and the query server.
//
// Section III-D and Section V run many source documents against the same
// targets; here that is (1) swmd_query_batch, a host call that runs a list of
// queries over the resident corpus, and (2) a server that keeps the corpus on
// the device and admits queries continuously.  Each admitted query gets a slot
// (parameter block, pinned staging, an event) and device memory for its K^T,
// KM^T (and u on the per-iteration paths) carved from a fixed arena, so
// admission is by the bytes a query of v_r words needs.  Queries on the
// column-split solver are admitted in groups (same layout and cost split) that
// run as one batched cost launch and one multi-query solver launch on the batch
// lane, two groups deep, so the next group is queued while one runs; other
// queries run alone on their slot's stream.  Finished slots are refilled at once.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "corpus.h"

using namespace swmd;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device buffer (offsets aligned to 256 bytes).
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::vector<std::pair<size_t, size_t>> free_list;  // (offset, length), sorted by offset

    void init(char *b, size_t n) {
        base = b;
        size = n;
        free_list.assign(1, {0, n});
    }
    void *alloc(size_t n) {
        n = (n + 255) & ~size_t(255);
        for (size_t i = 0; i < free_list.size(); ++i) {
            if (free_list[i].second >= n) {
                const size_t off = free_list[i].first;
                free_list[i].first += n;
                free_list[i].second -= n;
                if (free_list[i].second == 0) free_list.erase(free_list.begin() + (long)i);
                return base + off;
            }
        }
        return nullptr;
    }
    void release(void *p, size_t n) {
        n = (n + 255) & ~size_t(255);
        const size_t off = (size_t)((char *)p - base);
        auto it = std::lower_bound(free_list.begin(), free_list.end(), std::make_pair(off, size_t(0)));
        it = free_list.insert(it, {off, n});
        // merge with neighbours
        size_t i = (size_t)(it - free_list.begin());
        if (i + 1 < free_list.size() && free_list[i].first + free_list[i].second == free_list[i + 1].first) {
            free_list[i].second += free_list[i + 1].second;
            free_list.erase(free_list.begin() + (long)i + 1);
        }
        if (i > 0 && free_list[i - 1].first + free_list[i - 1].second == free_list[i].first) {
            free_list[i - 1].second += free_list[i].second;
            free_list.erase(free_list.begin() + (long)i);
        }
    }
};

struct Request {
    uint64_t ticket = 0;
    std::vector<int32_t> ids;
    std::vector<float> r;
    int vr = 0;
    float lambda = 1.f;
    int t = 0;
    int path = -1;   // resolved once, at admission
    int vrp = 0;     // its K^T layout
    int group = -1;  // >= 0: runs with the other requests of this key in one multi-query
                     // launch (column-split solver: layout and cost split); -1: alone
    double t_submit = 0, t_done = 0;
    int state = 0;  // 0 queued, 1 running, 2 finished
    int code = SWMD_OK;
    std::string err;
    std::vector<double> result;
};

struct ServerSlot {
    Slot ws;                  // small arrays owned here; K^T / KM^T / u from the arena
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int32_t *h_q = nullptr;   // pinned staging
    float *h_r = nullptr;
    int *h_status = nullptr;
    std::vector<double> result;   // the finished query's distances, copied from ws.out
    std::shared_ptr<Request> req;
    size_t arena_bytes = 0;
    void *arena_ptr = nullptr;
    int lane = -1;            // the batch lane running it (-1: its own stream)
    int lane_buf = -1;        // ... and the argument buffer of its group
};

// A stream on which groups of requests run as batched launch sequences, one after
// another in stream order.  Two argument buffers (device and pinned host copies of
// the per-query argument arrays): a group can be queued behind the running one, so
// the GPU does not wait while the host collects one group and stages the next.
constexpr int kLaneDepth = 2;
struct BatchLane {
    cudaStream_t stream = nullptr;
    char *d_args[kLaneDepth] = {};
    char *h_args[kLaneDepth] = {};
    size_t args_bytes = 0;
    int outstanding[kLaneDepth] = {};   // members of the group using each buffer (0: free)
};

size_t query_bytes(swmd_corpus *c, int vrp, int path) {
    size_t b = 2 * (size_t)c->Vu * vrp * kprec_bytes(c->opt.k_precision);
    if (path != SWMD_PATH_RESIDENT) b += (size_t)c->Nl * vrp * sizeof(float);
    if (path == SWMD_PATH_PLAIN) b += (size_t)std::max(c->nnz, c->slice_total) * sizeof(float);
    return b + 3 * 256;
}

}  // namespace

struct swmd_server {
    swmd_corpus *c = nullptr;
    swmd_serve_config cfg{};
    std::vector<ServerSlot> slots;
    std::vector<BatchLane> lanes;
    cudaStream_t copy_stream = nullptr;   // finished queries' distances to host memory
    std::vector<std::vector<double>> spare;   // result buffers given back by waiters (pages touched)
    Arena arena;
    char *arena_mem = nullptr;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> table;
    bool stopping = false;
    std::thread worker;
    uint64_t next_ticket = 1;
    // statistics
    std::vector<double> lat_ms;
    int64_t completed = 0, rejected = 0, batches = 0, admitted = 0;
    int waiters = 0;   // threads inside swmd_serve_wait (swmd_serve_stop frees only at 0)
    double t_first = -1, t_last = -1;
};

namespace {

void finish(swmd_server *S, ServerSlot &sl, int code, const std::string &err) {
    auto &R = *sl.req;
    R.code = code;
    R.err = err;
    R.state = 2;
    R.t_done = now_s();
    if (code == SWMD_OK || code == SWMD_ENUMERIC) R.result = std::move(sl.result);
    sl.result = std::vector<double>();
    S->completed++;
    S->lat_ms.push_back((R.t_done - R.t_submit) * 1e3);
    S->t_last = R.t_done;
    if (sl.arena_ptr) S->arena.release(sl.arena_ptr, sl.arena_bytes);
    sl.arena_ptr = nullptr;
    if (sl.lane >= 0) S->lanes[(size_t)sl.lane].outstanding[sl.lane_buf]--;
    sl.lane = -1;
    sl.lane_buf = -1;
    sl.req.reset();
}

size_t up256(size_t n) { return (n + 255) & ~size_t(255); }

// Batch shapes remembered (as captured graphs, or as seen once); beyond this many
// the memory is dropped and shapes start over.
constexpr size_t kMaxBatchShapes = 64;
size_t lane_args_bytes(int n) {
    return up256(sizeof(PrepArgs) * n) + up256(sizeof(CostArgs) * n) + up256(sizeof(ResidentArgs) * n);
}

// Launches a group of admitted requests (one column-split layout and cost split) on
// a batch lane: their queries are staged, then one batched parameter launch, one
// batched cost launch and one multi-query solver launch run them all; each slot's
// distances and status come back to its pinned staging and its event marks the end.
int launch_group(swmd_server *S, int li, int buf, const std::vector<ServerSlot *> &members) {
    swmd_corpus *c = S->c;
    BatchLane &L = S->lanes[(size_t)li];
    char *const h_args = L.h_args[buf];
    char *const d_args = L.d_args[buf];
    const int n = (int)members.size();
    const int kprec = c->opt.k_precision;
    const int vrp = members[0]->req->vrp;
    const size_t kbytes = (size_t)c->Vu * vrp * kprec_bytes(kprec);
    PrepArgs *hp = reinterpret_cast<PrepArgs *>(h_args);
    CostArgs *hc = reinterpret_cast<CostArgs *>(h_args + up256(sizeof(PrepArgs) * n));
    ResidentArgs *hr = reinterpret_cast<ResidentArgs *>(h_args + up256(sizeof(PrepArgs) * n) +
                                                        up256(sizeof(CostArgs) * n));
    const size_t off_c = up256(sizeof(PrepArgs) * n), off_r = off_c + up256(sizeof(CostArgs) * n);
    int split = 0;
    for (int i = 0; i < n; ++i) {
        ServerSlot &sl = *members[i];
        auto &R = *sl.req;
        char *p = static_cast<char *>(sl.arena_ptr);
        sl.ws.KT = p;
        sl.ws.KMT = p + up256(kbytes);
        sl.ws.u = nullptr;
        sl.ws.v = nullptr;
        sl.lane = li;
        sl.lane_buf = buf;
        std::memcpy(sl.h_q, R.ids.data(), sizeof(int32_t) * R.vr);
        std::memcpy(sl.h_r, R.r.data(), sizeof(float) * R.vr);
        SWMD_CK(cudaMemcpyAsync(sl.ws.q_in, sl.h_q, sizeof(int32_t) * R.vr, cudaMemcpyHostToDevice, L.stream));
        SWMD_CK(cudaMemcpyAsync(sl.ws.r_in, sl.h_r, sizeof(float) * R.vr, cudaMemcpyHostToDevice, L.stream));
        PrepArgs &pa = hp[i];
        pa = PrepArgs{};
        pa.qp = sl.ws.qp;
        pa.src_ids = sl.ws.q_in;
        pa.src_r = sl.ws.r_in;
        pa.q_ids = sl.ws.q_ids;
        pa.r = sl.ws.r;
        pa.out = sl.ws.out;
        pa.status = sl.ws.status;
        pa.lambda = R.lambda;
        pa.vr = R.vr;
        pa.vrp_cap = vrp;
        int s_ = 0, n_ = 0;
        resident_settings(c, R.vr, kprec, &s_, &n_, &split);
        CostArgs &ca = hc[i];
        ca = CostArgs{};
        ca.E = c->E;
        ca.d4 = c->d4;
        ca.used = c->used;
        ca.Vu = c->Vu;
        ca.q_ids = sl.ws.q_ids;
        ca.qp = sl.ws.qp;
        ca.V = c->V;
        ca.shift = c->opt.column_shift ? 1 : 0;
        ca.split = split;
        ca.KT = sl.ws.KT;
        ca.KMT = sl.ws.KMT;
        IterArgs ia{};
        ia.doc_ptr = c->doc_ptr;
        ia.nz = c->nz;
        ia.KT = sl.ws.KT;
        ia.KMT = sl.ws.KMT;
        ia.r = sl.ws.r;
        ia.doc_orig = c->doc_orig;
        ia.qp = sl.ws.qp;
        ia.N = c->Nl;
        ia.Vu = c->Vu;
        ia.first = 1;
        hr[i] = ResidentArgs{ia, R.t};
    }
    SWMD_CK(cudaMemcpyAsync(d_args, h_args, lane_args_bytes(n), cudaMemcpyHostToDevice, L.stream));
    SWMD_CK(launch_prep_batch(reinterpret_cast<const PrepArgs *>(d_args), n, c->V, L.stream));
    // the cost and solver launches one tile group at a time: the group's K^T and KM^T,
    // just written, are still in L2 when its solver runs
    const Mapping m = walk_mapping(c, vrp, SWMD_PATH_RESIDENT);
    const int step = cols_queries_per_group(c, vrp, kprec);
    for (int j0 = 0; j0 < n; j0 += step) {
        const int nj = std::min(step, n - j0);
        SWMD_CK(launch_cost_batch(hc[j0], vrp, kprec, nj, reinterpret_cast<const CostArgs *>(d_args + off_c) + j0,
                                  L.stream));
        int rc = run_resident_batch(c, hr[j0], m, kprec, members[j0]->req->vr, nj,
                                    reinterpret_cast<const ResidentArgs *>(d_args + off_r) + j0, L.stream);
        if (rc) return rc;
    }
    for (ServerSlot *sl : members) {
        SWMD_CK(cudaMemcpyAsync(sl->h_status, sl->ws.status, sizeof(int), cudaMemcpyDeviceToHost, L.stream));
        SWMD_CK(cudaEventRecord(sl->done, L.stream));
    }
    return SWMD_OK;
}

// Launches one admitted request on its slot.  Returns an SWMD code.
int launch_on_slot(swmd_server *S, ServerSlot &sl) {
    swmd_corpus *c = S->c;
    auto &R = *sl.req;
    const int path = R.path;
    const size_t kbytes = (size_t)c->Vu * R.vrp * kprec_bytes(c->opt.k_precision);
    char *p = static_cast<char *>(sl.arena_ptr);
    auto carve = [&](size_t n) {
        char *q = p;
        p += (n + 255) & ~size_t(255);
        return (void *)q;
    };
    sl.ws.KT = carve(kbytes);
    sl.ws.KMT = carve(kbytes);
    sl.ws.u = path != SWMD_PATH_RESIDENT ? (float *)carve((size_t)c->Nl * R.vrp * sizeof(float)) : nullptr;
    sl.ws.v_elems = path == SWMD_PATH_PLAIN ? std::max(c->nnz, c->slice_total) : 0;
    sl.ws.v = path == SWMD_PATH_PLAIN ? (float *)carve((size_t)sl.ws.v_elems * sizeof(float)) : nullptr;
    std::memcpy(sl.h_q, R.ids.data(), sizeof(int32_t) * R.vr);
    std::memcpy(sl.h_r, R.r.data(), sizeof(float) * R.vr);
    SWMD_CK(cudaMemcpyAsync(sl.ws.q_in, sl.h_q, sizeof(int32_t) * R.vr, cudaMemcpyHostToDevice, sl.stream));
    SWMD_CK(cudaMemcpyAsync(sl.ws.r_in, sl.h_r, sizeof(float) * R.vr, cudaMemcpyHostToDevice, sl.stream));
    int rc;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        rc = enqueue_query(c, sl.ws, sl.ws.q_in, sl.ws.r_in, R.vr, R.lambda, R.t, sl.ws.out,
                           sl.ws.status, sl.stream, false, path);
    }
    if (rc) return rc;
    SWMD_CK(cudaMemcpyAsync(sl.h_status, sl.ws.status, sizeof(int), cudaMemcpyDeviceToHost, sl.stream));
    SWMD_CK(cudaEventRecord(sl.done, sl.stream));
    return SWMD_OK;
}

void worker_main(swmd_server *S) {
    DeviceGuard guard(S->c->device);
    std::unique_lock<std::mutex> lk(S->m);
    for (;;) {
        bool running = false;
        for (auto &sl : S->slots) running |= (bool)sl.req;
        if (S->stopping && !running) break;
        if (!running && S->pending.empty()) {
            S->cv_work.wait(lk);
            continue;
        }
        // admit: fill free slots while the arena has room.  Requests on the
        // column-split solver go to a free batch lane together with every pending
        // request of the same group key (one multi-query launch); the others run
        // alone on their slot's stream.
        std::vector<ServerSlot *> launched;
        std::vector<std::pair<std::pair<int, int>, std::vector<ServerSlot *>>> groups;   // ((lane, buffer), members)
        if (!S->stopping) {
            size_t next_slot = 0;
            auto free_slot = [&]() -> ServerSlot * {
                while (next_slot < S->slots.size() && S->slots[next_slot].req) ++next_slot;
                return next_slot < S->slots.size() ? &S->slots[next_slot] : nullptr;
            };
            int lane = -1, lane_buf = -1;
            for (size_t li = 0; li < S->lanes.size() && lane < 0; ++li)
                for (int b = 0; b < kLaneDepth; ++b)
                    if (S->lanes[li].outstanding[b] == 0) {
                        lane = (int)li;
                        lane_buf = b;
                        break;
                    }
            int gkey = -1;
            std::vector<ServerSlot *> members;
            bool blocked = false;   // a request alone could not be admitted: keep FIFO order for them
            for (auto it = S->pending.begin(); it != S->pending.end();) {
                auto R = *it;
                if (R->path < 0) {   // the path and layout, once (options cannot change while served)
                    std::lock_guard<std::mutex> cl(S->c->mu);
                    R->path = resolve_path(S->c, R->vr);
                    R->vrp = choose_mapping(S->c, R->vr, R->path).vrp;
                    if (R->path == SWMD_PATH_RESIDENT &&
                        resident_solver(S->c, R->vr, S->c->opt.k_precision) == kSolverCols) {
                        int s_ = 0, n_ = 0, cs_ = 0;
                        resident_settings(S->c, R->vr, S->c->opt.k_precision, &s_, &n_, &cs_);
                        R->group = R->vrp * 8 + cs_;
                    }
                }
                const bool grouped = R->group >= 0;
                if (grouped && (lane < 0 || (gkey >= 0 && R->group != gkey))) { ++it; continue; }
                if (!grouped && blocked) { ++it; continue; }
                ServerSlot *sl = free_slot();
                if (!sl) break;
                const size_t need = query_bytes(S->c, R->vrp, R->path);
                void *mem = S->arena.alloc(need);
                if (!mem) {   // admission waits for memory to free up
                    if (grouped) { ++it; continue; }
                    blocked = true;
                    ++it;
                    continue;
                }
                it = S->pending.erase(it);
                sl->req = R;
                sl->arena_ptr = mem;
                sl->arena_bytes = need;
                R->state = 1;
                if (grouped) {
                    gkey = R->group;
                    members.push_back(sl);
                } else {
                    launched.push_back(sl);
                }
            }
            if (!members.empty()) {
                S->lanes[(size_t)lane].outstanding[lane_buf] = (int)members.size();
                groups.emplace_back(std::make_pair(lane, lane_buf), members);
            }
        }
        if (!launched.empty() || !groups.empty()) {
            S->batches += (int64_t)launched.size() + (int64_t)groups.size();
            for (auto &g : groups) S->admitted += (int64_t)g.second.size();
            S->admitted += (int64_t)launched.size();
        }
        lk.unlock();
        std::vector<std::pair<ServerSlot *, int>> failed;
        for (auto *sl : launched) {
            const int rc = launch_on_slot(S, *sl);
            if (rc) failed.push_back({sl, rc});
        }
        for (auto &g : groups) {
            int rc;
            {
                std::lock_guard<std::mutex> cl(S->c->mu);
                rc = launch_group(S, g.first.first, g.first.second, g.second);
            }
            if (rc) {
                cudaStreamSynchronize(S->lanes[(size_t)g.first.first].stream);
                for (ServerSlot *sl : g.second) failed.push_back({sl, rc});
            }
        }
        // poll in-flight slots
        std::vector<ServerSlot *> ready;
        for (auto &sl : S->slots) {
            if (!sl.req) continue;
            bool is_failed = false;
            for (auto &f : failed) is_failed |= f.first == &sl;
            if (is_failed) continue;
            if (sl.req->state == 1 && cudaEventQuery(sl.done) == cudaSuccess) ready.push_back(&sl);
        }
        if (!ready.empty()) {
            // the distances go from the slot's device buffer straight into host memory
            // the request keeps (recycled buffers, their pages already touched)
            lk.lock();
            for (auto *sl : ready)
                if (!S->spare.empty()) {
                    sl->result = std::move(S->spare.back());
                    S->spare.pop_back();
                }
            lk.unlock();
            cudaError_t ce = cudaSuccess;
            for (auto *sl : ready) {
                sl->result.resize((size_t)S->c->Nl);
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(sl->result.data(), sl->ws.out, sizeof(double) * S->c->Nl,
                                         cudaMemcpyDeviceToHost, S->copy_stream);
            }
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(S->copy_stream);
            if (ce != cudaSuccess) {
                const int rc = cuda_fail(ce, "serve: copy distances");
                for (auto *sl : ready) failed.push_back({sl, rc});
                ready.clear();
            }
        }
        const std::string last = swmd_last_error();
        lk.lock();
        for (auto &f : failed) {
            cudaStreamSynchronize(f.first->stream);   // nothing of it may still use its memory
            finish(S, *f.first, f.second, last);
        }
        for (auto *sl : ready) {
            const int code = status_to_code(*sl->h_status);
            finish(S, *sl, code, code ? std::string(swmd_last_error()) : std::string());
        }
        if (!failed.empty() || !ready.empty()) S->cv_done.notify_all();
        bool busy = false;
        for (auto &sl : S->slots) busy |= (bool)sl.req;
        if (busy && ready.empty() && launched.empty() && groups.empty()) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(
                std::max(5, std::min(S->cfg.max_wait_us, 200))));
            lk.lock();
        }
    }
    // fail whatever is still queued
    for (auto &R : S->pending) {
        R->state = 2;
        R->code = SWMD_ESTOPPED;
        R->err = "server stopped";
    }
    S->pending.clear();
    S->cv_done.notify_all();
}

}  // namespace

extern "C" {

int swmd_query_batch(swmd_corpus *c, int32_t n_queries, const int64_t *q_ptr,
                     const int32_t *h_word_ids, const float *h_weights, const float *h_lambdas,
                     int32_t max_iter, double *h_out) {
    if (!c || n_queries < 0 || (n_queries > 0 && (!q_ptr || !h_lambdas || !h_out)))
        return set_error(SWMD_EINVAL, "swmd_query_batch: bad arguments");
    if (max_iter < 0) return set_error(SWMD_EINVAL, "swmd_query_batch: max_iter must be >= 0");
    if (n_queries == 0 || c->Nl == 0) return SWMD_OK;
    if (q_ptr[0] != 0) return set_error(SWMD_EINVAL, "swmd_query_batch: q_ptr[0] must be 0");
    std::vector<int32_t> ids;
    std::vector<float> rs;
    std::vector<int64_t> off((size_t)n_queries + 1, 0);
    std::vector<int32_t> vrs((size_t)n_queries);
    for (int32_t i = 0; i < n_queries; ++i) {
        const int64_t n = q_ptr[i + 1] - q_ptr[i];
        if (n < 0 || n > INT32_MAX) return set_error(SWMD_EINVAL, "swmd_query_batch: bad q_ptr");
        std::vector<int32_t> qi((size_t)std::max<int64_t>(n, 1));
        std::vector<float> qr((size_t)std::max<int64_t>(n, 1));
        int32_t vr = 0;
        int rc = swmd_select(c->V, (int32_t)n, h_word_ids + q_ptr[i], h_weights + q_ptr[i], qi.data(),
                             qr.data(), &vr);
        if (rc) return set_error(rc, "swmd_query_batch: query %d: %s", i, swmd_last_error());
        if (vr > c->opt.max_vr)
            return set_error(SWMD_EINVAL, "swmd_query_batch: query %d has %d words (max %d)", i, vr,
                             c->opt.max_vr);
        const float lam = h_lambdas[i];
        if (!(lam > 0.f) || std::isinf(lam))
            return set_error(SWMD_EINVAL, "swmd_query_batch: lambda of query %d", i);
        ids.insert(ids.end(), qi.begin(), qi.begin() + vr);
        rs.insert(rs.end(), qr.begin(), qr.begin() + vr);
        vrs[i] = vr;
        off[i + 1] = off[i] + vr;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    cudaStream_t st = c->stream;
    const int kprec = c->opt.k_precision;
    const size_t kb = kprec_bytes(kprec);

    // Each query takes its own path (resolve_path: a function of v_r and the
    // tuning).  Resident queries of one layout run as one batched cost launch and
    // one batched solver launch (on corpora of kAutoResidentDocs documents and more,
    // as one launch pair per query); per-iteration queries run one after another on
    // the corpus's slot.
    std::vector<int> path((size_t)n_queries), vrp((size_t)n_queries, 0);
    // (layout VRP, solver, rows per lane, cost split) -> resident queries: everything
    // a batched launch shares
    std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
    std::vector<int> others;                  // per-iteration queries
    for (int32_t i = 0; i < n_queries; ++i) {
        path[i] = resolve_path(c, vrs[i]);
        if (c->opt.tol > 0.f && path[i] != SWMD_PATH_FUSED)
            return set_error(SWMD_EINVAL, "tol > 0 (convergence mode) needs the fused per-iteration path");
        if (path[i] == SWMD_PATH_RESIDENT) {
            vrp[i] = layout_vrp(c, vrs[i], SWMD_PATH_RESIDENT);
            int s_ = 0, n_ = 0, cs_ = 0;
            resident_settings(c, vrs[i], kprec, &s_, &n_, &cs_);
            groups[std::make_tuple(vrp[i], resident_solver(c, vrs[i], kprec), n_, cs_)].push_back(i);
        } else {
            others.push_back(i);
        }
    }
    auto up = [](size_t n) { return (n + 255) & ~size_t(255); };
    // device workspace: per resident query K^T, KM^T, parameter block, ids, r; then
    // the outputs, the statuses, the staged query arrays and the argument arrays
    std::vector<size_t> kt_off((size_t)n_queries, 0);
    size_t bytes = 0;
    for (int32_t i = 0; i < n_queries; ++i) {
        if (path[i] != SWMD_PATH_RESIDENT) continue;
        kt_off[i] = bytes;
        bytes += 2 * up((size_t)c->Vu * vrp[i] * kb) + up(sizeof(QParams)) + 2 * up(sizeof(float) * vrp[i]);
    }
    const size_t o_out = bytes;
    bytes += up(sizeof(double) * (size_t)n_queries * c->Nl);
    const size_t o_status = bytes;
    bytes += up(sizeof(int) * (size_t)n_queries);
    const size_t o_ids = bytes;
    bytes += up(sizeof(int32_t) * std::max<size_t>(ids.size(), 1));
    const size_t o_r = bytes;
    bytes += up(sizeof(float) * std::max<size_t>(rs.size(), 1));
    const size_t o_prep = bytes;
    bytes += up(sizeof(PrepArgs) * n_queries);
    const size_t o_cost = bytes;
    bytes += up(sizeof(CostArgs) * n_queries);
    const size_t o_res = bytes;
    bytes += up(sizeof(ResidentArgs) * n_queries);
    if (c->batch_ws_bytes < bytes) {
        if (c->batch_ws) {
            cudaStreamSynchronize(st);
            clear_graphs(c);   // the captured batches point into the old workspace
            corpus_free(c, c->batch_ws);
            c->batch_ws = nullptr;
            c->batch_ws_bytes = 0;
        }
        cudaError_t e = corpus_malloc(c, &c->batch_ws, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "swmd_query_batch: workspace");
        c->batch_ws_bytes = bytes;
    }
    char *ws = static_cast<char *>(c->batch_ws);
    int32_t *d_ids = reinterpret_cast<int32_t *>(ws + o_ids);
    float *d_r = reinterpret_cast<float *>(ws + o_r);
    double *d_out = reinterpret_cast<double *>(ws + o_out);
    int *d_status = reinterpret_cast<int *>(ws + o_status);
    std::vector<PrepArgs> prep;
    std::vector<CostArgs> cost((size_t)n_queries);
    std::vector<ResidentArgs> res((size_t)n_queries);
    for (int32_t i = 0; i < n_queries; ++i) {
        if (path[i] != SWMD_PATH_RESIDENT) continue;
        char *b = ws + kt_off[i];
        void *KT = b;
        void *KMT = b + up((size_t)c->Vu * vrp[i] * kb);
        QParams *qp = reinterpret_cast<QParams *>(b + 2 * up((size_t)c->Vu * vrp[i] * kb));
        int *q_ids = reinterpret_cast<int *>(reinterpret_cast<char *>(qp) + up(sizeof(QParams)));
        float *r = reinterpret_cast<float *>(reinterpret_cast<char *>(q_ids) + up(sizeof(float) * vrp[i]));
        PrepArgs p{};
        p.qp = qp;
        p.src_ids = d_ids + off[i];
        p.src_r = d_r + off[i];
        p.q_ids = q_ids;
        p.r = r;
        p.out = d_out + (size_t)i * c->Nl;
        p.status = d_status + i;
        p.lambda = h_lambdas[i];
        p.vr = vrs[i];
        p.vrp_cap = vrp[i];
        p.pad = 0;
        prep.push_back(p);
        CostArgs &ca = cost[i];
        ca = CostArgs{};
        ca.E = c->E;
        ca.d4 = c->d4;
        ca.used = c->used;
        ca.Vu = c->Vu;
        ca.q_ids = q_ids;
        ca.qp = qp;
        ca.V = c->V;
        ca.shift = c->opt.column_shift ? 1 : 0;
        {
            int s_ = 0, n_ = 0, cs_ = 0;
            resident_settings(c, vrs[i], kprec, &s_, &n_, &cs_);
            ca.split = cs_;
        }
        ca.KT = KT;
        ca.KMT = KMT;
        IterArgs ia{};
        ia.doc_ptr = c->doc_ptr;
        ia.nz = c->nz;
        ia.KT = KT;
        ia.KMT = KMT;
        ia.r = r;
        ia.doc_orig = c->doc_orig;
        ia.qp = qp;
        ia.doc0 = 0;
        ia.N = c->Nl;
        ia.Vu = c->Vu;
        ia.first = 1;
        res[i] = ResidentArgs{ia, max_iter};
    }
    // group-contiguous copies of the argument arrays (grid row y of a group's
    // launch reads element y of its slice)
    std::vector<CostArgs> cost_g;
    std::vector<ResidentArgs> res_g;
    std::vector<std::pair<std::tuple<int, int, int, int>, size_t>> gstart;   // (group, first index in the grouped arrays)
    for (auto &g : groups) {
        gstart.emplace_back(g.first, cost_g.size());
        for (int i : g.second) {
            cost_g.push_back(cost[i]);
            res_g.push_back(res[i]);
        }
    }
    if (!ids.empty())
        SWMD_CK(cudaMemcpyAsync(d_ids, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice, st));
    if (!rs.empty())
        SWMD_CK(cudaMemcpyAsync(d_r, rs.data(), sizeof(float) * rs.size(), cudaMemcpyHostToDevice, st));
    if (!prep.empty()) {
        SWMD_CK(cudaMemcpyAsync(ws + o_prep, prep.data(), sizeof(PrepArgs) * prep.size(), cudaMemcpyHostToDevice, st));
        SWMD_CK(cudaMemcpyAsync(ws + o_cost, cost_g.data(), sizeof(CostArgs) * cost_g.size(), cudaMemcpyHostToDevice, st));
        SWMD_CK(cudaMemcpyAsync(ws + o_res, res_g.data(), sizeof(ResidentArgs) * res_g.size(), cudaMemcpyHostToDevice, st));
    }
    if (!others.empty() && !c->main.external && c->main.kprec != kprec) {
        // the per-iteration queries use the corpus's slot: size it before any capture
        clear_graphs(c);
        int rc = alloc_slot(c, c->main, c->opt.max_vr, kprec, false);
        if (rc) return rc;
    }
    // The device work of the batch: statuses cleared, one parameter launch, per
    // layout group one cost and one solver launch, then the per-iteration queries.
    // Everything it reads from the host side is in the workspace already, except
    // the per-iteration queries' lambda and the iteration count, which are part of
    // the key of the captured graph below.
    auto body = [&]() -> int {
        SWMD_CK(cudaMemsetAsync(d_status, 0, sizeof(int) * (size_t)n_queries, st));
        if (!prep.empty()) {
            SWMD_CK(launch_prep_batch(reinterpret_cast<const PrepArgs *>(ws + o_prep), (int)prep.size(), c->V, st));
            for (size_t gi = 0; gi < gstart.size(); ++gi) {
                const int v = std::get<0>(gstart[gi].first);
                const size_t g0 = gstart[gi].second;
                const std::vector<int> &members = groups[gstart[gi].first];
                const int ng = (int)members.size();
                const Mapping m = walk_mapping(c, v, SWMD_PATH_RESIDENT);
                // From kAutoResidentDocs documents up one query's launches fill the GPU
                // many times over, and queries run side by side only compete for L2
                // (each gathers its own K^T); there the group's queries run one after
                // another (still one graph, no host round trips).  Smaller corpora run
                // the group as one batched cost and one batched solver launch.
                // The column-split solver takes a tile group of queries per cost and
                // solver launch pair: the group's K^T and KM^T, just written, are still
                // in L2 when its solver runs.
                const int step = std::get<1>(gstart[gi].first) == kSolverCols ? cols_queries_per_group(c, v, kprec)
                                 : c->Nl >= kAutoResidentDocs                  ? 1
                                                                               : ng;
                for (int j0 = 0; j0 < ng; j0 += step) {
                    const int nj = std::min(step, ng - j0);
                    SWMD_CK(launch_cost_batch(cost_g[g0 + j0], v, kprec, nj,
                                              reinterpret_cast<const CostArgs *>(ws + o_cost) + g0 + j0, st));
                    int rc = run_resident_batch(c, res_g[g0 + j0], m, kprec, vrs[members[j0]], nj,
                                                reinterpret_cast<const ResidentArgs *>(ws + o_res) + g0 + j0, st);
                    if (rc) return rc;
                }
            }
        }
        for (int i : others) {
            int rc = enqueue_query(c, c->main, d_ids + off[i], d_r + off[i], vrs[i], h_lambdas[i], max_iter,
                                   d_out + (size_t)i * c->Nl, d_status + i, st, false);
            if (rc) return rc;
        }
        return SWMD_OK;
    };
    if (!c->opt.use_graph) {
        int rc = body();
        if (rc) return rc;
    } else {
        // one CUDA graph per batch shape: the queries' paths, layouts and sizes, the
        // per-iteration queries' lambdas, the iteration count and the workspace
        std::vector<int64_t> key{n_queries, max_iter, kprec, c->opt.column_shift,
                                 (int64_t)(uintptr_t)c->batch_ws};
        for (int32_t i = 0; i < n_queries; ++i) {
            key.push_back(path[i]);
            key.push_back(vrs[i]);
            if (path[i] != SWMD_PATH_RESIDENT) {
                uint32_t lb;
                std::memcpy(&lb, &h_lambdas[i], sizeof lb);
                key.push_back(lb);
            }
        }
        auto it = c->batch_graphs.find(key);
        if (it == c->batch_graphs.end() && !c->batch_seen.count(key)) {
            // a shape seen for the first time runs eagerly: capturing and instantiating
            // a graph pays only for shapes that come back
            if (c->batch_seen.size() >= kMaxBatchShapes) c->batch_seen.clear();
            c->batch_seen.insert(key);
            int rc = body();
            if (rc) return rc;
        } else if (it == c->batch_graphs.end()) {
            if (c->batch_graphs.size() >= kMaxBatchShapes) {
                for (auto &kv : c->batch_graphs) cudaGraphExecDestroy(kv.second);
                c->batch_graphs.clear();
            }
            c->batch_seen.erase(key);
            cudaGraph_t g = nullptr;
            SWMD_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
            int rc = body();
            cudaError_t e = cudaStreamEndCapture(st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            SWMD_CK(e);
            cudaGraphExec_t ge = nullptr;
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            SWMD_CK(e);
            it = c->batch_graphs.emplace(key, ge).first;
            SWMD_CK(cudaGraphLaunch(it->second, st));
        } else {
            SWMD_CK(cudaGraphLaunch(it->second, st));
        }
    }
    std::vector<int> h_status((size_t)n_queries, 0);
    SWMD_CK(cudaMemcpyAsync(h_out, d_out, sizeof(double) * (size_t)n_queries * c->Nl, cudaMemcpyDeviceToHost, st));
    SWMD_CK(cudaMemcpyAsync(h_status.data(), d_status, sizeof(int) * (size_t)n_queries, cudaMemcpyDeviceToHost, st));
    SWMD_CK(cudaStreamSynchronize(st));
    int all = 0;
    for (int x : h_status) all |= x;
    return status_to_code(all);
}

void swmd_default_serve_config(swmd_serve_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->max_batch = 32;
    cfg->memory_budget = (int64_t)4 << 30;
    cfg->max_wait_us = 200;
    cfg->queue_capacity = 4096;
}

int swmd_serve_start(swmd_corpus *c, const swmd_serve_config *cfg_in, swmd_server **out) {
    if (!c || !out) return set_error(SWMD_EINVAL, "swmd_serve_start: NULL argument");
    *out = nullptr;
    swmd_serve_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else swmd_default_serve_config(&cfg);
    if (cfg.max_batch < 1 || cfg.max_batch > 1024 || cfg.memory_budget <= 0 || cfg.queue_capacity < 1)
        return set_error(SWMD_EINVAL, "swmd_serve_start: bad configuration");
    // the largest single query: every path a query may take, at max_vr words
    size_t largest = 0;
    for (int p : {SWMD_PATH_FUSED, SWMD_PATH_PLAIN, SWMD_PATH_RESIDENT}) {
        if (c->opt.path != SWMD_PATH_AUTO && p != c->opt.path) continue;
        if (c->opt.path == SWMD_PATH_AUTO && p == SWMD_PATH_PLAIN) continue;
        const Mapping mx = choose_mapping(c, c->opt.max_vr, p);
        largest = std::max(largest, query_bytes(c, std::max(mx.vrp, max_vrp_of(c->opt.max_vr)), p));
    }
    if ((size_t)cfg.memory_budget < largest)
        return set_error(SWMD_ENOMEM, "swmd_serve_start: memory_budget %lld below one query of %d words (%zu bytes)",
                         (long long)cfg.memory_budget, c->opt.max_vr, largest);
    DeviceGuard guard(c->device);
    auto *S = new swmd_server();
    S->c = c;
    S->cfg = cfg;
    auto bail = [&](int code) {
        for (auto &sl : S->slots) {
            sl.ws.KT = sl.ws.KMT = nullptr;
            sl.ws.u = sl.ws.v = nullptr;
            free_slot(S->c, sl.ws);
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
            cudaFreeHost(sl.h_q); cudaFreeHost(sl.h_r); cudaFreeHost(sl.h_status);
        }
        for (auto &L : S->lanes) {
            if (L.stream) cudaStreamDestroy(L.stream);
            for (int b = 0; b < kLaneDepth; ++b) {
                corpus_free(S->c, L.d_args[b]);
                cudaFreeHost(L.h_args[b]);
            }
        }
        if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
        corpus_free(S->c, S->arena_mem);
        delete S;
        return code;
    };
    cudaError_t e = corpus_malloc(c, reinterpret_cast<void **>(&S->arena_mem), (size_t)cfg.memory_budget);
    if (e != cudaSuccess) return bail(cuda_fail(e, "swmd_serve_start: arena"));
    S->arena.init(S->arena_mem, (size_t)cfg.memory_budget);
    if ((e = cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(e, "swmd_serve_start: copy stream"));
    // result buffers for the first max_batch queries, their pages touched now (a copy
    // into fresh memory would first fault them in)
    S->spare.resize((size_t)cfg.max_batch, std::vector<double>((size_t)std::max(c->Nl, 1)));
    S->slots.resize((size_t)cfg.max_batch);
    const int vrp = max_vrp_of(c->opt.max_vr);
    for (auto &sl : S->slots) {
        Slot &w = sl.ws;
        e = corpus_malloc(c, reinterpret_cast<void **>(&w.q_ids), sizeof(int) * vrp);
        if (e == cudaSuccess) e = corpus_malloc(c, reinterpret_cast<void **>(&w.r), sizeof(float) * vrp);
        if (e == cudaSuccess) e = corpus_malloc(c, reinterpret_cast<void **>(&w.qp), sizeof(QParams));
        if (e == cudaSuccess) e = corpus_malloc(c, reinterpret_cast<void **>(&w.out), sizeof(double) * std::max(c->Nl, 1));
        if (e == cudaSuccess) e = corpus_malloc(c, reinterpret_cast<void **>(&w.status), sizeof(int));
        if (e == cudaSuccess) e = corpus_malloc(c, reinterpret_cast<void **>(&w.conv), sizeof(unsigned) * (1 + kMaxConvIters));
        if (e == cudaSuccess) e = cudaMemset(w.conv, 0, sizeof(unsigned) * (1 + kMaxConvIters));
        if (e == cudaSuccess) e = corpus_malloc(c, reinterpret_cast<void **>(&w.q_in), sizeof(int) * vrp);
        if (e == cudaSuccess) e = corpus_malloc(c, reinterpret_cast<void **>(&w.r_in), sizeof(float) * vrp);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_q, sizeof(int32_t) * vrp);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_r, sizeof(float) * vrp);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_status, sizeof(int));
        if (e != cudaSuccess) return bail(cuda_fail(e, "swmd_serve_start: slot"));
        w.vrp_cap = vrp;
        w.kprec = c->opt.k_precision;
        w.external = true;
    }
    {
        std::lock_guard<std::mutex> cl(c->mu);
        ++c->servers;
    }
    // One batch lane: a group of queries of one layout fills the GPU by itself, and
    // two groups side by side would only slow each other down.
    S->lanes.resize(1);
    for (auto &L : S->lanes) {
        L.args_bytes = lane_args_bytes(cfg.max_batch);
        e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
        for (int b = 0; b < kLaneDepth && e == cudaSuccess; ++b) {
            e = corpus_malloc(c, reinterpret_cast<void **>(&L.d_args[b]), L.args_bytes);
            if (e == cudaSuccess) e = cudaMallocHost(&L.h_args[b], L.args_bytes);
        }
        if (e != cudaSuccess) return bail(cuda_fail(e, "swmd_serve_start: batch lane"));
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return SWMD_OK;
}

int swmd_serve_submit(swmd_server *S, const int32_t *h_ids, const float *h_weights, int32_t n_words,
                      float lambda, int32_t max_iter, uint64_t *ticket) {
    if (!S || !ticket) return set_error(SWMD_EINVAL, "swmd_serve_submit: NULL argument");
    auto R = std::make_shared<Request>();
    R->ids.resize((size_t)std::max(n_words, 1));
    R->r.resize((size_t)std::max(n_words, 1));
    int rc = swmd_select(S->c->V, n_words, h_ids, h_weights, R->ids.data(), R->r.data(), &R->vr);
    if (rc) return rc;
    if (R->vr > S->c->opt.max_vr)
        return set_error(SWMD_EINVAL, "swmd_serve_submit: %d words (max %d)", R->vr, S->c->opt.max_vr);
    if (!(lambda > 0.f) || std::isinf(lambda) || max_iter < 0)
        return set_error(SWMD_EINVAL, "swmd_serve_submit: lambda must be finite > 0, max_iter >= 0");
    R->lambda = lambda;
    R->t = max_iter;
    std::lock_guard<std::mutex> lk(S->m);
    if (S->stopping) return set_error(SWMD_ESTOPPED, "swmd_serve_submit: server stopped");
    if ((int)S->pending.size() >= S->cfg.queue_capacity) {
        S->rejected++;
        return set_error(SWMD_ENOMEM, "swmd_serve_submit: queue full (%d)", S->cfg.queue_capacity);
    }
    R->ticket = S->next_ticket++;
    R->t_submit = now_s();
    if (S->t_first < 0) S->t_first = R->t_submit;
    S->table[R->ticket] = R;
    S->pending.push_back(R);
    *ticket = R->ticket;
    S->cv_work.notify_one();
    return SWMD_OK;
}

int swmd_serve_wait(swmd_server *S, uint64_t ticket, double *h_out_dist, int32_t timeout_ms) {
    if (!S) return set_error(SWMD_EINVAL, "swmd_serve_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->m);
    auto it = S->table.find(ticket);
    if (it == S->table.end()) return set_error(SWMD_EINVAL, "swmd_serve_wait: unknown ticket %llu", (unsigned long long)ticket);
    auto R = it->second;
    auto ready = [&] { return R->state == 2; };
    ++S->waiters;
    bool ok = true;
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    if (!ok) {
        --S->waiters;
        S->cv_done.notify_all();   // a stopping server waits for the last waiter to leave
        return set_error(SWMD_ETIMEDOUT, "swmd_serve_wait: ticket %llu not ready after %d ms",
                         (unsigned long long)ticket, timeout_ms);
    }
    auto again = S->table.find(ticket);   // another waiter of the same ticket may have taken it
    if (again == S->table.end()) {
        --S->waiters;
        S->cv_done.notify_all();
        return set_error(SWMD_EINVAL, "swmd_serve_wait: ticket %llu was collected by another waiter",
                         (unsigned long long)ticket);
    }
    S->table.erase(again);
    std::vector<double> res = std::move(R->result);
    const int code = R->code;
    const std::string err = R->err;
    // the copy into the caller's buffer runs outside the lock (the server stays alive
    // while this thread counts as a waiter); the buffer then goes back to the pool
    lk.unlock();
    if (!res.empty() && h_out_dist) std::memcpy(h_out_dist, res.data(), sizeof(double) * res.size());
    lk.lock();
    if (!res.empty() && S->spare.size() < 2 * S->slots.size()) S->spare.push_back(std::move(res));
    --S->waiters;
    S->cv_done.notify_all();
    lk.unlock();
    if (code) return set_error(code, "%s", err.c_str());
    return SWMD_OK;
}

int swmd_serve_stats(swmd_server *S, swmd_serve_stats_t *out) {
    if (!S || !out) return set_error(SWMD_EINVAL, "swmd_serve_stats: NULL argument");
    std::lock_guard<std::mutex> lk(S->m);
    std::memset(out, 0, sizeof *out);
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->batches = S->batches;
    out->mean_batch = S->batches ? (double)S->admitted / S->batches : 0.0;
    if (S->completed > 0 && S->t_last > S->t_first) out->qps = S->completed / (S->t_last - S->t_first);
    if (!S->lat_ms.empty()) {
        std::vector<double> l = S->lat_ms;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {
            const double x = p * (double)(l.size() - 1);
            const size_t i = (size_t)x;
            const double f = x - (double)i;
            return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
    }
    return SWMD_OK;
}

int swmd_serve_stop(swmd_server *S) {
    if (!S) return SWMD_OK;
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stopping = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    {
        // every pending request has failed with SWMD_ESTOPPED: let the threads blocked
        // in swmd_serve_wait collect that before the server goes away
        std::unique_lock<std::mutex> lk(S->m);
        S->cv_done.wait(lk, [&] { return S->waiters == 0; });
    }
    {
        std::lock_guard<std::mutex> cl(S->c->mu);
        --S->c->servers;
    }
    DeviceGuard guard(S->c->device);
    for (auto &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        sl.ws.KT = sl.ws.KMT = nullptr;
        sl.ws.u = sl.ws.v = nullptr;
        free_slot(S->c, sl.ws);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        cudaFreeHost(sl.h_q); cudaFreeHost(sl.h_r); cudaFreeHost(sl.h_status);
    }
    for (auto &L : S->lanes) {
        if (L.stream) {
            cudaStreamSynchronize(L.stream);
            cudaStreamDestroy(L.stream);
        }
        for (int b = 0; b < kLaneDepth; ++b) {
            corpus_free(S->c, L.d_args[b]);
            cudaFreeHost(L.h_args[b]);
        }
    }
    if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
    corpus_free(S->c, S->arena_mem);
    delete S;
    return SWMD_OK;
}

}  // extern "C"
