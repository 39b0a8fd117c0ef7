// Internal: the corpus object behind swmd_corpus* and the query engine shared by
// the single-query, batch and serving entry points.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <set>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "swmd.h"

namespace swmd {

int set_error(int code, const char *fmt, ...);

// Makes `dev` the current device for a scope and restores the caller's device after.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int cuda_fail(cudaError_t e, const char *what);

#define SWMD_CK(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return ::swmd::cuda_fail(e_, #call); \
    } while (0)

// The device allocator of a corpus (swmd_set_allocator; NULL functions: cudaMalloc).
struct Allocator {
    swmd_alloc_fn alloc = nullptr;
    swmd_free_fn release = nullptr;
    void *user = nullptr;
};

// Device-side parameter block of one query slot.  Kernels read it through a
// pointer, so a captured graph is reused for every query of the same shape.
struct SlotParams {
    QParams qp;
};

// Per-query device workspace: K^T, KM^T, u and the small query arrays.
struct Slot {
    int vrp_cap = 0;      // VRP the buffers were sized for
    int kprec = -1;
    void *KT = nullptr;
    void *KMT = nullptr;
    float *u = nullptr;
    float *v = nullptr;   // plain path only: SDDMM output at the sliced positions
    int64_t v_elems = 0;  // capacity of v (checked against the corpus's slice_total)
    int *q_ids = nullptr; // [vrp_cap]
    float *r = nullptr;   // [vrp_cap], zero padded
    QParams *qp = nullptr;
    double *out = nullptr;   // [Nl] distances (caller order)
    int *status = nullptr;
    unsigned *conv = nullptr;   // [1 + kMaxConvIters]: convergence mode record
    int *q_in = nullptr;     // host-API staging of the query
    float *r_in = nullptr;
    int64_t bytes = 0;
    bool external = false;   // buffers managed by a server (never reallocated here)
    bool carved_io = false;  // status follows out, r_in follows q_in (vrp_cap ints) in one allocation
    int cur_vrp = 0;         // padding of the K^T layout the last query / cost step wrote
    int cur_vr = 0;          // ... and the query size it was written for
    int last_t = 0;          // max_iter and path of the last query enqueued on the slot
    int last_path = -1;
};

// Key of a captured launch sequence: everything baked into the launches.
// vrp, q, p, t, path, kprec, shift, resident solver, rows per lane, cost split, slot
using GraphKey = std::tuple<int, int, int, int, int, int, int, int, int, int, const void *>;

struct Segment {
    long d0, d1;   // documents [d0, d1) in internal order
};

}  // namespace swmd

struct swmd_corpus {
    int V = 0, N = 0, d = 0, d4 = 0, Vu = 0;
    int64_t nnz = 0;
    int doc_begin = 0, doc_end = 0;
    int Nl = 0;          // documents held = doc_end - doc_begin
    int device = 0;
    int sms = 0;
    swmd_options opt{};
    cudaStream_t stream = nullptr;

    float *E = nullptr;
    int *used = nullptr;
    int *doc_ptr = nullptr;
    int2 *nz = nullptr;
    // the same nonzeros in slices of 32 documents (per-iteration walks)
    int *slice_ptr = nullptr;
    int2 *slice_nz = nullptr;
    int n_slices = 0;
    int64_t slice_total = 0;       // entries including the slices' padding
    int *doc_orig = nullptr;
    std::vector<int> len_sorted;   // document lengths in internal order (host)
    double mean_len = 0;

    // tile sets of the resident solver, one per nonzero budget (kTileBudgets)
    int *tiles_dev = nullptr;
    std::vector<int> tile_off;     // offset of each set in tiles_dev
    std::vector<int> tile_count;   // tiles in each set
    int tile_threads = 0, tile_npl = 0;   // geometry the sets were built for
    // warp tasks of the register-resident solver, one list per rows-per-lane value
    int4 *tasks_dev = nullptr;
    int task_off[9] = {0};         // indexed by rows per lane (1..8)
    int task_count[9] = {0};
    // warp tasks of the column-split register solver, one list per layout (VRP 16,
    // 32, 64, 128) over the documents [col_first, Nl) it holds: documents are in
    // decreasing length, so those too long for the layout's buckets (cols_max_len)
    // are the first col_first; col_long: the list has buckets above 32 rows
    int4 *col_tasks_dev = nullptr;
    int col_off[swmd::kColLayouts] = {0};
    int col_count[swmd::kColLayouts] = {0};
    int col_first[swmd::kColLayouts] = {0};
    int col_long[swmd::kColLayouts] = {0};
    // register-solver tasks (per rows-per-lane list) that cover exactly the documents
    // [0, col_first) of the layouts of 16 and 32 columns: the register solver takes
    // them when a column-split query runs on a corpus with longer documents
    int task_prefix[9][2] = {{0}};

    swmd::Slot main;               // workspace of the single-query path
    void *batch_ws = nullptr;      // workspace of swmd_query_batch (grown on demand)
    size_t batch_ws_bytes = 0;
    void *pair_ws = nullptr;       // swmd_wmd_pairs: packed pairs, results, status (grown on demand)
    size_t pair_ws_bytes = 0;
    float *pair_kws = nullptr;     // 1-to-1 pairs: per-block K and K.*M regions too large
    size_t pair_kws_bytes = 0;     // for shared memory (grown on demand)
    int64_t base_bytes = 0;
    void *h_io = nullptr;          // pinned staging of swmd_query: [ids | weights] then the status word
    size_t h_io_in_bytes = 0;

    std::map<swmd::GraphKey, cudaGraphExec_t> graphs;
    std::map<std::vector<int64_t>, cudaGraphExec_t> batch_graphs;   // swmd_query_batch shapes
    std::set<std::vector<int64_t>> batch_seen;   // shapes run once, eagerly (captured when seen again)
    std::map<std::tuple<int, int, int>, swmd::Mapping> tuned;  // (vr bucket, path, kprec)
    // autotuned resident-path settings per (v_r, K precision): solver, rows per lane, cost split
    std::map<std::pair<int, int>, std::tuple<int, int, int>> tuned_resident;
    // autotuned path (RESIDENT or FUSED) per (v_r, K precision), used by SWMD_PATH_AUTO
    std::map<std::pair<int, int>, int> tuned_path;
    // autotuned queries per tile of the multi-query column-split walk per (VRP, K precision)
    std::map<std::pair<int, int>, int> tuned_qpt;
    size_t l2_bytes = 0;           // the device's L2 cache
    std::mutex mu;                 // serialises use of `main` and the graph cache
    swmd::Allocator allocator;     // the allocator in force when the corpus was created
    std::mutex alloc_mu;
    std::unordered_map<void *, size_t> alloc_sizes;   // live blocks of a set allocator
    int servers = 0;               // servers attached (under mu): tuning and option changes wait
};

namespace swmd {

// The K^T / u row length a workspace needs for queries of up to max_vr words.
int max_vrp_of(int max_vr);
int alloc_slot(swmd_corpus *c, Slot &s, int max_vr, int kprec, bool with_v);
void free_slot(swmd_corpus *c, Slot &s);
// Device memory of the corpus's allocator (cudaMalloc when none was set);
// corpus_free(c, NULL) does nothing.
cudaError_t corpus_malloc(swmd_corpus *c, void **p, size_t bytes);
void corpus_free(swmd_corpus *c, void *p);
Mapping choose_mapping(swmd_corpus *c, int vr, int path);
int layout_vrp(swmd_corpus *c, int vr, int path);
// The tight resident layout (v_r padded to the solver's multiple of 4, 8 or 16)
// of every resident solver but the column-split one.
int tight_vrp(int vr);
// The concrete path a query of vr words takes (resolves SWMD_PATH_AUTO).
int resolve_path(swmd_corpus *c, int vr);
// Corpora with fewer documents than this take the resident path under SWMD_PATH_AUTO
// unless tuned otherwise.
constexpr int kAutoResidentDocs = 20000;
constexpr int kAutoResidentVr = 24;
Mapping walk_mapping(swmd_corpus *c, int vrp, int path);
// Enqueues a whole query whose ids / r are already in device memory (d_ids,
// d_r), writing the distances to d_out and the status to d_status.
// path >= 0: the path already resolved for this query (a server resolves it once,
// at admission); -1: resolve_path.
int enqueue_query(swmd_corpus *c, Slot &s, const int *d_ids, const float *d_r, int vr,
                  float lambda, int t, double *d_out, int *d_status, cudaStream_t st,
                  bool allow_graph, int path = -1);
int status_to_code(int st);
// Destroys every captured graph of the corpus (single queries and batches).
void clear_graphs(swmd_corpus *c);
// Launches the all-iterations solver of resident_solver (the register walk that
// re-gathers rows from L2 when no other solver takes the layout).
// vr: the query's words (it selects the solver, see resident_solver).
int run_resident(swmd_corpus *c, const ResidentArgs &ra, Mapping m, int kprec, int vr, cudaStream_t st);
// The same for nq queries of one layout and one solver in one launch (d_batch:
// device array of their arguments; `shape` is any one of them, vr any one's size).
int run_resident_batch(swmd_corpus *c, const ResidentArgs &shape, Mapping m, int kprec, int vr, int nq,
                       const ResidentArgs *d_batch, cudaStream_t st);
// Resident solvers (swmd_options.solver).
constexpr int kSolverAuto = 0, kSolverRegs = 1, kSolverTiled = 2, kSolverL2 = 3, kSolverCols = 4;
// The solver a resident query of vr words runs: swmd_options.solver, else the
// autotuned one, else the column-split register solver when its layout holds every
// document in buckets of up to 32 rows, else kSolverAuto (register solver for
// VRP <= 32, else the shared-memory tiled one).  Never kSolverCols for a layout it
// does not take (cols_takes).
int resident_solver(swmd_corpus *c, int vr, int kprec);
// Whether the column-split solver takes a query of vr words on this corpus: its
// layout (cols_vrp) holds every document, or (16 and 32 columns) all but the
// longest, which the register solver then runs in a launch before it.
// whole: set to whether it holds every document.
bool cols_takes(swmd_corpus *c, int vr, bool *whole = nullptr);
// Queries per (query group, document task) tile of the multi-query column-split
// walk for a layout: swmd_options.queries_per_tile, else the autotuned value, else
// as many (1..8) as keep their K^T and KM^T within a quarter of L2.
int cols_queries_per_group(swmd_corpus *c, int vrp, int kprec);
constexpr int kTileBudgets[] = {64, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048};
constexpr int kNumTileBudgets = 10;
// (Re)builds the resident solver's tile sets for the corpus's current
// tile_threads / nnz_per_lane (allocates: only at creation or on an option change).
int build_tiles(swmd_corpus *c);
// Builds the register-resident solvers' warp task lists (at corpus creation).
int build_tasks(swmd_corpus *c);
// 1-to-1 pairs (pairs.cu): enqueues the distances of n_pairs selected, normalised
// (query, target) pairs held in device memory; max_q / max_x bound every pair's sizes.
struct PairJob {
    int n_pairs;
    const int64_t *q_ptr;
    const int *q_ids;
    const float *r;
    const int64_t *x_ptr;
    const int *x_ids;
    const float *cx;
    int max_q, max_x;
    float lambda;
    int t;
    float tol;
    double *out;
    int *iters;     // may be NULL
    int *status;
};
constexpr int kPairMaxWords = 4096;
// status bit of the pair kernel (beside the ST_* bits of common.cuh): a pair side
// outside its declared size bound
constexpr int ST_BAD_SIZE = 16;
int enqueue_pairs(swmd_corpus *c, const PairJob &job, cudaStream_t st);
// Effective resident settings for a query of vr words: explicit options, else
// autotuned, else defaults (0).
void resident_settings(swmd_corpus *c, int vr, int kprec, int *solver, int *npl_want, int *split);

}  // namespace swmd
