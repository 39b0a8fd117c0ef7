/*
 * swmd.h -- C ABI of the GB300 Sinkhorn Word Mover's Distance library (libswmd).
 *
 * The library computes the entropic Sinkhorn WMD of one query document against
 * every document of a corpus, as the paper "A New Parallel Algorithm for Sinkhorn
 * Word-Movers Distance Using Fused SDDMM-SpMM" (arXiv 2107.06433) states the
 * problem: sinkhorn_wmd(r, c, vecs, lambda, max_iter) -> WMD[N] (Section III-B1),
 * computed with Algorithm 1 (Section III-A) in its sparse, fused SDDMM-SpMM
 * form (Sections III-B4 and III-C).
 *
 * Conventions for every call:
 *   - Return value: SWMD_OK (0) or one of the SWMD_E* codes below.  Nothing
 *     throws across the ABI.  swmd_last_error() gives a message for the last
 *     failing call on the calling thread.
 *   - Pointers named h_* or documented as host memory are host pointers owned by
 *     the caller; the library copies what it needs during the call and does not
 *     keep them.  Pointers named d_* are device pointers on the corpus's GPU,
 *     owned by the caller, that must stay valid until the stream work of the
 *     call has completed.
 *   - A corpus (and a server) owns every device allocation it makes (through
 *     swmd_set_allocator's functions when set, else cudaMalloc).  Calls on
 *     one corpus are not thread-safe unless stated; use one server or one
 *     corpus per thread.
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL means the
 *     corpus's own stream.
 */
#ifndef SWMD_H
#define SWMD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SWMD_API __attribute__((visibility("default")))
#else
#define SWMD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define SWMD_OK 0
#define SWMD_EINVAL 1     /* an argument or input violates the documented contract */
#define SWMD_ENOMEM 2     /* a host or device allocation failed, or admission refused */
#define SWMD_ECUDA 3      /* a CUDA runtime call failed; the message names it */
#define SWMD_ETIMEDOUT 4  /* a wait ran out of time */
#define SWMD_ENUMERIC 5   /* a NaN, an infinity or a vanished denominator was produced */
#define SWMD_ESTOPPED 6   /* the server has been stopped */

/* K and K.*M storage precision (accumulation is always FP32). */
#define SWMD_K_FP32 0
#define SWMD_K_BF16 1
#define SWMD_K_FP16 2

/* How the t Sinkhorn iterations run.
 *   FUSED:    one fused SDDMM-SpMM launch per iteration (Section III-C), u
 *             kept in HBM between iterations.
 *   PLAIN:    separate SDDMM and SpMM launches per iteration, the unfused
 *             formulation of Section III-B4 (writes v, then reads it back).
 *   RESIDENT: all t iterations and the final step of a document in one launch,
 *             u held on chip; legal because the documents (columns of c) are
 *             independent problems in Algorithm 1.
 *   AUTO:     RESIDENT or FUSED for each query: the choice swmd_autotune measured
 *             for its v_r, else RESIDENT when the resident solver is the
 *             column-split one and it holds every document (swmd_options.solver 4,
 *             the default on corpora of documents up to 32 words), else RESIDENT
 *             for corpora under 20,000
 *             documents or v_r up to 24 and FUSED otherwise (on large corpora the
 *             per-iteration walk beats the other resident solvers for wide queries).  The choice depends only on v_r and
 *             the tuning, so a query's result is the same alone, batched or served. */
#define SWMD_PATH_FUSED 0
#define SWMD_PATH_PLAIN 1
#define SWMD_PATH_RESIDENT 2
#define SWMD_PATH_AUTO 3

typedef struct swmd_corpus swmd_corpus;
typedef struct swmd_server swmd_server;

typedef struct swmd_options {
    int32_t k_precision;   /* SWMD_K_*; default SWMD_K_FP32 */
    int32_t path;          /* SWMD_PATH_*; default SWMD_PATH_AUTO */
    int32_t use_graph;     /* 1: replay the query's launches as a captured CUDA graph (default 1) */
    int32_t column_shift;  /* 1: K'[k,w] = exp(-lambda (M[k,w] - min_k M[k,w])), an exact
                              rescaling of the columns of K (default 1) */
    int32_t max_vr;        /* largest query (distinct words) the workspace must hold;
                              default 128, at most 128 */
    int32_t device;        /* CUDA device ordinal; -1 = the current device (default) */
    int32_t doc_begin;     /* documents [doc_begin, doc_end) of the CSR columns are loaded;
                              -1/-1 = all.  One replica per GPU loads its own range. */
    int32_t doc_end;
    int32_t team_lanes;    /* per-iteration paths: 0 = the sliced walk (default: VRP / 8
                              lanes per document in FP32, VRP / 16 in BF16/FP16); else
                              the general document walk with this many lanes per
                              document (1..32, power of 2), used with lanes_per_nz */
    int32_t lanes_per_nz;  /* per-iteration paths, general walk: lanes sharing one
                              nonzero's dot (power of 2 dividing team_lanes) */
    int32_t tile_threads;  /* resident path: threads per block (64, 128 or 256; 0 = 128) */
    int32_t nnz_per_lane;  /* resident path: nonzeros (rows of K^T) per lane and pass; a
                              document of n nonzeros gets about n / nnz_per_lane lanes
                              (0 = chosen from the query size) */
    int32_t tile_nnz;      /* resident path: nonzeros staged per block (0 = as many as fit
                              in about 100 KB of shared memory) */
    int32_t cost_split;    /* cost kernel: 0 = automatic (the tiled product-form kernel
                              for layouts of 16, 32, 64 and 128 columns, else the row
                              kernel with 2 threads per word, 1 from 65,536 used words
                              up); 1, 2 or 4 = the row kernel with that many threads
                              sharing one word's embedding row */
    int32_t solver;        /* resident path kernel: 0 = automatic (4 when every document has
                              at most 32 words, else 1 for v_r <= 32 and 2 above),
                              1 = K^T rows in registers, whole rows per lane (v_r <= 32),
                              2 = rows staged in shared memory, 3 = rows re-gathered from
                              L2 each iteration, 4 = K^T rows in registers split by columns
                              (eight per lane) over row groups of VRP / 8 lanes, one to
                              eight groups per document; v_r padded to a power of two from
                              16 to 128.  It holds documents of up to 96 words at 16 and 32
                              columns, 32 at 64 and 128; at 16 and 32 columns longer
                              documents run on solver 1 in a launch before it, at 64 and 128
                              a corpus with longer documents makes 4 act as 0 */
    float tol;             /* 0 (default): exactly max_iter x-updates, as the paper's
                              experiments run.  > 0: Algorithm 1's "while x changes": the
                              fused per-iteration path stops after the x-update in which
                              max over documents and query words of |u (K v) - r| (the row
                              marginal of P against r) falls below tol; max_iter (at most
                              4096) caps it.  SWMD_PATH_AUTO then takes the fused path;
                              the resident and plain paths refuse tol > 0 (SWMD_EINVAL). */
    int32_t queries_per_tile; /* swmd_query_batch and the server, column-split solver:
                              queries of one layout that share a (query group, document
                              task) tile of the one-launch multi-query walk; 0 = the
                              swmd_autotune_batch choice, else as many (1..8) as keep
                              their K^T and KM^T within a quarter of the L2 cache */
} swmd_options;

/* ------------------------------------------------------------------ device memory */
/* Device memory of corpora and servers.  By default the library takes it with
 * cudaMalloc and returns it with cudaFree.  swmd_set_allocator makes every corpus
 * created afterwards -- and that corpus's servers, batch and 1-to-1 pair workspaces
 * -- take it from alloc(bytes, device, stream, user) and return it with
 * release(ptr, bytes, device, stream, user) instead (the Python binding passes
 * PyTorch's caching allocator).  alloc returns NULL when it cannot serve the
 * request (the call then fails with SWMD_ENOMEM) and must return 256-byte aligned
 * device memory of `device`; `stream` (a cudaStream_t) is the corpus's stream, on
 * which the memory is used.  A corpus keeps the allocator it was created with until
 * it is destroyed.  Both NULL restores cudaMalloc / cudaFree; one NULL is
 * SWMD_EINVAL.  The library calls them from the calling thread of the entry point
 * that allocates or frees (swmd_create_corpus, swmd_query_batch, swmd_wmd_pairs*,
 * swmd_serve_start / _stop, swmd_destroy_corpus, and option changes that grow the
 * workspace), never from a server's worker thread.  The paper has no counterpart. */
typedef void *(*swmd_alloc_fn)(size_t bytes, int32_t device, void *stream, void *user);
typedef void (*swmd_free_fn)(void *ptr, size_t bytes, int32_t device, void *stream, void *user);
SWMD_API int swmd_set_allocator(swmd_alloc_fn alloc, swmd_free_fn release, void *user);

/* Fills *opt with the defaults listed above. */
SWMD_API void swmd_default_options(swmd_options *opt);

/* Message of the last failing call on this thread ("" if none).  The pointer
 * stays valid until the next call on this thread. */
SWMD_API const char *swmd_last_error(void);

/* ------------------------------------------------------------------ a0: query selection */
/* Algorithm 1, first line, and Section III-B1: the query r is a histogram over
 * the vocabulary; keep its positive entries (I = r > 0) and normalise them to
 * sum 1.  Input: n (id, weight) pairs in host memory; ids repeat freely (their
 * weights add up), weights must be finite and >= 0, ids in [0, V).
 * Output (host, caller-allocated, capacity n): out_ids ascending, out_r
 * summing to 1 (rounded from FP64).  *out_vr receives the number of distinct
 * words.  SWMD_EINVAL if an id or weight is invalid or nothing is positive. */
SWMD_API int swmd_select(int32_t V, int32_t n, const int32_t *h_ids, const float *h_weights,
                int32_t *h_out_ids, float *h_out_r, int32_t *out_vr);

/* ------------------------------------------------------------------ multi-GPU */
/* Document ranges for `parts` GPUs.  The columns of c are independent problems
 * (Algorithm 1 never mixes them), so the corpus shards by contiguous document
 * ranges with no exchange during a query; the ranges are balanced by nonzeros,
 * the cross-GPU form of the equal-nnz split of Section III-D.
 *   doc_nnz[N] (int64, host): nonzeros of each document (column counts of c).
 *   out_bounds[parts+1] (int32, host): range g is [out_bounds[g], out_bounds[g+1]),
 *   out_bounds[0] = 0, out_bounds[parts] = N, non-decreasing.
 * Host-only (no CUDA call); SWMD_EINVAL for parts < 1 or a negative count.  Pass a
 * range as swmd_options.doc_begin / doc_end when creating each GPU's corpus. */
SWMD_API int swmd_partition_documents(int32_t N, const int64_t *doc_nnz, int32_t parts,
                                      int32_t *out_bounds);

/* ------------------------------------------------------------------ corpus */
/* Section III-B1: c is a V x N sparse matrix passed as CSR, c[i, j] the
 * frequency of word i in target document j; vecs is the V x d embedding matrix.
 *   row_ptr[V+1] (int64, host): CSR row offsets, row_ptr[0] = 0, non-decreasing,
 *       row_ptr[V] = nnz.
 *   doc_idx[nnz] (int32, host): column (document) of each nonzero, in [0, N).
 *   val[nnz] (float, host): the frequencies, finite and > 0.  Each column is
 *       normalised to sum 1 here, in FP64 (the paper's columns sum to one).
 *   emb[V*d] (float, host): row-major embeddings.
 * Every document must have at least one word (an empty column has no defined
 * distance): SWMD_EINVAL otherwise.  nnz < 2^31.  The corpus copies everything
 * to the device, builds a document-major copy of c (documents ordered by
 * length for load balance, words of a document ascending) and keeps only the
 * vocabulary words that occur in c for the cost-matrix kernel.
 * opt may be NULL (defaults).  On success *out owns the device memory. */
SWMD_API int swmd_create_corpus(int32_t V, int32_t N, int64_t nnz, const int64_t *row_ptr,
                       const int32_t *doc_idx, const float *val, const float *emb, int32_t d,
                       const swmd_options *opt, swmd_corpus **out);

/* Frees every device and host resource of the corpus.  NULL is ignored. */
SWMD_API void swmd_destroy_corpus(swmd_corpus *corpus);

typedef struct swmd_corpus_info {
    int32_t V, N, d;
    int32_t V_used;        /* vocabulary words that occur in c */
    int64_t nnz;
    int32_t doc_begin, doc_end;
    int32_t device;
    int64_t device_bytes;  /* bytes the corpus holds on the device, workspace included */
} swmd_corpus_info;

SWMD_API int swmd_corpus_get_info(const swmd_corpus *corpus, swmd_corpus_info *out);

/* The corpus's current options (as created, or as last set). */
SWMD_API int swmd_corpus_get_options(const swmd_corpus *corpus, swmd_options *out);

/* Changes the iteration path / K precision / graph use / mapping of later
 * queries (fields as in swmd_options; the corpus-shape fields are ignored). */
SWMD_API int swmd_corpus_set_options(swmd_corpus *corpus, const swmd_options *opt);

/* ------------------------------------------------------------------ whole query */
/* The paper's call sinkhorn_wmd(r, c, vecs, lambda, max_iter) (Section III-B1,
 * Algorithm 1): distances of the query to every document of the corpus.
 *   h_word_ids[n_words], h_weights[n_words]: the query as in swmd_select.
 *   lambda: finite, > 0 (K = exp(-lambda M)).
 *   max_iter: number t >= 0 of x-updates, then the final step.
 *   h_out_dist[N] (host, caller-allocated): WMD_j for j in the corpus's
 *       document range, in CSR column order, as double.
 * Blocks until the result is in h_out_dist.  SWMD_ENUMERIC if a NaN, an
 * infinity or a vanished K^T u appeared (the output is still written). */
SWMD_API int swmd_query(swmd_corpus *corpus, const int32_t *h_word_ids, const float *h_weights,
               int32_t n_words, float lambda, int32_t max_iter, double *h_out_dist);

/* Same computation with a query already selected and normalised (swmd_select)
 * and resident on the device, asynchronously on `stream`:
 *   d_ids[v_r] (int32, device): distinct word ids in [0, V).
 *   d_r[v_r] (float, device): weights summing to 1, all > 0.
 *   d_out[N] (double, device): the distances.
 * Returns after enqueueing; d_status (int32, device, may be NULL) receives 0 or
 * an SWMD_E* code when the stream reaches it (ids out of range: SWMD_EINVAL;
 * numerical failure: SWMD_ENUMERIC).  1 <= v_r <= max_vr. */
SWMD_API int swmd_query_device(swmd_corpus *corpus, const int32_t *d_ids, const float *d_r, int32_t v_r,
                      float lambda, int32_t max_iter, double *d_out, int32_t *d_status,
                      void *stream);

/* The query of swmd_query_device for callers that cannot allocate device
 * memory when they query -- for example a server whose memory pool already owns
 * the device's free memory, or a latency-critical request path that must avoid
 * the implicit synchronisation of cudaMalloc / cudaFree.  (The paper has no
 * counterpart: it is an interface for such callers, not a step of the method.)
 *   Arguments, layout, ownership and result as in swmd_query_device; the path is
 *   always SWMD_PATH_RESIDENT.  The corpus is created beforehand as usual.
 *   This call allocates nothing: the query's scratch (its parameter block, ids,
 *   weights, K^T and KM^T) lives in one fixed device array of 16 MiB inside the
 *   library, which every GPU that loads the library holds until the process
 *   exits.  A query needing more (2 x V_used x VRP x bytes per K element, plus
 *   under 2 KiB) is refused with SWMD_EINVAL and a message naming the sizes.
 *   The first call on a device looks up the array's device address on that
 *   device (cudaGetSymbolAddress); make that first call before any stream
 *   capture.
 *   All calls share the one array and it keeps the last call's contents; each
 *   call rewrites everything it reads (the status word is cleared by the call).
 *   Calls whose work overlaps on the GPU -- on different streams, or from
 *   different threads or corpora on the same device -- race on the array: order
 *   them on one stream or wait between them. */
SWMD_API int swmd_query_noalloc(swmd_corpus *corpus, const int32_t *d_ids, const float *d_r,
                                int32_t v_r, float lambda, int32_t max_iter, double *d_out,
                                int32_t *d_status, void *stream);

/* ------------------------------------------------------------------ the steps */
/* The steps of swmd_query_device, one call each, for timing and testing; they
 * share the corpus's workspace and must be called in this order for one query.
 * All are asynchronous on `stream`.  swmd_step_cost lays K^T out for the
 * corpus's current path (swmd_get_mapping); the later steps of the same query
 * walk that layout whatever their own path.
 *
 * a0 (device part) + a1, cost matrix and kernel (Algorithm 1 first line; Table I
 * "M = cdist(...)", "K = exp(-M*lamb)"; Section III-C "K.*M"): copies the
 * selected query (d_ids[v_r], d_r[v_r] as in swmd_query_device; d_r may be NULL
 * when only K is wanted) into the workspace, then for every used word w and query
 * word k computes M[k,w] = ||E[q_k] - E[w]||_2, K = exp(-lambda M) (column-shifted
 * if enabled) and K.*M, stored word-major (K^T[w][k], the KT layout of Section
 * III-B4).  d_status (may be NULL) becomes the status word of this query for the
 * later steps too. */
SWMD_API int swmd_step_cost(swmd_corpus *corpus, const int32_t *d_ids, const float *d_r,
                            int32_t v_r, float lambda, int32_t *d_status, void *stream);

/* a2 + a3, n_iter Sinkhorn x-updates (Algorithm 1 loop; Algorithms 2-3 fused as
 * SDDMM_SpMM, Section III-C): per document j and nonzero (w, c_wj),
 * s = K^T[w] . u_j, tau = c_wj / s, acc_j += tau K^T[w]; then u_j = r / acc_j
 * (that is x = diag(1/r) K v and u = 1/x).  first != 0 starts from x = 1/v_r.
 * path: SWMD_PATH_FUSED (one launch per iteration) or SWMD_PATH_PLAIN (an SDDMM
 * launch writing v, then an SpMM launch reading it). */
SWMD_API int swmd_step_iterate(swmd_corpus *corpus, int32_t v_r, int32_t n_iter, int32_t first,
                               int32_t path, void *stream);

/* a4, final step (Algorithm 1 last two lines, SDDMM_SpMM type 2 of Section
 * III-C): u = 1/x, v = c ./ (K^T u), WMD_j = sum_k u_kj ((K.*M) v)_kj, evaluated
 * per nonzero as sum_w c_wj (KM^T[w] . u_j) / (K^T[w] . u_j) with an FP64
 * per-document sum.  t0 != 0 means no iteration ran (u = v_r).  d_out[N]
 * (double, device) receives the distances in CSR column order. */
SWMD_API int swmd_step_final(swmd_corpus *corpus, int32_t v_r, int32_t t0, double *d_out,
                             void *stream);

/* a3 x max_iter + a4 in one launch (SWMD_PATH_RESIDENT), after swmd_step_cost. */
SWMD_API int swmd_step_resident(swmd_corpus *corpus, int32_t v_r, int32_t max_iter,
                                double *d_out, void *stream);

/* The layout and lane mapping the corpus uses for a query of v_r words on `path`
 * (SWMD_PATH_AUTO: the path it resolves to): out[0] = VRP (v_r padded: the row
 * length of K^T, KM^T and u), out[1] = Q, out[2] = P.  P > 0: the general walk,
 * P sub-teams of Q lanes own a document, each sub-team one nonzero at a time.
 * P = 0: the sliced walk (the per-iteration paths' default), VRP / 8 (FP32) or
 * VRP / 16 (BF16/FP16) lanes own a document, each lane a contiguous 32-byte slice
 * of every row; on the resident path P = 0 names the resident solvers. */
SWMD_API int swmd_get_mapping(swmd_corpus *corpus, int32_t v_r, int32_t path, int32_t *out3);

/* The number of x-updates the corpus's last single query (swmd_query,
 * swmd_query_device, or a per-iteration query of swmd_query_batch) applied: its
 * max_iter, or fewer when swmd_options.tol stopped it.  Synchronises the corpus's
 * stream. */
SWMD_API int swmd_last_iterations(swmd_corpus *corpus, int32_t *out_iterations);

/* The concrete path (SWMD_PATH_RESIDENT, FUSED or PLAIN) a query of v_r words
 * takes on this corpus: the corpus's path, or SWMD_PATH_AUTO's choice. */
SWMD_API int swmd_resolve_path(swmd_corpus *corpus, int32_t v_r, int32_t *out_path);

/* ------------------------------------------------------------------ 1-to-1 WMD */
/* The paper's per-pair variant (Section III-E, Table II, right column): the WMD of
 * each of n_pairs independent (query, target) pairs of histograms over the corpus's
 * vocabulary and embeddings, with the cost matrix built only over the target's v_x
 * distinct words, so a pair costs O(v_x v_r d + t v_x v_r) instead of the 1-to-N
 * query's O(V v_r d + t nnz v_r).  It is Algorithm 1 with c the target histogram
 * as a single column (a word outside the target has c = 0 and adds nothing), so a
 * pair's distance equals that document's entry of the 1-to-N result up to rounding.
 * Use it when a query meets few documents (re-ranking candidates, pairwise
 * distances); the corpus's c is not used, only its embeddings and column_shift.
 *   Pair p: query words h_q_ids[h_q_ptr[p] .. h_q_ptr[p+1]) with h_q_weights,
 *   target words h_x_ids[h_x_ptr[p] .. h_x_ptr[p+1]) with h_x_weights (host
 *   arrays; h_q_ptr[0] = h_x_ptr[0] = 0, non-decreasing).  Each side is selected
 *   and normalised like a query (swmd_select: repeated ids add up, zero weights
 *   drop, sum 1); after that each side has 1 .. 4096 distinct words.
 *   lambda finite > 0; max_iter >= 0 x-updates; tol: 0 = exactly max_iter updates,
 *   > 0 = stop once max_k |u_k (K v)_k - r_k| < tol (Algorithm 1's "while x
 *   changes") with max_iter as the cap -- per pair.
 *   h_out[n_pairs] (double): the distances; h_iters[n_pairs] (int32, may be NULL):
 *   the x-updates each pair ran.
 * FP32 arithmetic (K and K.*M in FP32 whatever the corpus's k_precision), FP64
 * final sum.  Blocks until the results are in host memory.  SWMD_EINVAL names the
 * first invalid pair side; SWMD_ENUMERIC as for swmd_query. */
SWMD_API int swmd_wmd_pairs(swmd_corpus *corpus, int32_t n_pairs, const int64_t *h_q_ptr,
                            const int32_t *h_q_ids, const float *h_q_weights,
                            const int64_t *h_x_ptr, const int32_t *h_x_ids,
                            const float *h_x_weights, float lambda, int32_t max_iter, float tol,
                            double *h_out, int32_t *h_iters);

/* swmd_wmd_pairs on sides already selected and normalised (distinct ids, weights
 * > 0 summing to 1) and resident on the device, asynchronously on `stream`:
 *   d_q_ptr[n_pairs+1], d_x_ptr[n_pairs+1] (int64), d_q_ids / d_x_ids (int32),
 *   d_r / d_c (float): as in swmd_wmd_pairs, in device memory.  Distinct ids are
 *   the caller's promise (not checked).
 *   max_q_words, max_x_words (1 .. 4096): bounds on every pair's side sizes; they
 *   size the launch's shared memory, so tight bounds run faster.
 *   d_out[n_pairs] (double), d_iters[n_pairs] (int32, may be NULL), d_status
 *   (int32, required): the status word is OR-ed with the SWMD_E* condition bits of
 *   the kernels (the caller zeroes it); a pair with an id outside [0, V), a weight
 *   that is not finite and > 0, or a side outside [1, bound] gets a NaN distance.
 * When K and K.*M of the largest pair (8 (max_q_words + 1) max_x_words bytes)
 * exceed 48 KiB they live in a per-block region of global memory that the corpus
 * allocates (at most 2 GiB) the first time a call needs it; that allocation
 * synchronises the device, so make one call with the largest bounds before any
 * stream capture. */
SWMD_API int swmd_wmd_pairs_device(swmd_corpus *corpus, int32_t n_pairs, const int64_t *d_q_ptr,
                                   const int32_t *d_q_ids, const float *d_r,
                                   const int64_t *d_x_ptr, const int32_t *d_x_ids,
                                   const float *d_c, int32_t max_q_words, int32_t max_x_words,
                                   float lambda, int32_t max_iter, float tol, double *d_out,
                                   int32_t *d_iters, int32_t *d_status, void *stream);

/* Debug builds only (the library built with build(debug=True), whose kernels check
 * the corpus indices they follow and report one outside its array in the status
 * word instead of reading there): overwrites the compact word id of one nonzero of
 * the corpus's device copy with `value`, to test those checks from the host.
 *   what 0: nonzero `index` (0 .. nnz-1) of the document-major copy (the resident
 *   solvers read it); what 1: entry `index` of the sliced copy (the per-iteration
 *   walks read it; its padding entries too).
 * A later query whose kernels meet the planted id returns SWMD_EINVAL naming the
 * failed bounds check.  Release builds return SWMD_EINVAL and change nothing.
 * Synchronous.  A test hook: the paper has no counterpart. */
SWMD_API int swmd_debug_plant(swmd_corpus *corpus, int32_t what, int64_t index, int32_t value);

/* Copies a workspace array to host memory for inspection (tests):
 *   what 0: K^T  [V_used][v_r] as float (FP32/BF16/FP16 widened)
 *   what 1: KM^T [V_used][v_r] as float
 *   what 2: u    [N][v_r] as float, CSR column order
 *   what 3: the used word ids [V_used] as int32
 * h_dst must hold the stated number of elements.  Synchronous. */
SWMD_API int swmd_debug_read(swmd_corpus *corpus, int32_t what, int32_t v_r, void *h_dst);

/* ------------------------------------------------------------------ autotuning */
typedef struct swmd_tune_result {
    int32_t vrp;           /* the resident layout of the chosen solver (VRP for v_r) */
    int32_t solver;        /* chosen resident solver (see swmd_options.solver) */
    int32_t nnz_per_lane;  /* chosen rows of K^T per lane (register solver) */
    int32_t cost_split;    /* chosen cost kernel (see swmd_options.cost_split) */
    float default_ms;      /* whole-query time with the settings before tuning */
    float best_ms;         /* whole-query time with the chosen settings */
    int32_t candidates;    /* configurations timed */
    int32_t path;          /* the path chosen for this v_r (SWMD_PATH_RESIDENT or, under
                              SWMD_PATH_AUTO, SWMD_PATH_FUSED when that was faster) */
} swmd_tune_result;

/* Times the resident-path kernels of this corpus for queries of v_r words over
 * the candidate solvers and lane mappings (column-split register solver; register
 * solver rows per lane; shared-memory solver; the cost kernel: product form or
 * row kernel with 1, 2 or 4 threads per word), each `reps` times (>= 1) with CUDA events on a query of v_r distinct
 * words, and keeps the fastest: later queries of v_r words with the same K
 * precision use it unless swmd_options fixes the field.  On a corpus with SWMD_PATH_AUTO it also times the
 * per-iteration fused path and records, for this v_r, whichever path was faster.
 * The corpus's path must be SWMD_PATH_RESIDENT or SWMD_PATH_AUTO.  Synchronous;
 * allocates nothing beyond the corpus's workspace; call it before serving from the
 * corpus (a running server reads the tuning).  A tuned setting may change the
 * rounding of later results (within the FP32 tolerance), never their meaning.  The
 * paper has no counterpart (it tuned by hand for Xeon and PIUMA, Sections IV-V). */
SWMD_API int swmd_autotune(swmd_corpus *corpus, int32_t v_r, int32_t reps, swmd_tune_result *out);

/* ------------------------------------------------------------------ batch */
typedef struct swmd_batch_tune_result {
    int32_t layouts;        /* column-split layouts (VRP values) the batch holds */
    int32_t vrp[4];         /* those layouts ... */
    int32_t queries_per_tile[4];   /* ... and the tile size chosen for each */
    float default_ms;       /* the batch with the default tile sizes */
    float best_ms;          /* the batch with the chosen ones */
    int32_t candidates;     /* batches timed */
} swmd_batch_tune_result;

/* Times swmd_query_batch on this batch (arguments as in swmd_query_batch; the
 * distances are discarded) for every queries_per_tile candidate (1, 2, 4, 8) of the
 * column-split layouts it holds, `reps` times each (>= 1), and keeps the fastest
 * for each layout and K precision: later batches use it unless
 * swmd_options.queries_per_tile fixes it.  Synchronous; refused while a server is
 * attached.  The tile size changes which queries share a tile, never a distance's
 * bits.  The paper has no counterpart (Section III-D's hierarchical threading was
 * chosen by hand). */
SWMD_API int swmd_autotune_batch(swmd_corpus *corpus, int32_t n_queries, const int64_t *q_ptr,
                                 const int32_t *h_word_ids, const float *h_weights,
                                 const float *h_lambdas, int32_t max_iter, int32_t reps,
                                 swmd_batch_tune_result *out);

/* Several queries at once (Section III-D notes that many source documents can
 * run together; the paper's multi-query experiment, Section V):
 *   q_ptr[n_queries+1] (int64, host): query i is entries q_ptr[i]..q_ptr[i+1]-1
 *       of h_word_ids / h_weights (each as in swmd_query).
 *   h_lambdas[n_queries] (float, host): lambda of each query.
 *   h_out[n_queries * N] (double, host): row i = the distances of query i.
 * Each query takes its own path (swmd_resolve_path).  The resident queries of one
 * K^T layout and solver run as batched cost and solver launches.  With the
 * column-split solver a launch pair takes one group of swmd_options.queries_per_tile
 * queries (or the autotuned or L2-sized number), so the group's K^T is still in L2
 * when its solver runs, and the solver walks (query, document task) tiles: a
 * task's nonzeros are read from DRAM once for the group.  The other resident
 * solvers run the layout's queries as grid rows of one launch pair on corpora
 * under 20,000 documents and one launch pair per query above.  The per-iteration
 * queries run one after another.  The device work of the whole call runs eagerly
 * the first time a batch shape (the queries' paths and sizes, the per-iteration
 * queries' lambdas, max_iter) is seen, is captured as a CUDA graph the second
 * time, and is replayed after that (up to 64 shapes are remembered).  The
 * workspace grows on demand and is kept.  The result of each query equals its swmd_query result bit for bit.
 * Returns the first failing query's error, or SWMD_ENUMERIC if any query flagged
 * a NaN / infinity (the distances are still written). */
SWMD_API int swmd_query_batch(swmd_corpus *corpus, int32_t n_queries, const int64_t *q_ptr,
                     const int32_t *h_word_ids, const float *h_weights, const float *h_lambdas,
                     int32_t max_iter, double *h_out);

/* ------------------------------------------------------------------ serving */
typedef struct swmd_serve_config {
    int32_t max_batch;         /* queries admitted into one device batch (default 32) */
    int64_t memory_budget;     /* device bytes for in-flight queries' K, K.*M and u (default 4 GiB) */
    int32_t max_wait_us;       /* a partial batch is launched after this wait (default 200) */
    int32_t queue_capacity;    /* pending requests accepted before submit refuses (default 4096) */
    int32_t reserved[4];
} swmd_serve_config;

typedef struct swmd_serve_stats_t {
    int64_t completed;
    int64_t rejected;
    double qps;        /* completed / seconds since start */
    double p50_ms;     /* submit-to-result latency percentiles over completed requests */
    double p99_ms;
    double mean_batch; /* mean queries per device batch */
    int64_t batches;
} swmd_serve_stats_t;

SWMD_API void swmd_default_serve_config(swmd_serve_config *cfg);

/* Starts a serving thread over a resident corpus.  Requests are admitted into
 * device batches as memory (K, K.*M and u of each query) frees up, and a batch
 * runs while later requests queue (continuous batching).  cfg may be NULL.
 * SWMD_ENOMEM if memory_budget is below the bytes one query of max_vr words needs.
 * Host memory: max_batch result buffers of N doubles, recycled through
 * swmd_serve_wait (up to 2 max_batch are kept).
 * While a server is attached, swmd_autotune and swmd_corpus_set_options on its
 * corpus are refused (SWMD_EINVAL): a request's path and layout are resolved once,
 * when it is admitted. */
SWMD_API int swmd_serve_start(swmd_corpus *corpus, const swmd_serve_config *cfg, swmd_server **out);

/* Queues one query (host arrays copied during the call).  *ticket identifies it.
 * SWMD_ENOMEM (and the request is counted as rejected) when queue_capacity requests
 * are already pending; SWMD_ESTOPPED once swmd_serve_stop has begun. */
SWMD_API int swmd_serve_submit(swmd_server *srv, const int32_t *h_ids, const float *h_weights,
                      int32_t n_words, float lambda, int32_t max_iter, uint64_t *ticket);

/* Waits up to timeout_ms (< 0: forever) for the result of `ticket` and copies
 * its N distances to h_out_dist.  SWMD_ETIMEDOUT if it is not ready in time
 * (the request stays queued and can be waited for again).  A result is handed out
 * once: a wait on a ticket already collected, or collected by a concurrent waiter,
 * returns SWMD_EINVAL. */
SWMD_API int swmd_serve_wait(swmd_server *srv, uint64_t ticket, double *h_out_dist, int32_t timeout_ms);

SWMD_API int swmd_serve_stats(swmd_server *srv, swmd_serve_stats_t *out);

/* Stops the server after finishing in-flight batches; pending requests fail
 * with SWMD_ESTOPPED, and threads blocked in swmd_serve_wait on them return that
 * code before the server is freed.  No call may use the server after this returns. */
SWMD_API int swmd_serve_stop(swmd_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* SWMD_H */
