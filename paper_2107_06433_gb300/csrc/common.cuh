// Internal declarations shared by the kernel files and the C-ABI layer of libswmd.
//
// Device data layout (document-major, the transpose of the paper's V x N CSR c):
//   doc_ptr[Nl+1]  int32   offsets of each document's nonzeros; documents are kept
//                          in decreasing-length order (internal order) so that the
//                          documents sharing a warp have similar lengths.
//   nz[nnz]        int2    (compact word id, bits of the FP32 normalised count);
//                          words ascending inside a document.
//   doc_orig[Nl]   int32   internal -> caller's column index (relative to doc_begin).
//   used[Vu]       int32   compact word id -> vocabulary id (words that occur in c).
//   E[V][d4]       float   embeddings, rows padded with zeros to d4 = roundup(d, 4).
// Per query (workspace):
//   KT[Vu][VRP], KMT[Vu][VRP]  K^T and (K.*M)^T, word-major (KT[vocab][v_r] of
//                          Section III-B4), FP32 / BF16 / FP16, padded columns 0.
//   u[Nl][VRP]             float, document-major (u[num_docs][v_r] of Section
//                          III-B4), padded entries 0.
//   VRP = v_r rounded up to the kernel's padding (a multiple of 4).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace swmd {

// Bits of the device status word.
constexpr int ST_BAD_ID = 1;       // a query id outside [0, V)
constexpr int ST_NUMERIC = 2;      // NaN / Inf / zero denominator
constexpr int ST_GUARD = 4;        // the FP64 guard of K^T u was taken (informational)
constexpr int ST_BAD_R = 8;        // a query weight that is not finite and > 0
constexpr int ST_BOUNDS = 32;      // debug builds: a corpus index outside its array

// Debug builds (SWMD_DEBUG_CHECKS=1, build(debug=True)) check the corpus indices the
// kernels follow -- compact word ids and document offsets -- before using them: an
// index outside [0, n) sets ST_BOUNDS in the status word and is replaced by 0, so
// nothing outside the arrays is read (no trap, no assert).  Release builds use the
// index as it is.
#ifndef SWMD_DEBUG_CHECKS
#define SWMD_DEBUG_CHECKS 0
#endif
__device__ __forceinline__ int checked_index(int i, long n, int *status) {
#if SWMD_DEBUG_CHECKS
    if (i < 0 || (long)i >= n) {
        atomicOr(status, ST_BOUNDS);
        return 0;
    }
#else
    (void)n;
    (void)status;
#endif
    return i;
}

// Query parameters read by the kernels from device memory, so that a captured
// graph stays valid when lambda or v_r change.
struct QParams {
    float lambda;
    int vr;
    float u0;        // initial u = 1/x = v_r
    int pad;
    double *out;     // where the final kernel writes the distances (caller order)
    int *status;     // status word of this query
};

// Documents per slice of the sliced nonzero layout, and the multiple its row
// count is padded to (so a walk takes rows in fours without bounds checks).
constexpr int kSliceDocs = 32;
constexpr int kSliceRows = 4;

struct IterArgs {
    const int *doc_ptr;
    const int2 *nz;
    const void *KT;
    const void *KMT;
    float *u;
    const float *r;        // [VRP], zero-padded
    float *v;              // plain path: [nnz] SDDMM output
    const int *doc_orig;
    const QParams *qp;
    long doc0;             // first document (internal order) of this launch
    int N;                 // documents in this launch
    int Vu;                // rows of K^T (compact words): bounds of the debug checks
    int first;             // 1: u = v_r (x = 1/v_r), do not read u
    double *out;           // if not NULL, the distances go here instead of qp->out
    // sliced nonzeros (per-iteration walks): slices of 32 documents, entry (i, t)
    // of slice s at slice_ptr[s] + 32 i + t; v (plain path) uses the same positions
    const int *slice_ptr;
    const int2 *slice_nz;
    int n_slices;
    // convergence mode (tol > 0): conv[1 + i] holds the largest |u (K v) - r| of
    // iteration i (float bits, atomicMax), conv[0] the x-updates applied; launch
    // `it` does nothing once iteration it - 1 came below tol
    float tol;
    unsigned *conv;
    int it;
};

constexpr int kMaxConvIters = 4096;

struct CostArgs {
    const float *E;
    int d4;
    const int *used;
    int Vu;
    const int *q_ids;
    const QParams *qp;
    int V;
    int shift;
    int split;     // threads per word in the row kernel (1, 2, 4)
    void *KT;
    void *KMT;
};

struct ResidentArgs {
    IterArgs it;
    int t;                 // Sinkhorn iterations
};

// One mapping of the per-document walk: a team of P*Q lanes owns a document, P
// nonzeros are in flight at a time and Q lanes share one nonzero's dot product.
struct Mapping {
    int vrp;
    int q;
    int p;
};

// Launchers (return cudaError_t of the launch).
cudaError_t launch_cost(const CostArgs &a, int vrp, int kprec, cudaStream_t s);
// Batched forms: grid row y runs query y with d_batch[y] (device array); `shape`
// supplies the fields shared by the batch (corpus arrays, sizes).
cudaError_t launch_cost_batch(const CostArgs &shape, int vrp, int kprec, int nq,
                              const CostArgs *d_batch, cudaStream_t s);
struct PrepArgs {
    QParams *qp;
    const int *src_ids;
    const float *src_r;
    int *q_ids;
    float *r;
    double *out;
    int *status;
    float lambda;
    int vr;
    int vrp_cap;
    int pad;
};
cudaError_t launch_prep_batch(const PrepArgs *d_args, int nq, int V, cudaStream_t s);
// Writes the parameter block of a query and copies / validates its ids and
// weights into the slot (zero padded to vrp_cap).  src_ids / src_r may be NULL
// to leave that array as it is.
cudaError_t launch_prep(QParams *qp, float lambda, int vr, int V, const int *src_ids,
                        const float *src_r, int *q_ids, float *r, int vrp_cap, double *out,
                        int *status, cudaStream_t s);
cudaError_t launch_fused(const IterArgs &a, Mapping m, int kprec, int sms, cudaStream_t s);
cudaError_t launch_sddmm(const IterArgs &a, Mapping m, int kprec, int sms, cudaStream_t s);
cudaError_t launch_spmm(const IterArgs &a, Mapping m, int kprec, int sms, cudaStream_t s);
cudaError_t launch_final(const IterArgs &a, Mapping m, int kprec, int sms, cudaStream_t s);
cudaError_t launch_resident(const ResidentArgs &a, Mapping m, int kprec, int sms,
                            cudaStream_t s);
// Walks over the sliced nonzeros with lanes over k (VRP in {4, 8, 16, 32, 64, 128}).
cudaError_t launch_fused3(const IterArgs &a, int vrp, int kprec, int sms, cudaStream_t s);
cudaError_t launch_sddmm3(const IterArgs &a, int vrp, int kprec, int sms, cudaStream_t s);
cudaError_t launch_spmm3(const IterArgs &a, int vrp, int kprec, int sms, cudaStream_t s);
cudaError_t launch_final3(const IterArgs &a, int vrp, int kprec, int sms, cudaStream_t s);
// Documents packed into tiles of at most `nt` nonzeros (at most 64 documents,
// consecutive in the internal order): tiles[0..n_tiles] are document offsets.
struct TileSet {
    const int *tiles;
    int n_tiles;
    int nt;        // nonzeros staged per block
    int threads;   // threads per block
    int npl;       // nonzeros per lane and pass (team size rule)
};
// Lanes of the team that owns a document of `len` nonzeros in the tiled resident
// solver: the power of two in [4, 32] that gives about `npl` nonzeros per lane and
// pass.  A function of the document alone, so a document's arithmetic (and
// result) does not depend on which documents share its tile, batch or GPU.
__host__ __device__ inline int team_lanes_for(int len, int npl) {
    int g = 4;
    while (g < 32 && g * npl < len) g *= 2;
    return g;
}
// Team size of the register-resident solver: the power of two in [1, 32] that
// covers `len` nonzeros with at most `npl` per lane (longer documents use 32
// lanes and re-read their excess rows).  A function of the document alone.
__host__ __device__ inline int reg_team_lanes(int len, int npl) {
    int g = 1;
    while (g < 32 && g * npl < len) g *= 2;
    return g;
}
// Warp tasks of the register-resident solver: (first document, team size,
// documents) -- consecutive documents of one team size, 32 / team size at most.
struct TaskSet {
    const int4 *tasks;
    int n_tasks;
    int npl;
    int max_len;   // longest document (sizes the per-warp overflow buffer)
};
int regs_rows_per_lane(int vrp, int want);
// one translation unit per K precision (resident_regs_{fp32,bf16,fp16}.cu)
cudaError_t launch_regs_fp32(const ResidentArgs &a, int vrp, const TaskSet &ts, int sms, cudaStream_t s,
                             int nq, const ResidentArgs *batch);
cudaError_t launch_regs_bf16(const ResidentArgs &a, int vrp, const TaskSet &ts, int sms, cudaStream_t s,
                             int nq, const ResidentArgs *batch);
cudaError_t launch_regs_fp16(const ResidentArgs &a, int vrp, const TaskSet &ts, int sms, cudaStream_t s,
                             int nq, const ResidentArgs *batch);
cudaError_t launch_resident_regs(const ResidentArgs &a, int vrp, int kprec, const TaskSet &ts,
                                 int sms, cudaStream_t s, int nq = 1,
                                 const ResidentArgs *d_batch = nullptr);
size_t tiled_smem_bytes(int vrp, int kbytes, int nt);
bool tiled_supported(int vrp, int kprec);
cudaError_t launch_resident_tiled(const ResidentArgs &a, int vrp, int kprec, const TileSet &ts,
                                  int sms, cudaStream_t s, int nq = 1,
                                  const ResidentArgs *d_batch = nullptr);
bool mapping_supported(Mapping m);
int vrp_for(int vr, int q);

// ---------------------------------------------------------------- K element access
// Four consecutive K values (16 B in FP32, 8 B in BF16/FP16), widened to float.
template <class T> struct KIO;

template <> struct KIO<float> {
    static __device__ __forceinline__ float4 load4(const float *base, long idx4) {
        return __ldg(reinterpret_cast<const float4 *>(base) + idx4);
    }
    static __device__ __forceinline__ void store4(float *base, long idx4, float4 v) {
        reinterpret_cast<float4 *>(base)[idx4] = v;
    }
};

template <> struct KIO<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load4(const __nv_bfloat16 *base, long idx4) {
        uint2 raw = __ldg(reinterpret_cast<const uint2 *>(base) + idx4);
        __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&raw.x);
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&raw.y);
        float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ void store4(__nv_bfloat16 *base, long idx4, float4 v) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
        __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
        uint2 raw;
        raw.x = *reinterpret_cast<uint32_t *>(&a);
        raw.y = *reinterpret_cast<uint32_t *>(&b);
        reinterpret_cast<uint2 *>(base)[idx4] = raw;
    }
};

template <> struct KIO<__half> {
    static __device__ __forceinline__ float4 load4(const __half *base, long idx4) {
        uint2 raw = __ldg(reinterpret_cast<const uint2 *>(base) + idx4);
        __half2 a = *reinterpret_cast<__half2 *>(&raw.x);
        __half2 b = *reinterpret_cast<__half2 *>(&raw.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ void store4(__half *base, long idx4, float4 v) {
        __half2 a = __floats2half2_rn(v.x, v.y);
        __half2 b = __floats2half2_rn(v.z, v.w);
        uint2 raw;
        raw.x = *reinterpret_cast<uint32_t *>(&a);
        raw.y = *reinterpret_cast<uint32_t *>(&b);
        reinterpret_cast<uint2 *>(base)[idx4] = raw;
    }
};

inline size_t kprec_bytes(int kprec) { return kprec == 0 ? 4 : 2; }

// ---------------------------------------------------------------- launch settings
// Launch settings of one kernel, kept per device and read under a lock.
// cudaFuncSetAttribute applies to the current device only, and the occupancy a
// grid is sized from depends on the device, so neither may be shared between the
// GPUs one process drives.
constexpr int kMaxDevices = 64;
struct LaunchCache {
    std::mutex mu;
    size_t smem_set[kMaxDevices] = {};   // dynamic shared-memory limit raised to, per device
    bool carve_set[kMaxDevices] = {};    // preferred carveout set on the device
    int per_sm[kMaxDevices] = {};        // resident blocks per SM ...
    size_t key[kMaxDevices] = {};        // ... measured for this (shared memory, threads)

    // Blocks of `kern` per SM on the current device at `threads` threads and `smem`
    // bytes of dynamic shared memory, raising the kernel's dynamic shared-memory
    // limit on this device to `smem` first; carveout >= 0 also sets the
    // preferred shared-memory carveout (percent) once per device (a hint: a refusal
    // is ignored).
    template <class K>
    cudaError_t blocks_per_sm(K kern, int threads, size_t smem, int carveout, int *out) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lk(mu);
        // (raised for any size above the last: the 48 KiB default covers static and
        // dynamic shared memory together)
        if (smem > smem_set[dev]) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            smem_set[dev] = smem;
            key[dev] = 0;
        }
        if (carveout >= 0 && !carve_set[dev]) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carveout) !=
                cudaSuccess)
                (void)cudaGetLastError();
            carve_set[dev] = true;
            key[dev] = 0;
        }
        const size_t k = (smem << 12) + (size_t)threads + 1;   // threads < 4096
        if (key[dev] != k) {
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess || n < 1) {
                (void)cudaGetLastError();
                n = 1;
            }
            per_sm[dev] = n;
            key[dev] = k;
        }
        *out = per_sm[dev];
        return cudaSuccess;
    }
};

// ---------------------------------------------------------------- column-split solver
// Arguments of the column-split register solver (resident_cols.cu).  The per-query
// fields come from a ResidentArgs (it.KT, it.KMT at a power-of-two VRP in 4..128,
// it.r zero-padded to VRP, it.qp, it.out, t).
struct ColArgs {
    const int *doc_ptr;
    const int2 *nz;
    const int *doc_orig;
    const int4 *tasks;     // (first document, documents, bucket, 0) warp tasks
    int n_tasks;
    int long_docs;         // the tasks include buckets of 48, 64 or 96 rows
    int kprec;
    int Vu;                // rows of K^T (debug checks)
    long nnz;              // nonzeros (debug checks)
    ResidentArgs q0;                 // the query when `queries` is NULL
    const ResidentArgs *queries;     // else: device array of nq queries of this layout, run
    int nq;                          // in one launch over (group of q_per_group queries,
    int q_per_group;                 // document task) tiles
};
// Rows a document of `len` words occupies in the column-split solver for layout
// `vrp` (the bucket: 8, 16, 24, 32, 48, 64 or 96 rows, those the layout's row groups
// can hold); 0 if too long for the layout.
int cols_bucket(int len, int vrp);
// The longest document the column-split solver holds in layout `vrp`: 96 words at
// 16 and 32 columns, 32 at 64 and 128.
int cols_max_len(int vrp);
constexpr int kColMaxRowsPerLane = 12;   // rows a lane holds with eight columns
// Columns of every row a lane holds (P = 8) and lanes of a row group (Q = vrp / P).
__host__ __device__ constexpr int cols_p(int) { return 8; }
__host__ __device__ constexpr int cols_q(int vrp) { return vrp / cols_p(vrp); }
// A bucket of lmax rows is held by G row groups of Q lanes, each group RL = lmax / G
// rows: the smallest power of two G with RL a multiple of Q and at most 12 (at most
// Q when Q > 12: the 128-column layout's 16-lane groups hold 16 rows), G Q <= 32
// lanes; 0 when there is none (the bucket does not exist for that layout).
__host__ __device__ constexpr int cols_groups(int lmax, int vrp) {
    for (int g = 1; g <= 8; g *= 2) {
        const int rl = lmax / g, q = cols_q(vrp);
        const int cap = q > kColMaxRowsPerLane ? q : kColMaxRowsPerLane;
        if (lmax % g == 0 && rl % q == 0 && rl <= cap && g * q <= 32) return g;
    }
    return 0;
}
__host__ __device__ constexpr bool cols_fits(int lmax, int vrp) { return cols_groups(lmax, vrp) > 0; }
// Lanes that own one document of a bucket (G Q).
__host__ __device__ constexpr int cols_team(int lmax, int vrp) { return cols_groups(lmax, vrp) * cols_q(vrp); }
// Documents of a bucket one warp task holds (32 / cols_team).
int cols_docs_per_task(int lmax, int vrp);
bool cols_supported(int vrp);
// The layout (VRP) the column-split solver uses for a query of vr words: the
// power of two >= max(vr, 16).
int cols_vrp(int vr);
// Index of a column-split layout in the corpus's task lists (VRP 16, 32, 64, 128).
inline int cols_index(int vrp) { return vrp == 16 ? 0 : vrp == 32 ? 1 : vrp == 64 ? 2 : 3; }
constexpr int kColLayouts = 4;
// Runs all t iterations and the final step for every document of the tasks, for
// a.q0, or (a.queries != NULL) for the a.nq = nq queries of a.queries in one launch.
cudaError_t launch_resident_cols(const ColArgs &a, int vrp, int sms, cudaStream_t s, int nq);
// The same for task lists with buckets of 48 to 96 rows (a.long_docs; 16 and 32 columns).
cudaError_t launch_resident_cols_long(const ColArgs &a, int vrp, int sms, cudaStream_t s, int nq);


}  // namespace swmd
