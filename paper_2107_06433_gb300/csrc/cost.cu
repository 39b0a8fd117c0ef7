// a1: cost matrix and Sinkhorn kernel for one query.
//
// Algorithm 1 (first line) and Table I: M = cdist(vecs[sel], vecs) with the
// Euclidean distance of Section II-A, K = exp(-lambda M); Section III-C adds K.*M
// (the third dense input of SDDMM_SpMM type 2).  Only vocabulary words that
// occur in the corpus get a row: no nonzero of c ever reads the others.
//
// Two forms.  Layouts of 16, 32 and 64 columns (and the 64-column chunks of 128)
// take k_cost_tile, which evaluates M^2 = |q|^2 + |e|^2 - 2 q.e as a register-tiled
// product and falls back to the difference form near M = 0 (below).  The others,
// and any layout when a cost split is asked for, take the row kernels:
//
// Mapping: T adjacent threads own one word w and split the VRP query words,
// KPT = VRP / T each.  The query rows are staged transposed in shared memory,
// DC dimensions at a time, and read as float4 broadcasts; each thread streams
// its word's embedding row with float4 loads.  Distances use the direct
// difference form sum_d (q_d - e_d)^2 (no |q|^2 + |e|^2 - 2 q.e cancellation),
// evaluated two query words per instruction with the packed f32x2 FMA of sm_100+.
// Output rows K^T[w][0..VRP) and KM^T[w][0..VRP) are written with vector stores;
// columns k >= v_r are zero.  With column_shift, K[k,w] = exp(-lambda (M[k,w] -
// min_k M[k,w])): a rescaling of column w of K that leaves every x-update and the
// distance unchanged and keeps the largest entry of each column at 1.
#include <type_traits>

#include "common.cuh"

namespace swmd {
namespace {

constexpr int kCostThreads = 128;
constexpr int kDC = 32;  // embedding dimensions per shared-memory stage

// acc + (q - e)^2 on a pair of query words: the difference is rounded once (an FMA
// of e by -1 plus q is the exact q - e, rounded once: the same as a subtraction),
// then one FMA.  Both are packed f32x2 FMAs of sm_100+.
__device__ __forceinline__ float2 sqdiff_acc2(float2 q, float2 e, float2 acc) {
    const float2 t = __ffma2_rn(e, make_float2(-1.f, -1.f), q);
    return __ffma2_rn(t, t, acc);
}

// Column factor b_w of the stored K (an exact rescaling of column w, like the
// shift): 1 except for FP16 storage, where b_w = 2^14 / max(1, max_k M[k,w]) lifts
// the shifted column (largest entry 1) out of FP16's subnormal range while K b_w
// and K.*M b_w stay below 2^14.
template <class KT_t>
__device__ __forceinline__ float storage_scale(float mmax) {
    if constexpr (std::is_same<KT_t, __half>::value) return 16384.f / fmaxf(1.f, mmax);
    return 1.f;
}

// Scratch place of the distance M[w][k] while a wide layout's cost is computed in
// 32-column chunks: inside the word's own output rows, columns below vrp / 2 in
// the K^T row and the others in the KM^T row, as FP32 (a row of vrp elements of
// kbytes bytes holds vrp kbytes / 4 floats, at least vrp / 2).
__device__ __forceinline__ float *cost_scratch(const CostArgs &a, long wi, int k, int vrp, int kbytes) {
    const long stride = (long)vrp * kbytes / 4;
    const int half = vrp / 2;
    float *base = reinterpret_cast<float *>(k < half ? a.KT : a.KMT);
    return base + wi * stride + (k < half ? k : k - half);
}

template <class KT_t> __device__ __forceinline__ KT_t to_k(float x);
template <> __device__ __forceinline__ float to_k<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 to_k<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __half to_k<__half>(float x) { return __float2half_rn(x); }

template <int KPT, int T, class KT_t>
__device__ __noinline__ void k_cost_body(const CostArgs &a) {
    constexpr int VRP = KPT * T;
    constexpr int ROW = KPT + 4;  // padded slice: T slices of a stage row in distinct banks
    static_assert(KPT % 4 == 0, "KPT must be a multiple of 4");
    __shared__ __align__(16) float sq[kDC][T][ROW];

    const int vr = a.qp->vr;
    const float lam = a.qp->lambda;
    const int tid = threadIdx.x;
    const int sub = tid % T;
    const long wi = (long)blockIdx.x * (kCostThreads / T) + tid / T;
    const bool active = wi < a.Vu;
    const float *erow = a.E + (size_t)(active ? __ldg(a.used + wi) : 0) * a.d4;

    float2 acc[KPT / 2];
#pragma unroll
    for (int i = 0; i < KPT / 2; ++i) acc[i] = make_float2(0.f, 0.f);

    for (int d0 = 0; d0 < a.d4; d0 += kDC) {
        const int dn = min(kDC, a.d4 - d0);
        __syncthreads();
#pragma unroll 4
        for (int i = tid; i < dn * VRP; i += kCostThreads) {
            // query word fastest across threads: independent loads, and the stores
            // of a warp fill consecutive slots
            const int dd = i / VRP, k = i - dd * VRP;
            float val = 0.f;
            if (k < vr) {
                const int qid = __ldg(a.q_ids + k);
                if (qid >= 0 && qid < a.V) val = __ldg(a.E + (size_t)qid * a.d4 + d0 + dd);
            }
            sq[dd][k / KPT][k % KPT] = val;
        }
        __syncthreads();
        if (active) {
#pragma unroll 2
            for (int dd = 0; dd < dn; dd += 4) {
                const float4 e = __ldg(reinterpret_cast<const float4 *>(erow + d0 + dd));
                const float ev[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 e2 = make_float2(ev[j], ev[j]);
                    const float4 *qrow = reinterpret_cast<const float4 *>(&sq[dd + j][sub][0]);
#pragma unroll
                    for (int c = 0; c < KPT / 4; ++c) {
                        const float4 qv = qrow[c];
                        acc[2 * c] = sqdiff_acc2(make_float2(qv.x, qv.y), e2, acc[2 * c]);
                        acc[2 * c + 1] = sqdiff_acc2(make_float2(qv.z, qv.w), e2, acc[2 * c + 1]);
                    }
                }
            }
        }
    }

    float m[KPT];
#pragma unroll
    for (int i = 0; i < KPT / 2; ++i) {
        m[2 * i] = sqrtf(acc[i].x);
        m[2 * i + 1] = sqrtf(acc[i].y);
    }
    float mn = INFINITY, mx = 0.f;
#pragma unroll
    for (int kk = 0; kk < KPT; ++kk)
        if (sub * KPT + kk < vr) {
            mn = fminf(mn, m[kk]);
            mx = fmaxf(mx, m[kk]);
        }
#pragma unroll
    for (int o = 1; o < T; o <<= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (!active) return;
    const float sh = (a.shift && mn < INFINITY) ? mn : 0.f;
    const float bw = a.shift ? storage_scale<KT_t>(mx) : 1.f;

    KT_t *KT = reinterpret_cast<KT_t *>(a.KT);
    KT_t *KMT = reinterpret_cast<KT_t *>(a.KMT);
    const long base4 = (wi * VRP + sub * KPT) / 4;
#pragma unroll
    for (int c = 0; c < KPT / 4; ++c) {
        float kv[4], kmv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = sub * KPT + 4 * c + j;
            const float mm = m[4 * c + j];
            const float kk = (k < vr) ? expf(-lam * (mm - sh)) : 0.f;
            kv[j] = kk * bw;
            kmv[j] = (kk * mm) * bw;
        }
        KIO<KT_t>::store4(KT, base4 + c, make_float4(kv[0], kv[1], kv[2], kv[3]));
        KIO<KT_t>::store4(KMT, base4 + c, make_float4(kmv[0], kmv[1], kmv[2], kmv[3]));
    }
}

template <int KPT, int T, class KT_t>
__global__ void __launch_bounds__(kCostThreads) k_cost(const __grid_constant__ CostArgs a0, const CostArgs *batch) {
    // one query per grid row when batched (batch[blockIdx.y]), else the argument
    if (batch) k_cost_body<KPT, T, KT_t>(batch[blockIdx.y]);
    else k_cost_body<KPT, T, KT_t>(a0);
}

// Query blocks of up to 32 words: the whole transposed query block Q^T[d4][VRP]
// sits in shared memory (loaded once per persistent block).  TS adjacent threads
// own one word and take its embedding row's float4 chunks in turn (chunk i goes
// to thread i mod TS, so the TS threads read consecutive 16-byte pieces), with 4
// chunks per thread in flight (register double buffer); the main loop has no
// barrier.  The TS partial sums are combined with shuffles at the end.
// chunk >= 0: the query columns [32 chunk, 32 chunk + 32) of a wider layout of
// vrp_full columns (VRP = 32): the distances M are written to the rows' scratch
// (cost_scratch), to be turned into K and K.*M by k_cost_finish.
template <int VRP, int TS, class KT_t>
__device__ __noinline__ void k_cost_rows_body(const CostArgs &a, int chunk, int vrp_full) {
    static_assert(VRP % 4 == 0 && VRP <= 32, "VRP");
    static_assert(TS == 1 || TS == 2 || TS == 4, "TS");
    extern __shared__ __align__(16) float sQ[];   // sQ[dim * VRP + k] = E[q_k][dim], 0 for k >= v_r
    const int col0 = chunk >= 0 ? VRP * chunk : 0;
    const int vr = chunk >= 0 ? max(0, min(VRP, a.qp->vr - col0)) : a.qp->vr;
    const float lam = a.qp->lambda;
    const int d4 = a.d4;
    {
        // Q^T staged with float4 loads, query word fastest across threads (so the
        // transposed stores hit consecutive banks); the iterations are independent,
        // so their loads overlap instead of running one L2 round trip at a time
        const int n4q = d4 / 4;
#pragma unroll 4
        for (int i = threadIdx.x; i < n4q * VRP; i += kCostThreads) {
            const int c = i / VRP, k = i - c * VRP;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < vr) {
                const int qid = __ldg(a.q_ids + col0 + k);
                if (qid >= 0 && qid < a.V) v = __ldg(reinterpret_cast<const float4 *>(a.E + (size_t)qid * d4) + c);
            }
            sQ[(4 * c) * VRP + k] = v.x;
            sQ[(4 * c + 1) * VRP + k] = v.y;
            sQ[(4 * c + 2) * VRP + k] = v.z;
            sQ[(4 * c + 3) * VRP + k] = v.w;
        }
    }
    __syncthreads();
    // Two words per thread when one thread owns a word (TS = 1, large vocabularies):
    // each query value read from shared memory then serves both (the shared-memory
    // reads, not the FMAs, bounded the one-word form: 392 -> 332 us on 461,821 words).
    constexpr int W = TS == 1 ? 2 : 1;
    constexpr int PF = W == 1 ? 4 : 2;   // float4 chunks per word and thread in flight
    const int n4 = d4 / 4;
    const int t = threadIdx.x % TS;
    KT_t *KT = reinterpret_cast<KT_t *>(a.KT);
    KT_t *KMT = reinterpret_cast<KT_t *>(a.KMT);
    const long lanes_words = kCostThreads / TS;   // words per block and pass of one word per thread
    const long per_block = lanes_words * W;
    // every thread of a TS-group runs the same trip count (shuffles need the whole warp)
    for (long base = (long)blockIdx.x * per_block; base < a.Vu; base += (long)gridDim.x * per_block) {
        long wi[W];
        bool active[W];
        const float4 *row[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            wi[w] = base + threadIdx.x / TS + w * lanes_words;
            active[w] = wi[w] < a.Vu;
            row[w] = reinterpret_cast<const float4 *>(a.E + (size_t)(active[w] ? __ldg(a.used + wi[w]) : 0) * d4);
        }
        float2 acc[W][VRP / 2];
#pragma unroll
        for (int w = 0; w < W; ++w)
#pragma unroll
            for (int i = 0; i < VRP / 2; ++i) acc[w][i] = make_float2(0.f, 0.f);
        float4 buf[PF][W];
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int ch = j * TS + t;
#pragma unroll
            for (int w = 0; w < W; ++w) buf[j][w] = ch < n4 ? __ldg(row[w] + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int c0 = 0; c0 < n4; c0 += PF * TS) {
            float4 nxt[PF][W];
#pragma unroll
            for (int j = 0; j < PF; ++j) {
                const int ch = c0 + (PF + j) * TS + t;
#pragma unroll
                for (int w = 0; w < W; ++w) nxt[j][w] = ch < n4 ? __ldg(row[w] + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < PF; ++j) {
                const int ch = c0 + j * TS + t;
                if (ch < n4) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float2 e2[W];
#pragma unroll
                        for (int w = 0; w < W; ++w) {
                            const float ev = e == 0 ? buf[j][w].x : e == 1 ? buf[j][w].y : e == 2 ? buf[j][w].z : buf[j][w].w;
                            e2[w] = make_float2(ev, ev);
                        }
                        // query pairs read as float4: two register pairs, no repacking
                        const float4 *qrow = reinterpret_cast<const float4 *>(sQ + (4 * ch + e) * VRP);
#pragma unroll
                        for (int c = 0; c < VRP / 4; ++c) {
                            const float4 qv = qrow[c];
#pragma unroll
                            for (int w = 0; w < W; ++w) {
                                acc[w][2 * c] = sqdiff_acc2(make_float2(qv.x, qv.y), e2[w], acc[w][2 * c]);
                                acc[w][2 * c + 1] = sqdiff_acc2(make_float2(qv.z, qv.w), e2[w], acc[w][2 * c + 1]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < PF; ++j)
#pragma unroll
                for (int w = 0; w < W; ++w) buf[j][w] = nxt[j][w];
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
            float m[VRP];
#pragma unroll
            for (int i = 0; i < VRP / 2; ++i) {
                float x = acc[w][i].x, y = acc[w][i].y;
#pragma unroll
                for (int o = 1; o < TS; o <<= 1) {
                    x += __shfl_xor_sync(0xffffffffu, x, o);
                    y += __shfl_xor_sync(0xffffffffu, y, o);
                }
                m[2 * i] = sqrtf(x);
                m[2 * i + 1] = sqrtf(y);
            }
            if (!active[w]) continue;
            if (chunk >= 0) {
                // this chunk's distances into the row's scratch (columns >= v_r: not read)
#pragma unroll
                for (int c = 0; c < VRP / 4; ++c) {
                    if (c % TS != t) continue;
                    float *dst = cost_scratch(a, wi[w], col0 + 4 * c, vrp_full, (int)sizeof(KT_t));
                    *reinterpret_cast<float4 *>(dst) = make_float4(m[4 * c], m[4 * c + 1], m[4 * c + 2], m[4 * c + 3]);
                }
                continue;
            }
            float mn = INFINITY, mx = 0.f;
#pragma unroll
            for (int k = 0; k < VRP; ++k)
                if (k < vr) {
                    mn = fminf(mn, m[k]);
                    mx = fmaxf(mx, m[k]);
                }
            const float sh = (a.shift && mn < INFINITY) ? mn : 0.f;
            const float bw = a.shift ? storage_scale<KT_t>(mx) : 1.f;
#pragma unroll
            for (int c = 0; c < VRP / 4; ++c) {
                if (c % TS != t) continue;
                float kv[4], kmv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = 4 * c + j;
                    const float kk = (k < vr) ? expf(-lam * (m[k] - sh)) : 0.f;
                    kv[j] = kk * bw;
                    kmv[j] = (kk * m[k]) * bw;
                }
                KIO<KT_t>::store4(KT, wi[w] * (VRP / 4) + c, make_float4(kv[0], kv[1], kv[2], kv[3]));
                KIO<KT_t>::store4(KMT, wi[w] * (VRP / 4) + c, make_float4(kmv[0], kmv[1], kmv[2], kmv[3]));
            }
        }
    }
}

template <int VRP, int TS, class KT_t>
__global__ void __launch_bounds__(kCostThreads) k_cost_rows(const __grid_constant__ CostArgs a0, const CostArgs *batch,
                                                            int chunk, int vrp_full) {
    // one query per grid row when batched (batch[blockIdx.y]), else the argument
    if (batch) k_cost_rows_body<VRP, TS, KT_t>(batch[blockIdx.y], chunk, vrp_full);
    else k_cost_rows_body<VRP, TS, KT_t>(a0, chunk, vrp_full);
}

// K and K.*M of the rows whose distances the chunked row kernel left in the
// scratch: one warp per word, lane l takes columns l, l + 32, ...; the column's
// minimum (shift) and maximum (FP16 scale) over the query words first.
template <int VRP, class KT_t>
__device__ __noinline__ void k_cost_finish_body(const CostArgs &a) {
    constexpr int J = VRP / 32;
    const int vr = a.qp->vr;
    const float lam = a.qp->lambda;
    const int lane = threadIdx.x & 31;
    const long w0 = ((long)blockIdx.x * kCostThreads + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * kCostThreads) >> 5;
    KT_t *KT = reinterpret_cast<KT_t *>(a.KT);
    KT_t *KMT = reinterpret_cast<KT_t *>(a.KMT);
    for (long wi = w0; wi < a.Vu; wi += nw) {
        float m[J];
        float mn = INFINITY, mx = 0.f;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k = lane + 32 * j;
            m[j] = *cost_scratch(a, wi, k, VRP, (int)sizeof(KT_t));
            if (k < vr) {
                mn = fminf(mn, m[j]);
                mx = fmaxf(mx, m[j]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        const float sh = (a.shift && mn < INFINITY) ? mn : 0.f;
        const float bw = a.shift ? storage_scale<KT_t>(mx) : 1.f;
        __syncwarp();   // every lane has read the row's scratch before it is overwritten
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k = lane + 32 * j;
            const float kk = (k < vr) ? expf(-lam * (m[j] - sh)) : 0.f;
            KT[wi * VRP + k] = to_k<KT_t>(kk * bw);
            KMT[wi * VRP + k] = to_k<KT_t>((kk * m[j]) * bw);
        }
        __syncwarp();
    }
}

template <int VRP, class KT_t>
__global__ void __launch_bounds__(kCostThreads) k_cost_finish(const __grid_constant__ CostArgs a0, const CostArgs *batch) {
    if (batch) k_cost_finish_body<VRP, KT_t>(batch[blockIdx.y]);
    else k_cost_finish_body<VRP, KT_t>(a0);
}

// ---------------------------------------------------------------- the product form
//
// The same distances from M^2 = |q|^2 + |e|^2 - 2 q.e: the block is then a plain
// product E_used Q^T (one FMA per word, query word and dimension, half the direct
// form's two), register-tiled like a GEMM.  The product form cancels where M is
// small against |q| and |e| (a query word that is itself a corpus word has M = 0
// exactly, and the form leaves an O(1e-7) residue there, so M ~ 3e-4): every entry
// with M^2 below a quarter of |q|^2 + |e|^2 is evaluated again in the direct
// difference form.  The product form's rounding error is a few eps (|q|^2 + |e|^2)
// (2 |q.e| <= |q|^2 + |e|^2), so above that threshold it is a few eps relative to
// M^2, the same order as the direct form's.
//
// Tiles: a block of 4 warps owns 128 words (32 per warp); lane (wg = lane % 8,
// qg = lane / 8) of a warp holds the dots of its warp's words wg + 8 j (j < 4) with
// query words [qg KQ, qg KQ + KQ), KQ = VRP / 4, as packed f32x2 FMAs over query
// pairs.  The embedding rows go through shared memory 16 dimensions at a time
// (cp.async, three stages in flight, zero-filled past the vocabulary and past d);
// the transposed query block Q^T stays in shared memory.  Three blocks per SM
// (about 70 KB of shared memory and 136 registers a thread each at 32 columns) measured
// faster than two blocks of 4 warps with 8 words a thread or of 8 warps with 4.
constexpr int kTileDK = 16;              // embedding dimensions per stage
constexpr int kTileLd = kTileDK + 4;     // floats per word row of a stage: 8 consecutive rows of
                                         // float4 reads fall in distinct banks
constexpr int kTileStages = 3;           // stages in flight
constexpr int kTileCT = 128;             // threads per block
constexpr int kTileNW = 4;               // words per thread
constexpr int kTileMinB = 3;             // blocks per SM the registers are fitted to
constexpr int kTileWords = kTileCT / 32 * 8 * kTileNW;   // words per block tile: 8 NW per warp
constexpr size_t kCostTileSmemMax = 110 * 1024;          // largest dynamic shared memory taken

__host__ __device__ constexpr bool cost_tile_vrp(int vrp) { return vrp == 16 || vrp == 32 || vrp == 64; }
// Blocks per SM the registers are fitted to: 64-column layouts hold twice the dots
// and Q^T (about 107 KB of shared memory in all at d = 300), so two.
__host__ __device__ constexpr int cost_tile_min_blocks(int vrp) { return vrp >= 64 ? 2 : kTileMinB; }
// Partial sums of |q|^2 per query word (each over a share of the dimensions).
__host__ __device__ constexpr int cost_tile_qparts(int vrp) { return kTileCT / vrp < 4 ? kTileCT / vrp : 4; }

// Dynamic shared memory of the product-form kernel: the stages, Q^T over d4
// rounded up to whole stages, the tile's |e|^2, partial and whole |q|^2.
inline size_t cost_tile_smem(int d4, int vrp) {
    const size_t dq = (size_t)(d4 + kTileDK - 1) / kTileDK * kTileDK;
    return ((size_t)kTileStages * kTileWords * kTileLd + dq * vrp + kTileWords +
            (size_t)(cost_tile_qparts(vrp) + 1) * vrp) * sizeof(float);
}

// 16 bytes global -> shared on the asynchronous path (L2 only); valid = false
// copies nothing and writes zeros.  No memory clobber: the copies only target a
// stage buffer that every thread finished reading before the barrier preceding
// their issue, and the wait below (which has one) orders the reads after them.
__device__ __forceinline__ void cp_async16_zfill(float *smem, const float *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// sum_d (q_d - e_d)^2 over the d4 dimensions: query column k of the staged Q^T
// (row stride vrp) against an embedding row in global memory.
__device__ __noinline__ float direct_sq(const float *sQ, int vrp, int k, const float *erow, int d4) {
    float s = 0.f;
    for (int d = 0; d < d4; d += 4) {
        const float4 e = __ldg(reinterpret_cast<const float4 *>(erow + d));
        float t = sQ[d * vrp + k] - e.x;
        s = fmaf(t, t, s);
        t = sQ[(d + 1) * vrp + k] - e.y;
        s = fmaf(t, t, s);
        t = sQ[(d + 2) * vrp + k] - e.z;
        s = fmaf(t, t, s);
        t = sQ[(d + 3) * vrp + k] - e.w;
        s = fmaf(t, t, s);
    }
    return s;
}

// chunk >= 0: the query columns [VRP chunk, VRP chunk + VRP) of a wider layout of
// vrp_full columns; the distances go to the rows' scratch (cost_scratch), for
// k_cost_finish.
template <int VRP, class KT_t>
__device__ __noinline__ void k_cost_tile_body(const CostArgs &a, int chunk, int vrp_full) {
    static_assert(cost_tile_vrp(VRP), "VRP");
    constexpr int KQ = VRP / 4;                 // query words per thread
    constexpr int NW = kTileNW;                 // words per thread
    constexpr int CT = kTileCT;
    constexpr int TW = kTileWords;
    constexpr int CPT = TW * (kTileDK / 4) / CT;   // 16-byte copies per thread and stage
    constexpr int EPT = TW / CT;                   // |e|^2 sums per thread
    constexpr int QP = cost_tile_qparts(VRP);      // partial sums of |q_k|^2
    static_assert(CT % 32 == 0 && CT >= QP * VRP && QP >= 1 && CPT >= 1 && EPT >= 1, "tile shape");
    extern __shared__ __align__(16) float smem[];
    const int d4 = a.d4;
    const int dq = (d4 + kTileDK - 1) / kTileDK * kTileDK;
    float *const sE = smem;                                    // [stages][TW][kTileLd]
    float *const sQ = sE + kTileStages * TW * kTileLd;         // [dq][VRP]
    float *const sEn = sQ + dq * VRP;                          // [TW]
    float *const sQp = sEn + TW;                               // [QP][VRP]
    float *const sQn = sQp + QP * VRP;                         // [VRP]

    // the arguments in registers (the asynchronous-copy waits are compiler barriers)
    const float *const E = a.E;
    const int *const used = a.used;
    const long Vu = a.Vu;
    const int shift = a.shift;
    KT_t *const KT = reinterpret_cast<KT_t *>(a.KT);
    KT_t *const KMT = reinterpret_cast<KT_t *>(a.KMT);
    const int col0 = chunk >= 0 ? VRP * chunk : 0;
    const int vr = chunk >= 0 ? max(0, min(VRP, a.qp->vr - col0)) : a.qp->vr;
    const float lam = a.qp->lambda;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wg = lane & 7, qg = lane >> 3;

    const int ntiles = (int)((Vu + TW - 1) / TW);
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int ns = dq / kTileDK;
    const int total = my_tiles * ns;   // stages this block runs, tile-major

    // Stage g (tile g / ns of this block, dimensions [16 (g % ns), +16)) into buffer
    // g % 3: thread tid copies dimensions 4 (tid % 4) .. + 4 of words tid / 4 + (CT / 4) r.
    auto issue = [&](int g) {
        if (g < total) {
            const long tile = (long)blockIdx.x + (long)(g / ns) * gridDim.x;
            const int dim = (g % ns) * kTileDK + 4 * (tid & 3);
            float *dst = sE + (g % kTileStages) * (TW * kTileLd) + (tid >> 2) * kTileLd + 4 * (tid & 3);
            int row[CPT];   // all word ids first, so their loads are in flight together
#pragma unroll
            for (int r = 0; r < CPT; ++r) {
                const long wi = tile * TW + (tid >> 2) + (CT / 4) * r;
                row[r] = wi < Vu ? __ldg(used + wi) : -1;
            }
#pragma unroll
            for (int r = 0; r < CPT; ++r) {
                const bool ok = row[r] >= 0 && dim < d4;
                cp_async16_zfill(dst + (CT / 4) * r * kTileLd, ok ? E + (size_t)row[r] * d4 + dim : E, ok);
            }
        }
        cp_async_commit();
    };

    // Q^T, zero past v_r and past d4 (query word fastest across threads)
    for (int i = tid; i < (dq / 4) * VRP; i += CT) {
        const int c = i / VRP, k = i - c * VRP;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < vr && 4 * c < d4) {
            const int qid = __ldg(a.q_ids + col0 + k);
            if (qid >= 0 && qid < a.V) v = __ldg(reinterpret_cast<const float4 *>(E + (size_t)qid * d4) + c);
        }
        sQ[(4 * c) * VRP + k] = v.x;
        sQ[(4 * c + 1) * VRP + k] = v.y;
        sQ[(4 * c + 2) * VRP + k] = v.z;
        sQ[(4 * c + 3) * VRP + k] = v.w;
    }
    for (int g = 0; g < kTileStages - 1; ++g) issue(g);
    __syncthreads();
    // |q_k|^2: QP partial sums over equal shares of the dimensions, added in order
    {
        const int k = tid % VRP, p = tid / VRP, len = dq / QP;
        if (p < QP) {
            float sum = 0.f;
            for (int dd = p * len; dd < (p + 1) * len; ++dd) sum = fmaf(sQ[dd * VRP + k], sQ[dd * VRP + k], sum);
            sQp[p * VRP + k] = sum;
        }
    }
    __syncthreads();
    if (tid < VRP) {
        float sum = sQp[tid];
#pragma unroll
        for (int p = 1; p < QP; ++p) sum += sQp[p * VRP + tid];
        sQn[tid] = sum;
    }
    // (read after the main loop's first barrier)

    float2 acc[NW][KQ / 2];   // the dots of query pairs
#pragma unroll
    for (int j = 0; j < NW; ++j)
#pragma unroll
        for (int i = 0; i < KQ / 2; ++i) acc[j][i] = make_float2(0.f, 0.f);
    float en[EPT];   // |e|^2 of the tile's words tid + CT r
#pragma unroll
    for (int r = 0; r < EPT; ++r) en[r] = 0.f;

    for (int g = 0; g < total; ++g) {
        cp_async_wait<kTileStages - 2>();   // this thread's copies of stage g have landed
        __syncthreads();                    // everyone's; the buffer of stage g - 1 is free
        issue(g + kTileStages - 1);
        const int s = g % ns;
        const float *buf = sE + (g % kTileStages) * (TW * kTileLd);
        const float *qs = sQ + s * kTileDK * VRP + qg * KQ;
        const float *wrow = buf + (warp * 8 * NW + wg) * kTileLd;
#pragma unroll
        for (int quad = 0; quad < kTileDK / 4; ++quad) {
            float4 ev[NW];
#pragma unroll
            for (int j = 0; j < NW; ++j) ev[j] = *reinterpret_cast<const float4 *>(wrow + 8 * j * kTileLd + 4 * quad);
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) {
                float qv[KQ];
#pragma unroll
                for (int c = 0; c < KQ / 4; ++c) {
                    const float4 q4 = *reinterpret_cast<const float4 *>(qs + (4 * quad + dd) * VRP + 4 * c);
                    qv[4 * c] = q4.x;
                    qv[4 * c + 1] = q4.y;
                    qv[4 * c + 2] = q4.z;
                    qv[4 * c + 3] = q4.w;
                }
#pragma unroll
                for (int j = 0; j < NW; ++j) {
                    const float e = dd == 0 ? ev[j].x : dd == 1 ? ev[j].y : dd == 2 ? ev[j].z : ev[j].w;
                    const float2 e2 = make_float2(e, e);
#pragma unroll
                    for (int i = 0; i < KQ / 2; ++i)
                        acc[j][i] = __ffma2_rn(make_float2(qv[2 * i], qv[2 * i + 1]), e2, acc[j][i]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < EPT; ++r)
#pragma unroll
            for (int c = 0; c < kTileDK / 4; ++c) {
                const float4 x = *reinterpret_cast<const float4 *>(buf + (tid + CT * r) * kTileLd + 4 * c);
                en[r] = fmaf(x.x, x.x, en[r]);
                en[r] = fmaf(x.y, x.y, en[r]);
                en[r] = fmaf(x.z, x.z, en[r]);
                en[r] = fmaf(x.w, x.w, en[r]);
            }
        if (s != ns - 1) continue;

        // the tile is complete: distances, then K and K.*M (or the chunk's scratch)
#pragma unroll
        for (int r = 0; r < EPT; ++r) {
            sEn[tid + CT * r] = en[r];
            en[r] = 0.f;
        }
        __syncthreads();
        const long tile = (long)blockIdx.x + (long)(g / ns) * gridDim.x;
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            const int wl = warp * 8 * NW + wg + 8 * j;
            const long wi = tile * TW + wl;
            const bool active = wi < Vu;
            const float enw = sEn[wl];
            float m[KQ];
#pragma unroll
            for (int i = 0; i < KQ; ++i) {
                const int k = qg * KQ + i;
                const float dot = (i & 1) ? acc[j][i / 2].y : acc[j][i / 2].x;
                const float nn = sQn[k] + enw;
                float d2 = fmaf(-2.f, dot, nn);
                if (active && !(d2 >= 0.25f * nn)) d2 = direct_sq(sQ, VRP, k, E + (size_t)__ldg(used + wi) * d4, d4);
                m[i] = sqrtf(fmaxf(d2, 0.f));
            }
#pragma unroll
            for (int i = 0; i < KQ / 2; ++i) acc[j][i] = make_float2(0.f, 0.f);
            if (chunk >= 0) {
                if (active)
#pragma unroll
                    for (int c = 0; c < KQ / 4; ++c) {
                        float *dst = cost_scratch(a, wi, col0 + qg * KQ + 4 * c, vrp_full, (int)sizeof(KT_t));
                        *reinterpret_cast<float4 *>(dst) = make_float4(m[4 * c], m[4 * c + 1], m[4 * c + 2], m[4 * c + 3]);
                    }
                continue;
            }
            // column shift (minimum over the query words) and FP16 scale (maximum): the
            // word's columns are spread over the lanes wg, wg + 8, wg + 16, wg + 24
            float mn = INFINITY, mx = 0.f;
#pragma unroll
            for (int i = 0; i < KQ; ++i)
                if (qg * KQ + i < vr) {
                    mn = fminf(mn, m[i]);
                    mx = fmaxf(mx, m[i]);
                }
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, 8));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, 16));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
            if (!active) continue;
            const float sh = (shift && mn < INFINITY) ? mn : 0.f;
            const float bw = shift ? storage_scale<KT_t>(mx) : 1.f;
#pragma unroll
            for (int c = 0; c < KQ / 4; ++c) {
                float kv[4], kmv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = qg * KQ + 4 * c + e;
                    const float kk = (k < vr) ? expf(-lam * (m[4 * c + e] - sh)) : 0.f;
                    kv[e] = kk * bw;
                    kmv[e] = (kk * m[4 * c + e]) * bw;
                }
                const long idx4 = (wi * VRP + qg * KQ) / 4 + c;
                KIO<KT_t>::store4(KT, idx4, make_float4(kv[0], kv[1], kv[2], kv[3]));
                KIO<KT_t>::store4(KMT, idx4, make_float4(kmv[0], kmv[1], kmv[2], kmv[3]));
            }
        }
    }
    cp_async_wait<0>();   // (the groups still open are empty)
}

template <int VRP, class KT_t>
__global__ void __launch_bounds__(kTileCT, cost_tile_min_blocks(VRP)) k_cost_tile(const __grid_constant__ CostArgs a0,
                                                                  const CostArgs *batch, int chunk, int vrp_full) {
    // one query per grid row when batched (batch[blockIdx.y]), else the argument
    if (batch) k_cost_tile_body<VRP, KT_t>(batch[blockIdx.y], chunk, vrp_full);
    else k_cost_tile_body<VRP, KT_t>(a0, chunk, vrp_full);
}

// Blocks: one per tile of words, at most the resident blocks of the device shared
// by the nq queries of a batch.
template <int VRP, class KT_t>
cudaError_t run_tile(const CostArgs &a, cudaStream_t s, int nq, const CostArgs *batch, int chunk = -1,
                     int vrp_full = 0) {
    auto kern = k_cost_tile<VRP, KT_t>;
    const size_t smem = cost_tile_smem(a.d4, VRP);
    static LaunchCache cache;
    int per_sm = 1;
    cudaError_t e = cache.blocks_per_sm(kern, kTileCT, smem, -1, &per_sm);
    if (e != cudaSuccess) return e;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long blocks = (a.Vu + kTileWords - 1) / kTileWords;
    long cap = ((long)sms * per_sm + nq - 1) / nq;
    if (cap < 1) cap = 1;
    if (blocks > cap) blocks = cap;
    if (blocks > 0) kern<<<dim3((unsigned)blocks, (unsigned)nq), kTileCT, smem, s>>>(a, batch, chunk, vrp_full);
    return cudaGetLastError();
}

template <int VRP, int TS, class KT_t>
cudaError_t run_rows(const CostArgs &a, cudaStream_t s, int nq, const CostArgs *batch, int chunk = -1,
                     int vrp_full = 0) {
    auto kern = k_cost_rows<VRP, TS, KT_t>;
    const size_t smem = (size_t)a.d4 * VRP * sizeof(float);
    static LaunchCache cache;
    int per_sm = 1;
    cudaError_t e = cache.blocks_per_sm(kern, kCostThreads, smem, -1, &per_sm);
    if (e != cudaSuccess) return e;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long per_block = kCostThreads / TS;
    long blocks = (a.Vu + per_block - 1) / per_block;
    long cap = ((long)sms * per_sm + nq - 1) / nq;   // resident blocks shared by the queries
    if (cap < 1) cap = 1;
    if (blocks > cap) blocks = cap;
    if (blocks > 0) kern<<<dim3((unsigned)blocks, (unsigned)nq), kCostThreads, smem, s>>>(a, batch, chunk, vrp_full);
    return cudaGetLastError();
}

// A layout wider than 32 columns: the row kernel on each 32-column chunk (distances
// to the scratch), then the finishing pass over whole rows.
template <int VRP, class KT_t>
cudaError_t run_finish(const CostArgs &a, cudaStream_t s, int nq, const CostArgs *batch) {
    auto kern = k_cost_finish<VRP, KT_t>;
    static LaunchCache cache;
    int per_sm = 1;
    cudaError_t e = cache.blocks_per_sm(kern, kCostThreads, 0, -1, &per_sm);
    if (e != cudaSuccess) return e;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long blocks = ((long)a.Vu * 32 + kCostThreads - 1) / kCostThreads;
    long cap = ((long)sms * per_sm + nq - 1) / nq;
    if (cap < 1) cap = 1;
    if (blocks > cap) blocks = cap;
    if (blocks > 0) kern<<<dim3((unsigned)blocks, (unsigned)nq), kCostThreads, 0, s>>>(a, batch);
    return cudaGetLastError();
}

template <int VRP, class KT_t>
cudaError_t run_chunked(const CostArgs &a, cudaStream_t s, int nq, const CostArgs *batch, int ts) {
    if (ts == 0 && VRP % 64 == 0 && cost_tile_smem(a.d4, 64) <= kCostTileSmemMax) {
        for (int ch = 0; ch < VRP / 64; ++ch) {   // 64-column chunks of the product form
            cudaError_t e = run_tile<64, KT_t>(a, s, nq, batch, ch, VRP);
            if (e != cudaSuccess) return e;
        }
        return run_finish<VRP, KT_t>(a, s, nq, batch);
    }
    for (int ch = 0; ch < VRP / 32; ++ch) {
        cudaError_t e = ts == 0 ? run_tile<32, KT_t>(a, s, nq, batch, ch, VRP)
                      : ts == 2 ? run_rows<32, 2, KT_t>(a, s, nq, batch, ch, VRP)
                      : ts == 4 ? run_rows<32, 4, KT_t>(a, s, nq, batch, ch, VRP)
                                : run_rows<32, 1, KT_t>(a, s, nq, batch, ch, VRP);
        if (e != cudaSuccess) return e;
    }
    return run_finish<VRP, KT_t>(a, s, nq, batch);
}

template <int KPT, int T, class KT_t>
cudaError_t run(const CostArgs &a, cudaStream_t s, int nq, const CostArgs *batch) {
    const int words_per_block = kCostThreads / T;
    const long blocks = (a.Vu + words_per_block - 1) / words_per_block;
    if (blocks > 0)
        k_cost<KPT, T, KT_t><<<dim3((unsigned)blocks, (unsigned)nq), kCostThreads, 0, s>>>(a, batch);
    return cudaGetLastError();
}

// The product-form kernel where it applies (layouts of 16, 32 and 64 columns, and
// the 64- or 32-column chunks of 128, within about 110 KB of shared memory) unless a
// cost split asks for the row kernel.

template <class KT_t>
cudaError_t dispatch(const CostArgs &a, int vrp, cudaStream_t s, int nq, const CostArgs *batch) {
    const bool rows_asked = a.split == 1 || a.split == 2 || a.split == 4;
    if (!rows_asked && cost_tile_vrp(vrp) && cost_tile_smem(a.d4, vrp) <= kCostTileSmemMax)
        return vrp == 16 ? run_tile<16, KT_t>(a, s, nq, batch)
             : vrp == 32 ? run_tile<32, KT_t>(a, s, nq, batch)
                         : run_tile<64, KT_t>(a, s, nq, batch);
    if (!rows_asked && (vrp == 64 || vrp == 128) && cost_tile_smem(a.d4, 32) <= kCostTileSmemMax)
        return vrp == 64 ? run_chunked<64, KT_t>(a, s, nq, batch, 0) : run_chunked<128, KT_t>(a, s, nq, batch, 0);
    if (vrp <= 32 && (size_t)a.d4 * vrp * sizeof(float) <= 100 * 1024) {
        // threads per word: 2 by default; 1 on large vocabularies, where one thread
        // per word already fills the GPU (measured 1.3-1.5x faster from 90,000 used
        // words up)
        const int ts = a.split == 1 || a.split == 2 || a.split == 4 ? a.split : (a.Vu >= 64 * 1024 ? 1 : 2);
        switch (vrp * 10 + ts) {
#define SWMD_ROWS(V)                                      \
    case V * 10 + 1: return run_rows<V, 1, KT_t>(a, s, nq, batch); \
    case V * 10 + 2: return run_rows<V, 2, KT_t>(a, s, nq, batch); \
    case V * 10 + 4: return run_rows<V, 4, KT_t>(a, s, nq, batch);
            SWMD_ROWS(4) SWMD_ROWS(8) SWMD_ROWS(12) SWMD_ROWS(16) SWMD_ROWS(20) SWMD_ROWS(24)
            SWMD_ROWS(28) SWMD_ROWS(32)
#undef SWMD_ROWS
            default: break;
        }
    }
    if ((vrp == 64 || vrp == 128) && (size_t)a.d4 * 32 * sizeof(float) <= 100 * 1024) {
        const int ts = a.split == 1 || a.split == 2 || a.split == 4 ? a.split : (a.Vu >= 64 * 1024 ? 1 : 2);
        return vrp == 64 ? run_chunked<64, KT_t>(a, s, nq, batch, ts) : run_chunked<128, KT_t>(a, s, nq, batch, ts);
    }
    switch (vrp) {
#define SWMD_COST_T1(V) \
    case V: return run<V, 1, KT_t>(a, s, nq, batch);
        SWMD_COST_T1(4) SWMD_COST_T1(8) SWMD_COST_T1(12) SWMD_COST_T1(16)
        SWMD_COST_T1(20) SWMD_COST_T1(24) SWMD_COST_T1(28) SWMD_COST_T1(32)
#undef SWMD_COST_T1
        case 40: return run<20, 2, KT_t>(a, s, nq, batch);
        case 48: return run<24, 2, KT_t>(a, s, nq, batch);
        case 56: return run<28, 2, KT_t>(a, s, nq, batch);
        case 64: return run<32, 2, KT_t>(a, s, nq, batch);
        case 80: return run<20, 4, KT_t>(a, s, nq, batch);
        case 96: return run<24, 4, KT_t>(a, s, nq, batch);
        case 112: return run<28, 4, KT_t>(a, s, nq, batch);
        case 128: return run<32, 4, KT_t>(a, s, nq, batch);
        default: return cudaErrorInvalidValue;
    }
}

// One block: parameter block, then the zero-padded query arrays.  Ids outside
// [0, V) and weights that are not finite and positive raise status bits; the
// cost kernel reads such ids as zero rows, so nothing is accessed out of range.
__global__ void k_prep(QParams *qp, float lambda, int vr, int V, const int *src_ids,
                       const float *src_r, int *q_ids, float *r, int vrp_cap, double *out,
                       int *status) {
    if (threadIdx.x == 0) {
        QParams p;
        p.lambda = lambda;
        p.vr = vr;
        p.u0 = (float)vr;
        p.pad = 0;
        p.out = out;
        p.status = status;
        *qp = p;
        *status = 0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < vrp_cap; k += blockDim.x) {
        if (src_ids) {
            int id = 0;
            if (k < vr) {
                id = src_ids[k];
                if (id < 0 || id >= V) atomicOr(status, ST_BAD_ID);
            }
            q_ids[k] = id;
        }
        if (src_r) {
            float w = 0.f;
            if (k < vr) {
                w = src_r[k];
                if (!(w > 0.f) || !(w < INFINITY)) atomicOr(status, ST_BAD_R);
            }
            r[k] = w;
        }
    }
}

// One block per query of a batch: the same work as k_prep for query blockIdx.x.
__global__ void k_prep_batch(const PrepArgs *args, int V) {
    const PrepArgs p = args[blockIdx.x];
    if (threadIdx.x == 0) {
        QParams q;
        q.lambda = p.lambda;
        q.vr = p.vr;
        q.u0 = (float)p.vr;
        q.pad = 0;
        q.out = p.out;
        q.status = p.status;
        *p.qp = q;
        *p.status = 0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < p.vrp_cap; k += blockDim.x) {
        int id = 0;
        float w = 0.f;
        if (k < p.vr) {
            id = p.src_ids[k];
            w = p.src_r[k];
            if (id < 0 || id >= V) atomicOr(p.status, ST_BAD_ID);
            if (!(w > 0.f) || !(w < INFINITY)) atomicOr(p.status, ST_BAD_R);
        }
        p.q_ids[k] = id;
        p.r[k] = w;
    }
}

}  // namespace

cudaError_t launch_prep_batch(const PrepArgs *d_args, int nq, int V, cudaStream_t s) {
    if (nq > 0) k_prep_batch<<<nq, 128, 0, s>>>(d_args, V);
    return cudaGetLastError();
}

cudaError_t launch_prep(QParams *qp, float lambda, int vr, int V, const int *src_ids,
                        const float *src_r, int *q_ids, float *r, int vrp_cap, double *out,
                        int *status, cudaStream_t s) {
    k_prep<<<1, 256, 0, s>>>(qp, lambda, vr, V, src_ids, src_r, q_ids, r, vrp_cap, out, status);
    return cudaGetLastError();
}

cudaError_t launch_cost(const CostArgs &a, int vrp, int kprec, cudaStream_t s) {
    return launch_cost_batch(a, vrp, kprec, 1, nullptr, s);
}

cudaError_t launch_cost_batch(const CostArgs &shape, int vrp, int kprec, int nq,
                              const CostArgs *d_batch, cudaStream_t s) {
    switch (kprec) {
        case 0: return dispatch<float>(shape, vrp, s, nq, d_batch);
        case 1: return dispatch<__nv_bfloat16>(shape, vrp, s, nq, d_batch);
        case 2: return dispatch<__half>(shape, vrp, s, nq, d_batch);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swmd
