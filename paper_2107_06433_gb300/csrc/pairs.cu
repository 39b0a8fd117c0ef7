// 1-to-1 Sinkhorn WMD: the distance of each of many independent (query, target)
// histogram pairs, with the cost matrix built over the target's own v_x words
// only (Section III-E, Table II, right column: O(v_x v_r w + t v_x v_r) per pair
// instead of the 1-to-N path's O(V v_r w + t nnz v_r)).  Algorithm 1 on a single
// column c: a vocabulary word outside the target has c = 0, so it adds nothing to
// x = K_over_r v or to the final sum, and dropping it is exact.
//
// One block of 256 threads (8 warps) owns one pair at a time (a grid-stride loop over
// pairs) and runs every step of Algorithm 1 for it on chip:
//   cost   M[k][j] = ||E[q_k] - E[x_j]||_2 for the v_r x v_x block, tiled 4 KPT query
//          words x 64 target words (four warp rows of KPT query words, two warp columns
//          of 32 target words), embedding dimensions staged 32 at a time in shared
//          memory, the next chunk already in flight in registers while the current one
//          is used (FP32, direct difference form, two-wide FMAs);
//          K = exp(-lambda (M - m_j)) with the column shift m_j = min_k M[k][j]
//          when the corpus uses it (an exact rescaling of column j), KM = K .* M;
//          K and KM stay in shared memory when they fit, else in a per-block
//          region of global memory that L1 holds;
//   iterate v_j = c_j / (K^T u)_j (SDDMM, one thread per target word, the FP64
//          guard below 2^-100 as on the 1-to-N path), y = K v (SpMM, one warp per
//          query word, lanes over target words, a fixed-order shuffle sum), u = r / y
//          -- t times, or until max_k |u_k y_k - r_k| < tol;
//   final  WMD = sum_j c_j (KM^T u)_j / (K^T u)_j, summed in FP64 in a fixed order.
// K and KM are kept as [target word j][query word k] with an odd row stride, so the
// SDDMM's lanes (over j) and the SpMM's lanes (over k) both read distinct banks.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "corpus.h"

namespace swmd {
namespace {

constexpr int kPT = 256;   // threads per block
constexpr int kPW = kPT / 32;   // warps per block
constexpr int kPJ = 64;    // target words per cost tile (two per lane)
constexpr int kPD = 32;    // embedding dimensions per staged chunk
// K and KM of the largest pair go to shared memory up to this many bytes
constexpr size_t kPairSmemK = 48 * 1024;
// the global K / KM regions of one launch stay under this many bytes
constexpr size_t kPairKwsMax = size_t(2) << 30;

struct PairArgs {
    const float *E;
    int d4;
    int V;
    PairJob job;
    float *kws;       // global K / KM regions (not used when they live in shared memory)
    long kws_stride;  // floats per block region
    int shift;
};

// Byte offsets of the shared-memory arrays (host and device agree on them).
struct PairLayout {
    int u, rr, red, v, cw, sq, sx, k;
    int kelems;   // floats of one of K / KM: row stride (max_q + 1) x max_x
    int bytes;
};

__host__ __device__ inline int take_floats(int &off, int floats) {
    const int o = off;
    off += ((floats + 3) & ~3) * 4;   // 16-byte aligned arrays
    return o;
}

__host__ __device__ inline PairLayout pair_layout(int max_q, int max_x, int tkk, bool smemk) {
    PairLayout L;
    int off = 128;   // kPW doubles of the final sum, kPW floats of the marginal error, a flag word
    L.u = take_floats(off, max_q);
    L.rr = take_floats(off, max_q);
    L.red = take_floats(off, max_q);
    L.v = take_floats(off, max_x);
    L.cw = take_floats(off, max_x);
    L.sq = take_floats(off, kPD * tkk);
    L.sx = take_floats(off, kPJ * (kPD + 1));
    L.kelems = (max_q + 1) * max_x;
    L.k = smemk ? take_floats(off, 2 * L.kelems) : 0;
    L.bytes = off;
    return L;
}

__device__ __forceinline__ float2 sqdiff2(float2 q, float x, float2 acc) {
    const float2 t = __ffma2_rn(make_float2(x, x), make_float2(-1.f, -1.f), q);
    return __ffma2_rn(t, t, acc);
}

// One d-chunk of the cost tile: kPJ target rows and TKK query rows, kPD dimensions,
// as float4s per thread (rows of 8 float4, consecutive threads along a row).
constexpr int kPX4 = kPJ * (kPD / 4) / kPT;   // float4s of target rows per thread
template <int TKK>
struct Chunk {
    static constexpr int NQ = (TKK * (kPD / 4) + kPT - 1) / kPT;
    float4 x[kPX4];
    float4 q[NQ];
};

template <int TKK>
__device__ __forceinline__ void load_chunk(Chunk<TKK> &c, const float *E, int d4, int d0,
                                           const int *xid, int jt, int vx, const int *qid, int kt,
                                           int vr, int tid) {
    const int dl = min(kPD, d4 - d0);   // a multiple of 4
#pragma unroll
    for (int i = 0; i < kPX4; ++i) {
        const int e = tid + i * kPT, row = e / (kPD / 4), seg = e % (kPD / 4);
        c.x[i] = (jt + row < vx && 4 * seg < dl)
                     ? __ldg(reinterpret_cast<const float4 *>(E + (long)xid[jt + row] * d4 + d0 + 4 * seg))
                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < Chunk<TKK>::NQ; ++i) {
        const int e = tid + i * kPT, row = e / (kPD / 4), seg = e % (kPD / 4);
        c.q[i] = (e < TKK * (kPD / 4) && kt + row < vr && 4 * seg < dl)
                     ? __ldg(reinterpret_cast<const float4 *>(E + (long)qid[kt + row] * d4 + d0 + 4 * seg))
                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Sx [kPJ][kPD + 1] (dimension fastest), Sq [kPD][TKK] (query word fastest)
template <int TKK>
__device__ __forceinline__ void store_chunk(const Chunk<TKK> &c, float *Sx, float *Sq, int tid) {
#pragma unroll
    for (int i = 0; i < kPX4; ++i) {
        const int e = tid + i * kPT, row = e / (kPD / 4), seg = e % (kPD / 4);
        float *dst = Sx + row * (kPD + 1) + 4 * seg;
        dst[0] = c.x[i].x; dst[1] = c.x[i].y; dst[2] = c.x[i].z; dst[3] = c.x[i].w;
    }
#pragma unroll
    for (int i = 0; i < Chunk<TKK>::NQ; ++i) {
        const int e = tid + i * kPT, row = e / (kPD / 4), seg = e % (kPD / 4);
        if (e < TKK * (kPD / 4)) {
            float *dst = Sq + (4 * seg) * TKK + row;
            dst[0] = c.q[i].x; dst[TKK] = c.q[i].y; dst[2 * TKK] = c.q[i].z; dst[3 * TKK] = c.q[i].w;
        }
    }
}

// K^T[j] . u over the pair's query words: two interleaved partial sums (even and odd
// k), added at the end -- a fixed order for every pair.
__device__ __forceinline__ float dot_ku(const float *kr, const float *u, int vr) {
    float s0 = 0.f, s1 = 0.f;
    int k = 0;
    for (; k + 1 < vr; k += 2) {
        s0 = fmaf(kr[k], u[k], s0);
        s1 = fmaf(kr[k + 1], u[k + 1], s1);
    }
    if (k < vr) s0 = fmaf(kr[k], u[k], s0);
    return s0 + s1;
}

__device__ __forceinline__ float warp_min(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

template <int KPT, bool SMEMK>
__global__ void __launch_bounds__(kPT, 2) k_pairs(const __grid_constant__ PairArgs a) {
    constexpr int TKK = 4 * KPT;   // query words per cost tile: KPT per warp row
    extern __shared__ __align__(16) unsigned char smem[];
    const PairJob &J = a.job;
    const PairLayout L = pair_layout(J.max_q, J.max_x, TKK, SMEMK);
    double *dred = reinterpret_cast<double *>(smem);
    float *errw = reinterpret_cast<float *>(smem + 8 * kPW);
    int *flag = reinterpret_cast<int *>(smem + 12 * kPW);
    float *u = reinterpret_cast<float *>(smem + L.u);
    float *rr = reinterpret_cast<float *>(smem + L.rr);
    float *red = reinterpret_cast<float *>(smem + L.red);
    float *v = reinterpret_cast<float *>(smem + L.v);
    float *cw = reinterpret_cast<float *>(smem + L.cw);
    float *Sq = reinterpret_cast<float *>(smem + L.sq);   // [kPD][TKK], query word fastest
    float *Sx = reinterpret_cast<float *>(smem + L.sx);   // [kPJ][kPD + 1]
    float *Kb, *KMb;
    if constexpr (SMEMK) {
        Kb = reinterpret_cast<float *>(smem + L.k);
        KMb = Kb + L.kelems;
    } else {
        Kb = a.kws + (long)blockIdx.x * a.kws_stride;
        KMb = Kb + a.kws_stride / 2;
    }
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int kg = w & 3, jh = w >> 2;   // cost tile: warp row (query words), warp column (target words)
    const float lam = J.lambda;

    for (int p = blockIdx.x; p < J.n_pairs; p += gridDim.x) {
        const int64_t q0 = J.q_ptr[p], x0 = J.x_ptr[p];
        const int64_t nq = J.q_ptr[p + 1] - q0, nx = J.x_ptr[p + 1] - x0;
        if (tid == 0) *flag = 0;
        __syncthreads();
        // sizes, ids and weights (u = v_r: x starts at 1 / v_r, Algorithm 1)
        if (nq < 1 || nq > J.max_q || nx < 1 || nx > J.max_x) {
            if (tid == 0) *flag = ST_BAD_SIZE;
        } else {
            int bad = 0;
            for (int k = tid; k < (int)nq; k += kPT) {
                const int id = J.q_ids[q0 + k];
                const float rk = J.r[q0 + k];
                bad |= (id < 0 || id >= a.V) ? ST_BAD_ID : 0;
                bad |= (rk > 0.f && rk <= FLT_MAX) ? 0 : ST_BAD_R;
                u[k] = (float)nq;
                rr[k] = rk;
            }
            for (int j = tid; j < (int)nx; j += kPT) {
                const int id = J.x_ids[x0 + j];
                const float cj = J.cx[x0 + j];
                bad |= (id < 0 || id >= a.V) ? ST_BAD_ID : 0;
                bad |= (cj > 0.f && cj <= FLT_MAX) ? 0 : ST_BAD_R;
                cw[j] = cj;
            }
            if (bad) atomicOr(flag, bad);
        }
        __syncthreads();
        const int fl = *flag;
        if (fl) {
            if (tid == 0) {
                J.out[p] = __longlong_as_double(0x7ff8000000000000ll);
                if (J.iters) J.iters[p] = 0;
                atomicOr(J.status, fl);
            }
            __syncthreads();
            continue;
        }
        const int vr = (int)nq, vx = (int)nx;
        const int VRS = vr | 1;   // odd row stride of K / KM
        const int *qid = J.q_ids + q0;
        const int *xid = J.x_ids + x0;

        // ---- cost: M for the v_r x v_x block, written to KMb first
        for (int jt = 0; jt < vx; jt += kPJ) {
            for (int kt = 0; kt < vr; kt += TKK) {
                float2 acc[KPT / 2];   // target word jt + 32 jh + lane, query words kt + kg KPT + ...
#pragma unroll
                for (int i = 0; i < KPT / 2; ++i) acc[i] = make_float2(0.f, 0.f);
                const bool busy = jt + 32 * jh < vx;   // warp-uniform: this warp column has words
                Chunk<TKK> ch;
                load_chunk<TKK>(ch, a.E, a.d4, 0, xid, jt, vx, qid, kt, vr, tid);
                for (int d0 = 0; d0 < a.d4; d0 += kPD) {
                    const int dl = min(kPD, a.d4 - d0);
                    __syncthreads();   // the previous chunk's readers are done
                    store_chunk<TKK>(ch, Sx, Sq, tid);
                    __syncthreads();
                    if (d0 + kPD < a.d4)   // the next chunk is in flight during this one's FMAs
                        load_chunk<TKK>(ch, a.E, a.d4, d0 + kPD, xid, jt, vx, qid, kt, vr, tid);
                    if (busy) {
                        const float *sx = Sx + (32 * jh + lane) * (kPD + 1);
                        const float *sq = Sq + kg * KPT;
#pragma unroll 4
                        for (int dd = 0; dd < dl; ++dd) {
                            const float e0 = sx[dd];
#pragma unroll
                            for (int i = 0; i < KPT / 2; ++i)
                                acc[i] = sqdiff2(*reinterpret_cast<const float2 *>(sq + dd * TKK + 2 * i), e0,
                                                 acc[i]);
                        }
                    }
                }
                const int j = jt + 32 * jh + lane;
                if (j < vx) {
#pragma unroll
                    for (int i = 0; i < KPT / 2; ++i) {
                        const int k = kt + kg * KPT + 2 * i;
                        if (k < vr) KMb[j * VRS + k] = sqrtf(acc[i].x);
                        if (k + 1 < vr) KMb[j * VRS + k + 1] = sqrtf(acc[i].y);
                    }
                }
            }
        }
        __syncthreads();
        // K = exp(-lambda (M - m_j)), KM = K .* M: one warp per target word
        for (int j = w; j < vx; j += kPT / 32) {
            float mn = INFINITY;
            for (int k = lane; k < vr; k += 32) mn = fminf(mn, KMb[j * VRS + k]);
            mn = warp_min(mn);
            const float sh = (a.shift && mn < INFINITY) ? mn : 0.f;
            for (int k = lane; k < vr; k += 32) {
                const float m = KMb[j * VRS + k];
                const float kk = expf(-lam * (m - sh));
                Kb[j * VRS + k] = kk;
                KMb[j * VRS + k] = kk * m;
            }
        }
        __syncthreads();

        // ---- iterations
        const bool conv = J.tol > 0.f;
        int it = 0;
        for (;;) {
            if (!conv && it == J.t) break;
            // SDDMM: v_j = c_j / (K^T u)_j
            for (int j = tid; j < vx; j += kPT) {
                const float *kr = Kb + j * VRS;
                const float s = dot_ku(kr, u, vr);
                float vj;
                if (s >= 0x1p-100f) {
                    vj = __fdividef(cw[j], s);
                } else {
                    double sd = 0.0;
                    for (int k = 0; k < vr; ++k) sd += (double)kr[k] * (double)u[k];
                    vj = sd > 0.0 ? (float)((double)cw[j] / sd) : 0.f;
                    atomicOr(J.status, sd > 0.0 ? ST_GUARD : ST_NUMERIC);
                }
                v[j] = vj;
            }
            __syncthreads();
            // SpMM y_k = sum_j K[k, j] v_j, one warp per query word; then x = K_over_r v,
            // u = 1 / x, i.e. u_k = r_k / y_k -- at once, or after the stopping test
            float errl = 0.f;
            for (int k = w; k < vr; k += kPT / 32) {
                float part = 0.f;
                for (int j = lane; j < vx; j += 32) part = fmaf(Kb[j * VRS + k], v[j], part);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                if (conv) {
                    const float e = fabsf(u[k] * part - rr[k]);
                    errl = fmaxf(errl, e <= FLT_MAX ? e : INFINITY);
                    if (lane == 0) red[k] = part;
                } else if (lane == 0) {
                    const float nu = __fdividef(rr[k], part);
                    if (!(nu < INFINITY)) atomicOr(J.status, ST_NUMERIC);
                    u[k] = nu;
                }
            }
            if (conv) {
                // "while x changes" (Algorithm 1): stop once the row marginal of
                // P = diag(u) K diag(v) is within tol of r, or after t updates
                if (lane == 0) errw[w] = errl;
                __syncthreads();
                float err = errw[0];
#pragma unroll
                for (int i = 1; i < kPW; ++i) err = fmaxf(err, errw[i]);
                if (err < J.tol || it == J.t) break;
                for (int k = tid; k < vr; k += kPT) {
                    const float nu = __fdividef(rr[k], red[k]);
                    if (!(nu < INFINITY)) atomicOr(J.status, ST_NUMERIC);
                    u[k] = nu;
                }
            }
            ++it;
            __syncthreads();
        }

        // ---- final: WMD = sum_j c_j (KM^T u)_j / (K^T u)_j
        double dsum = 0.0;
        for (int j = tid; j < vx; j += kPT) {
            const float *kr = Kb + j * VRS;
            const float *mr = KMb + j * VRS;
            const float s = dot_ku(kr, u, vr), sm = dot_ku(mr, u, vr);
            if (s >= 0x1p-100f) {
                dsum += (double)(cw[j] * __fdividef(sm, s));
            } else {
                double sd = 0.0, md = 0.0;
                for (int k = 0; k < vr; ++k) {
                    sd += (double)kr[k] * (double)u[k];
                    md += (double)mr[k] * (double)u[k];
                }
                if (sd > 0.0) dsum += (double)cw[j] * (md / sd);
                atomicOr(J.status, sd > 0.0 ? ST_GUARD : ST_NUMERIC);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        if (lane == 0) dred[w] = dsum;
        __syncthreads();
        if (tid == 0) {
            double dist = 0.0;
#pragma unroll
            for (int i = 0; i < kPW; ++i) dist += dred[i];
            if (!(fabs(dist) < INFINITY)) atomicOr(J.status, ST_NUMERIC);
            J.out[p] = dist;
            if (J.iters) J.iters[p] = it;
        }
        __syncthreads();   // shared state is rewritten by the next pair
    }
}

template <int KPT, bool SMEMK>
int launch_pairs_t(swmd_corpus *c, const PairArgs &base, cudaStream_t st) {
    PairArgs a = base;
    const PairJob &J = a.job;
    const PairLayout L = pair_layout(J.max_q, J.max_x, 4 * KPT, SMEMK);
    auto kern = k_pairs<KPT, SMEMK>;
    SWMD_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.bytes));
    int per_sm = 0;
    SWMD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPT, L.bytes));
    if (per_sm < 1) return set_error(SWMD_EINVAL, "1-to-1 pairs: %d bytes of shared memory do not fit", L.bytes);
    long grid = std::min<long>(J.n_pairs, (long)c->sms * per_sm);
    if (!SMEMK) {
        // one K / KM region per block, reused pair after pair
        a.kws_stride = 2L * L.kelems;
        const size_t region = sizeof(float) * (size_t)a.kws_stride;
        grid = std::min<long>(grid, std::max<long>(1, (long)(kPairKwsMax / region)));
        const size_t need = region * (size_t)grid;
        if (c->pair_kws_bytes < need) {
            if (c->pair_kws) {
                SWMD_CK(cudaDeviceSynchronize());   // earlier pairs may still use the old regions
                corpus_free(c, c->pair_kws);
                c->pair_kws = nullptr;
                c->pair_kws_bytes = 0;
            }
            SWMD_CK(corpus_malloc(c, reinterpret_cast<void **>(&c->pair_kws), need));
            c->pair_kws_bytes = need;
        }
        a.kws = c->pair_kws;
    }
    kern<<<(unsigned)grid, kPT, L.bytes, st>>>(a);
    SWMD_CK(cudaGetLastError());
    return SWMD_OK;
}

template <bool SMEMK>
int launch_pairs_k(swmd_corpus *c, const PairArgs &a, cudaStream_t st) {
    const int mq = a.job.max_q;
    if (mq <= 8) return launch_pairs_t<2, SMEMK>(c, a, st);
    if (mq <= 16) return launch_pairs_t<4, SMEMK>(c, a, st);
    if (mq <= 24) return launch_pairs_t<6, SMEMK>(c, a, st);
    return launch_pairs_t<8, SMEMK>(c, a, st);
}

int check_pair_scalars(float lambda, int32_t max_iter, float tol) {
    if (!(lambda > 0.f) || std::isinf(lambda))
        return set_error(SWMD_EINVAL, "lambda must be finite and > 0");
    if (max_iter < 0) return set_error(SWMD_EINVAL, "max_iter must be >= 0");
    if (!(tol >= 0.f) || std::isinf(tol)) return set_error(SWMD_EINVAL, "tol must be finite and >= 0");
    return SWMD_OK;
}

}  // namespace

int enqueue_pairs(swmd_corpus *c, const PairJob &job, cudaStream_t st) {
    if (job.n_pairs == 0) return SWMD_OK;
    PairArgs a{};
    a.E = c->E;
    a.d4 = c->d4;
    a.V = c->V;
    a.job = job;
    a.shift = c->opt.column_shift ? 1 : 0;
    const size_t kbytes = sizeof(float) * 2 * (size_t)(job.max_q + 1) * (size_t)job.max_x;
    if (kbytes <= kPairSmemK) return launch_pairs_k<true>(c, a, st);
    return launch_pairs_k<false>(c, a, st);
}

}  // namespace swmd

using namespace swmd;

extern "C" {

int swmd_wmd_pairs_device(swmd_corpus *c, int32_t n_pairs, const int64_t *d_q_ptr,
                          const int32_t *d_q_ids, const float *d_r, const int64_t *d_x_ptr,
                          const int32_t *d_x_ids, const float *d_c, int32_t max_q_words,
                          int32_t max_x_words, float lambda, int32_t max_iter, float tol,
                          double *d_out, int32_t *d_iters, int32_t *d_status, void *stream) {
    if (!c) return set_error(SWMD_EINVAL, "swmd_wmd_pairs_device: NULL corpus");
    if (n_pairs < 0) return set_error(SWMD_EINVAL, "swmd_wmd_pairs_device: n_pairs < 0");
    int rc = check_pair_scalars(lambda, max_iter, tol);
    if (rc) return rc;
    if (n_pairs == 0) return SWMD_OK;
    if (!d_q_ptr || !d_q_ids || !d_r || !d_x_ptr || !d_x_ids || !d_c || !d_out || !d_status)
        return set_error(SWMD_EINVAL, "swmd_wmd_pairs_device: NULL array");
    if (max_q_words < 1 || max_q_words > kPairMaxWords || max_x_words < 1 ||
        max_x_words > kPairMaxWords)
        return set_error(SWMD_EINVAL, "swmd_wmd_pairs_device: size bounds %d, %d outside [1, %d]",
                         max_q_words, max_x_words, kPairMaxWords);
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    PairJob job{n_pairs, d_q_ptr, d_q_ids, d_r, d_x_ptr, d_x_ids, d_c, max_q_words, max_x_words,
                lambda, max_iter, tol, d_out, d_iters, d_status};
    return enqueue_pairs(c, job, stream ? static_cast<cudaStream_t>(stream) : c->stream);
}

int swmd_wmd_pairs(swmd_corpus *c, int32_t n_pairs, const int64_t *h_q_ptr,
                   const int32_t *h_q_ids, const float *h_q_weights, const int64_t *h_x_ptr,
                   const int32_t *h_x_ids, const float *h_x_weights, float lambda,
                   int32_t max_iter, float tol, double *h_out, int32_t *h_iters) {
    if (!c) return set_error(SWMD_EINVAL, "swmd_wmd_pairs: NULL corpus");
    if (n_pairs < 0) return set_error(SWMD_EINVAL, "swmd_wmd_pairs: n_pairs < 0");
    int rc = check_pair_scalars(lambda, max_iter, tol);
    if (rc) return rc;
    if (n_pairs == 0) return SWMD_OK;
    if (!h_q_ptr || !h_x_ptr || !h_out) return set_error(SWMD_EINVAL, "swmd_wmd_pairs: NULL array");
    if (h_q_ptr[0] != 0 || h_x_ptr[0] != 0)
        return set_error(SWMD_EINVAL, "swmd_wmd_pairs: q_ptr[0] and x_ptr[0] must be 0");
    // a0 for both sides of every pair (Section III-B1): merge, drop zeros, normalise
    std::vector<int64_t> qp((size_t)n_pairs + 1, 0), xp((size_t)n_pairs + 1, 0);
    std::vector<int32_t> qi, xi;
    std::vector<float> qr, xc;
    int max_q = 1, max_x = 1;
    std::vector<int32_t> ids;
    std::vector<float> wts;
    for (int32_t p = 0; p < n_pairs; ++p) {
        for (int side = 0; side < 2; ++side) {
            const int64_t *ptr = side ? h_x_ptr : h_q_ptr;
            const int64_t lo = ptr[p], hi = ptr[p + 1];
            if (hi < lo || hi - lo > INT32_MAX)
                return set_error(SWMD_EINVAL, "swmd_wmd_pairs: pair %d: %s offsets not increasing", p,
                                 side ? "target" : "query");
            const int32_t n = (int32_t)(hi - lo);
            if (n > 0 && (!(side ? h_x_ids : h_q_ids) || !(side ? h_x_weights : h_q_weights)))
                return set_error(SWMD_EINVAL, "swmd_wmd_pairs: NULL id or weight array");
            ids.resize((size_t)std::max(n, 1));
            wts.resize((size_t)std::max(n, 1));
            int32_t k = 0;
            rc = swmd_select(c->V, n, n ? (side ? h_x_ids : h_q_ids) + lo : nullptr,
                             n ? (side ? h_x_weights : h_q_weights) + lo : nullptr, ids.data(),
                             wts.data(), &k);
            if (rc)
                return set_error(rc, "swmd_wmd_pairs: pair %d, %s: %s", p, side ? "target" : "query",
                                 std::string(swmd_last_error()).c_str());
            if (k > kPairMaxWords)
                return set_error(SWMD_EINVAL, "swmd_wmd_pairs: pair %d, %s: %d distinct words, at most %d",
                                 p, side ? "target" : "query", k, kPairMaxWords);
            auto &I = side ? xi : qi;
            auto &W = side ? xc : qr;
            I.insert(I.end(), ids.begin(), ids.begin() + k);
            W.insert(W.end(), wts.begin(), wts.begin() + k);
            (side ? xp : qp)[(size_t)p + 1] = (int64_t)I.size();
            (side ? max_x : max_q) = std::max(side ? max_x : max_q, (int)k);
        }
    }
    auto up = [](size_t n) { return (n + 255) & ~size_t(255); };
    const size_t nq = qi.size(), nx = xi.size(), np = (size_t)n_pairs;
    size_t bytes = 0;
    const size_t o_qp = bytes; bytes += up(sizeof(int64_t) * (np + 1));
    const size_t o_xp = bytes; bytes += up(sizeof(int64_t) * (np + 1));
    const size_t o_qi = bytes; bytes += up(sizeof(int32_t) * nq);
    const size_t o_qr = bytes; bytes += up(sizeof(float) * nq);
    const size_t o_xi = bytes; bytes += up(sizeof(int32_t) * nx);
    const size_t o_xc = bytes; bytes += up(sizeof(float) * nx);
    const size_t o_out = bytes; bytes += up(sizeof(double) * np);
    const size_t o_it = bytes; bytes += up(sizeof(int32_t) * np);
    const size_t o_st = bytes; bytes += up(sizeof(int32_t));

    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard guard(c->device);
    cudaStream_t st = c->stream;
    if (c->pair_ws_bytes < bytes) {
        if (c->pair_ws) {
            SWMD_CK(cudaStreamSynchronize(st));
            corpus_free(c, c->pair_ws);
            c->pair_ws = nullptr;
            c->pair_ws_bytes = 0;
        }
        cudaError_t e = corpus_malloc(c, &c->pair_ws, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "swmd_wmd_pairs: workspace");
        c->pair_ws_bytes = bytes;
    }
    char *ws = static_cast<char *>(c->pair_ws);
    SWMD_CK(cudaMemcpyAsync(ws + o_qp, qp.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice, st));
    SWMD_CK(cudaMemcpyAsync(ws + o_xp, xp.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice, st));
    SWMD_CK(cudaMemcpyAsync(ws + o_qi, qi.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
    SWMD_CK(cudaMemcpyAsync(ws + o_qr, qr.data(), sizeof(float) * nq, cudaMemcpyHostToDevice, st));
    SWMD_CK(cudaMemcpyAsync(ws + o_xi, xi.data(), sizeof(int32_t) * nx, cudaMemcpyHostToDevice, st));
    SWMD_CK(cudaMemcpyAsync(ws + o_xc, xc.data(), sizeof(float) * nx, cudaMemcpyHostToDevice, st));
    SWMD_CK(cudaMemsetAsync(ws + o_st, 0, sizeof(int32_t), st));
    PairJob job{n_pairs,
                reinterpret_cast<const int64_t *>(ws + o_qp),
                reinterpret_cast<const int *>(ws + o_qi),
                reinterpret_cast<const float *>(ws + o_qr),
                reinterpret_cast<const int64_t *>(ws + o_xp),
                reinterpret_cast<const int *>(ws + o_xi),
                reinterpret_cast<const float *>(ws + o_xc),
                max_q, max_x, lambda, max_iter, tol,
                reinterpret_cast<double *>(ws + o_out),
                reinterpret_cast<int *>(ws + o_it),
                reinterpret_cast<int *>(ws + o_st)};
    if ((rc = enqueue_pairs(c, job, st))) return rc;
    int h_status = 0;
    SWMD_CK(cudaMemcpyAsync(h_out, ws + o_out, sizeof(double) * np, cudaMemcpyDeviceToHost, st));
    if (h_iters)
        SWMD_CK(cudaMemcpyAsync(h_iters, ws + o_it, sizeof(int32_t) * np, cudaMemcpyDeviceToHost, st));
    SWMD_CK(cudaMemcpyAsync(&h_status, ws + o_st, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SWMD_CK(cudaStreamSynchronize(st));
    return status_to_code(h_status);
}

}  // extern "C"
