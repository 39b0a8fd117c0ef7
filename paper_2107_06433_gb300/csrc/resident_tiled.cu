// a3 x t + a4 in one launch, with each document's K^T and KM^T rows held in
// shared memory for all iterations.
//
// Algorithm 1 treats every column of c (every target document) independently, so
// the t x-updates and the final step of one document can run from start to end
// in one team of lanes, with u in registers.  What each iteration reads is the
// document's K^T rows (SDDMM and SpMM of the fused SDDMM_SpMM, Section III-C)
// and, in the final step, its KM^T rows.  Here those rows are gathered once per
// document into shared memory (cp.async), so the t + 1 passes read them from
// shared memory instead of re-gathering them from L2 each time.
//
// Work unit: a tile = consecutive documents (in decreasing-length order) of one
// team size G = team_lanes_for(length), at most threads / G of them and at most NT
// nonzeros together (a longer document forms a tile alone and reads its rows
// beyond NT from global memory).  A block stages a tile, then each team of G
// lanes owns one document.  Inside a team, Q lanes share one nonzero's dot
// (VRP / Q values each) and P = G / Q nonzeros are in flight.
// Division uses the fast reciprocal form (2 ulp), checked against the FP64 oracle.
#include "walk.cuh"

namespace swmd {
namespace {

constexpr int kTileThreads = 256;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

// four consecutive K values at element offset 4*idx4 of a row, from shared or global memory
template <class T> __device__ __forceinline__ float4 ld4(const T *p, int idx4);
template <> __device__ __forceinline__ float4 ld4<float>(const float *p, int idx4) {
    return reinterpret_cast<const float4 *>(p)[idx4];
}
template <> __device__ __forceinline__ float4 ld4<__nv_bfloat16>(const __nv_bfloat16 *p, int idx4) {
    const uint2 raw = reinterpret_cast<const uint2 *>(p)[idx4];
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
template <> __device__ __forceinline__ float4 ld4<__half>(const __half *p, int idx4) {
    const uint2 raw = reinterpret_cast<const uint2 *>(p)[idx4];
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

template <int VRP, int Q, class KT_t>
__device__ __noinline__ void k_resident_tiled_body(const ResidentArgs &ra, const int *tiles, int n_tiles, int NT, int npl) {
    constexpr int S = VRP / Q;
    constexpr int C = S / 4;
    constexpr int ROWB = VRP * (int)sizeof(KT_t);          // bytes of one row
    constexpr int UNIT = (ROWB % 16 == 0) ? 16 : 8;          // cp.async granule
    constexpr int CPR = ROWB / UNIT;                         // granules per row
    static_assert(ROWB % 8 == 0, "row must be a multiple of 8 bytes");
    const IterArgs a = ra.it;   // one copy of the arguments (read in every tile)

    extern __shared__ __align__(16) unsigned char smem_raw[];
    KT_t *sK = reinterpret_cast<KT_t *>(smem_raw);
    KT_t *sKM = sK + (size_t)NT * VRP;
    float *sC = reinterpret_cast<float *>(sKM + (size_t)NT * VRP);
    int *sW = reinterpret_cast<int *>(sC + NT);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int vr = a.qp->vr;
    const float u0 = a.qp->u0;
    int *const status = a.qp->status;
    double *const out = a.out ? a.out : a.qp->out;
    const KT_t *KT = reinterpret_cast<const KT_t *>(a.KT);
    const KT_t *KMT = reinterpret_cast<const KT_t *>(a.KMT);

    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int d0 = __ldg(tiles + tile), d1 = __ldg(tiles + tile + 1);
        const int D = d1 - d0;
        const int p0 = __ldg(a.doc_ptr + d0);
        const int n = __ldg(a.doc_ptr + d1) - p0;
        const int ns = n < NT ? n : NT;   // rows staged in shared memory

        __syncthreads();   // the previous tile's rows are no longer read
        for (int i = tid; i < ns; i += blockDim.x) {
            const int2 e = __ldg(a.nz + p0 + i);
            sW[i] = e.x;
            sC[i] = __int_as_float(e.y);
        }
        __syncthreads();
        for (int i = tid; i < ns * CPR; i += blockDim.x) {
            const int row = i / CPR, g = i - row * CPR;
            const size_t src = (size_t)sW[row] * ROWB + (size_t)g * UNIT;
            unsigned char *dk = reinterpret_cast<unsigned char *>(sK) + (size_t)row * ROWB + g * UNIT;
            unsigned char *dm = reinterpret_cast<unsigned char *>(sKM) + (size_t)row * ROWB + g * UNIT;
            const unsigned char *gk = reinterpret_cast<const unsigned char *>(KT) + src;
            const unsigned char *gm = reinterpret_cast<const unsigned char *>(KMT) + src;
            if constexpr (UNIT == 16) {
                cp_async16(dk, gk);
                cp_async16(dm, gm);
            } else {
                cp_async8(dk, gk);
                cp_async8(dm, gm);
            }
        }
        cp_async_wait_all();
        __syncthreads();

        // team geometry of this tile: every document in it has the same team size
        const int G = team_lanes_for(__ldg(a.doc_ptr + d0 + 1) - p0, npl);
        const int P = G / Q;
        const int team = tid / G;
        const int tl = tid - team * G;
        const int p = tl / Q;
        const int q = tl - p * Q;
        const bool has = team < D;
        const int doc = d0 + team;
        int beg = 0, len = 0;
        if (has) {
            beg = __ldg(a.doc_ptr + doc) - p0;
            len = __ldg(a.doc_ptr + doc + 1) - p0 - beg;
        }
        // warps whose teams all lack a document skip the tile
        if (!__any_sync(kFull, has)) continue;
        int rounds = (len + P - 1) / P;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rounds = max(rounds, __shfl_xor_sync(kFull, rounds, o));

        float uu[S];
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * (c * Q + q) + e;
                uu[4 * c + e] = (has && k < vr) ? u0 : 0.f;
            }

        for (int it = 0; it < ra.t; ++it) {
            float acc[S];
#pragma unroll
            for (int i = 0; i < S; ++i) acc[i] = 0.f;
            for (int i = 0; i < rounds; ++i) {
                const int idx = i * P + p;
                const bool valid = idx < len;
                const int li = beg + (valid ? idx : 0);
                float kr[S];
                float cval;
                if (li < NT) {
                    const KT_t *row = sK + (size_t)li * VRP;
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const float4 t = ld4<KT_t>(row, c * Q + q);
                        kr[4 * c] = t.x; kr[4 * c + 1] = t.y; kr[4 * c + 2] = t.z; kr[4 * c + 3] = t.w;
                    }
                    cval = sC[li];
                } else {
                    const int2 e = __ldg(a.nz + p0 + li);
                    const long row4 = (long)e.x * (VRP / 4);
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const float4 t = KIO<KT_t>::load4(KT, row4 + c * Q + q);
                        kr[4 * c] = t.x; kr[4 * c + 1] = t.y; kr[4 * c + 2] = t.z; kr[4 * c + 3] = t.w;
                    }
                    cval = __int_as_float(e.y);
                }
                float d4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int s = 0; s < S; ++s) d4[s & 3] = fmaf(kr[s], uu[s], d4[s & 3]);
                float dot = (d4[0] + d4[1]) + (d4[2] + d4[3]);
#pragma unroll
                for (int o = 1; o < Q; o <<= 1) dot += __shfl_xor_sync(kFull, dot, o);
                const bool tiny = valid && !(dot >= 0x1p-100f);
                float tau = valid ? __fdividef(cval, dot) : 0.f;
                if (__any_sync(kFull, tiny)) {
                    SWMD_COLD_PATH();
                    double dot64 = 0.0;
#pragma unroll
                    for (int s = 0; s < S; ++s) dot64 = fma((double)kr[s], (double)uu[s], dot64);
#pragma unroll
                    for (int o = 1; o < Q; o <<= 1) dot64 += __shfl_xor_sync(kFull, dot64, o);
                    if (tiny) {
                        tau = (dot64 > 0.0) ? (float)((double)cval / dot64) : 0.f;
                        if (q == 0) atomicOr(status, dot64 > 0.0 ? ST_GUARD : ST_NUMERIC);
                    }
                }
#pragma unroll
                for (int s = 0; s < S; ++s) acc[s] = fmaf(tau, kr[s], acc[s]);
            }
            for (int o = Q; o < G; o <<= 1)
#pragma unroll
                for (int s = 0; s < S; ++s) acc[s] += __shfl_xor_sync(kFull, acc[s], o);
            bool bad = false;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                // r is zero-padded to VRP, so padded entries of u stay 0
                const float4 r4 = __ldg(reinterpret_cast<const float4 *>(a.r) + c * Q + q);
                const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float nu = (has && rv[e] > 0.f) ? __fdividef(rv[e], acc[4 * c + e]) : 0.f;
                    bad |= !(nu < INFINITY);
                    uu[4 * c + e] = nu;
                }
            }
            if (bad && has) atomicOr(status, ST_NUMERIC);
        }

        double dist = 0.0;
        for (int i = 0; i < rounds; ++i) {
            const int idx = i * P + p;
            const bool valid = idx < len;
            const int li = beg + (valid ? idx : 0);
            float kr[S], km[S];
            float cval;
            if (li < NT) {
                const KT_t *row = sK + (size_t)li * VRP;
                const KT_t *mrow = sKM + (size_t)li * VRP;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float4 t = ld4<KT_t>(row, c * Q + q);
                    kr[4 * c] = t.x; kr[4 * c + 1] = t.y; kr[4 * c + 2] = t.z; kr[4 * c + 3] = t.w;
                    const float4 m = ld4<KT_t>(mrow, c * Q + q);
                    km[4 * c] = m.x; km[4 * c + 1] = m.y; km[4 * c + 2] = m.z; km[4 * c + 3] = m.w;
                }
                cval = sC[li];
            } else {
                const int2 e = __ldg(a.nz + p0 + li);
                const long row4 = (long)e.x * (VRP / 4);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float4 t = KIO<KT_t>::load4(KT, row4 + c * Q + q);
                    kr[4 * c] = t.x; kr[4 * c + 1] = t.y; kr[4 * c + 2] = t.z; kr[4 * c + 3] = t.w;
                    const float4 m = KIO<KT_t>::load4(KMT, row4 + c * Q + q);
                    km[4 * c] = m.x; km[4 * c + 1] = m.y; km[4 * c + 2] = m.z; km[4 * c + 3] = m.w;
                }
                cval = __int_as_float(e.y);
            }
            float d4[4] = {0.f, 0.f, 0.f, 0.f}, m4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int s = 0; s < S; ++s) {
                d4[s & 3] = fmaf(kr[s], uu[s], d4[s & 3]);
                m4[s & 3] = fmaf(km[s], uu[s], m4[s & 3]);
            }
            float dot = (d4[0] + d4[1]) + (d4[2] + d4[3]);
            float dm = (m4[0] + m4[1]) + (m4[2] + m4[3]);
#pragma unroll
            for (int o = 1; o < Q; o <<= 1) {
                dot += __shfl_xor_sync(kFull, dot, o);
                dm += __shfl_xor_sync(kFull, dm, o);
            }
            const bool tiny = valid && !(dot >= 0x1p-100f);
            double contrib = valid ? (double)(cval * (dm / dot)) : 0.0;
            if (__any_sync(kFull, tiny)) {
                SWMD_COLD_PATH();
                double dot64 = 0.0, dm64 = 0.0;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    dot64 = fma((double)kr[s], (double)uu[s], dot64);
                    dm64 = fma((double)km[s], (double)uu[s], dm64);
                }
#pragma unroll
                for (int o = 1; o < Q; o <<= 1) {
                    dot64 += __shfl_xor_sync(kFull, dot64, o);
                    dm64 += __shfl_xor_sync(kFull, dm64, o);
                }
                if (tiny) {
                    contrib = (double)cval * (dm64 / dot64);
                    if (q == 0) atomicOr(status, dot64 > 0.0 ? ST_GUARD : ST_NUMERIC);
                }
            }
            if (q == 0) dist += contrib;
        }
        for (int o = Q; o < G; o <<= 1) dist += __shfl_xor_sync(kFull, dist, o);
        if (has && tl == 0) {
            if (!(fabs(dist) < INFINITY)) atomicOr(status, ST_NUMERIC);
            out[__ldg(a.doc_orig + doc)] = dist;
        }
    }
}

template <int VRP, int Q, class KT_t>
__global__ void __launch_bounds__(kTileThreads)
k_resident_tiled(const __grid_constant__ ResidentArgs ra0, const ResidentArgs *batch, const int *tiles,
                 int n_tiles, int NT, int npl) {
    // one query per grid row when batched (batch[blockIdx.y]), else the argument
    if (batch) k_resident_tiled_body<VRP, Q, KT_t>(batch[blockIdx.y], tiles, n_tiles, NT, npl);
    else k_resident_tiled_body<VRP, Q, KT_t>(ra0, tiles, n_tiles, NT, npl);
}

template <int VRP, int Q, class KT_t>
cudaError_t run_tiled(const ResidentArgs &a, const TileSet &ts, int sms, cudaStream_t s, int nq,
                      const ResidentArgs *batch) {
    auto kern = k_resident_tiled<VRP, Q, KT_t>;
    const size_t smem = tiled_smem_bytes(VRP, (int)sizeof(KT_t), ts.nt);
    static LaunchCache cache;
    int per_sm = 1;
    cudaError_t e = cache.blocks_per_sm(kern, ts.threads, smem, 100, &per_sm);
    if (e != cudaSuccess) return e;
    int blocks = nq == 1 ? sms * per_sm : (sms * per_sm * 2 + nq - 1) / nq;
    if (blocks < 1) blocks = 1;
    if (blocks > ts.n_tiles) blocks = ts.n_tiles;
    if (blocks > 0)
        kern<<<dim3(blocks, nq), ts.threads, smem, s>>>(a, batch, ts.tiles, ts.n_tiles, ts.nt, ts.npl);
    return cudaGetLastError();
}

template <class KT_t>
cudaError_t dispatch_tiled(const ResidentArgs &a, int vrp, const TileSet &ts, int sms, cudaStream_t s,
                           int nq, const ResidentArgs *batch) {
    switch (vrp) {
#define SWMD_T1(V) \
    case V: return run_tiled<V, 1, KT_t>(a, ts, sms, s, nq, batch);
        SWMD_T1(4) SWMD_T1(8) SWMD_T1(12) SWMD_T1(16) SWMD_T1(20) SWMD_T1(24) SWMD_T1(28) SWMD_T1(32)
#undef SWMD_T1
        case 40: return run_tiled<40, 2, KT_t>(a, ts, sms, s, nq, batch);
        case 48: return run_tiled<48, 2, KT_t>(a, ts, sms, s, nq, batch);
        case 56: return run_tiled<56, 2, KT_t>(a, ts, sms, s, nq, batch);
        case 64: return run_tiled<64, 2, KT_t>(a, ts, sms, s, nq, batch);
        case 80: return run_tiled<80, 4, KT_t>(a, ts, sms, s, nq, batch);
        case 96: return run_tiled<96, 4, KT_t>(a, ts, sms, s, nq, batch);
        case 112: return run_tiled<112, 4, KT_t>(a, ts, sms, s, nq, batch);
        case 128: return run_tiled<128, 4, KT_t>(a, ts, sms, s, nq, batch);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t tiled_smem_bytes(int vrp, int kbytes, int nt) {
    return (size_t)nt * (2 * (size_t)vrp * kbytes + 8) + 16;
}

bool tiled_supported(int vrp, int kprec) {
    if (vrp % 4 || vrp < 4 || vrp > 128) return false;
    if (vrp > 32 && vrp % 8) return false;
    if (vrp > 64 && vrp % 16) return false;
    return (vrp * (int)kprec_bytes(kprec)) % 8 == 0;
}

cudaError_t launch_resident_tiled(const ResidentArgs &a, int vrp, int kprec, const TileSet &ts,
                                  int sms, cudaStream_t s, int nq, const ResidentArgs *batch) {
    switch (kprec) {
        case 0: return dispatch_tiled<float>(a, vrp, ts, sms, s, nq, batch);
        case 1: return dispatch_tiled<__nv_bfloat16>(a, vrp, ts, sms, s, nq, batch);
        case 2: return dispatch_tiled<__half>(a, vrp, ts, sms, s, nq, batch);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swmd
