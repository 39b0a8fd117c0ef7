// The per-document walk over c's nonzeros shared by the iteration kernels.
//
// Section III-B4 turns the dense K^T u of Algorithm 1 into an SDDMM evaluated only
// at c's nonzeros (Algorithm 2) followed by an SpMM (Algorithm 3); Section III-C
// fuses the two so v never reaches memory.  Here the walk is document-major (the
// CSC of c): one team of G = P*Q lanes owns document j, so the SpMM accumulation
// x[:, j] needs no atomics (the paper's word-major order needed them, Section
// III-D) and every document's result is independent of the others.
//
//   Kind::Fused  one x-update, SDDMM_SpMM type 1: for each nonzero (w, c_wj)
//                s = K^T[w].u_j, tau = c_wj / s, acc += tau K^T[w]; then
//                u_j[k] = r_k / acc[k]  (x = diag(1/r) K v, u = 1/x).
//   Kind::Sddmm  the unfused SDDMM: v[nz] = c_wj / (K^T[w].u_j) written to memory.
//   Kind::Spmm   the unfused SpMM: acc += v[nz] K^T[w]; then the u update.
//   Kind::Final  SDDMM_SpMM type 2 and the distance: WMD_j = sum over nonzeros of
//                c_wj (KM^T[w].u_j) / (K^T[w].u_j), FP64 per-document sum.
//
// Lane layout: P sub-teams of Q lanes.  Sub-team p handles nonzeros p, p+P, ...
// of the document; lane q of a sub-team holds the float4 chunks c*Q + q
// (c < S/4) of u_j, of acc and of the K^T row, so one row is read by Q lanes
// with consecutive 16-byte loads.  The Q partial dots are combined with
// butterfly shuffles, the P partial accumulators likewise at the end.
#pragma once

#include "common.cuh"

namespace swmd {

enum class Kind { Fused, Sddmm, Spmm, Final };

// The FP64 guard of K^T u runs only when some lane's FP32 dot fell below
// 2^-100.  The empty volatile asm at its entry keeps the compiler from turning
// the branch into predicated code evaluated on every nonzero: FP64 throughput is
// a small fraction of FP32 on this GPU.
#define SWMD_COLD_PATH() asm volatile("" ::: "memory")

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWalkThreads = 256;

template <int VRP, int Q, int P, class KT_t, Kind KIND>
__global__ void __launch_bounds__(kWalkThreads) k_walk(IterArgs a) {
    constexpr int G = P * Q;
    constexpr int S = VRP / Q;
    constexpr int C = S / 4;
    constexpr int TPW = 32 / G;
    static_assert(G <= 32 && (32 % G) == 0, "team must divide a warp");
    static_assert(VRP % (4 * Q) == 0, "VRP must be a multiple of 4Q");

    const int lane = threadIdx.x & 31;
    const int tl = lane & (G - 1);
    const int p = tl / Q;
    const int q = tl - p * Q;
    const int team_in_warp = lane / G;
    const long warp_global = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    const int vr = a.qp->vr;
    const float u0 = a.qp->u0;
    int *const status = a.qp->status;
    double *const out = a.out ? a.out : a.qp->out;
    const KT_t *KT = reinterpret_cast<const KT_t *>(a.KT);
    const KT_t *KMT = reinterpret_cast<const KT_t *>(a.KMT);

    for (long base = warp_global * TPW; base < a.N; base += nwarps * TPW) {
        const long doc = a.doc0 + base + team_in_warp;
        const bool has = base + team_in_warp < a.N;
        int beg = 0, end = 0;
        if (has) {
            beg = __ldg(a.doc_ptr + doc);
            end = __ldg(a.doc_ptr + doc + 1);
        }

        float uu[S];
        if constexpr (KIND != Kind::Spmm) {
            if (a.first) {
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        uu[4 * c + e] = (4 * (c * Q + q) + e < vr) ? u0 : 0.f;
            } else if (has) {
                const float4 *ur = reinterpret_cast<const float4 *>(a.u + doc * VRP);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float4 t = ur[c * Q + q];
                    uu[4 * c] = t.x; uu[4 * c + 1] = t.y; uu[4 * c + 2] = t.z; uu[4 * c + 3] = t.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < S; ++i) uu[i] = 0.f;
            }
        }

        float acc[S];
#pragma unroll
        for (int i = 0; i < S; ++i) acc[i] = 0.f;
        double dist = 0.0;

        int rounds = (end - beg + P - 1) / P;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rounds = max(rounds, __shfl_xor_sync(kFull, rounds, o));

        for (int i = 0; i < rounds; ++i) {
            const int idx = beg + i * P + p;
            const bool valid = idx < end;
            const int2 e = valid ? __ldg(a.nz + idx) : make_int2(0, 0);
            const float cval = __int_as_float(e.y);
            const long row4 = (long)e.x * (VRP / 4);

            float kr[S];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float4 t = KIO<KT_t>::load4(KT, row4 + c * Q + q);
                kr[4 * c] = t.x; kr[4 * c + 1] = t.y; kr[4 * c + 2] = t.z; kr[4 * c + 3] = t.w;
            }

            if constexpr (KIND == Kind::Spmm) {
                const float tau = valid ? __ldg(a.v + idx) : 0.f;
#pragma unroll
                for (int s = 0; s < S; ++s) acc[s] = fmaf(tau, kr[s], acc[s]);
            } else {
                float dot = 0.f;
#pragma unroll
                for (int s = 0; s < S; ++s) dot = fmaf(kr[s], uu[s], dot);
#pragma unroll
                for (int o = 1; o < Q; o <<= 1) dot += __shfl_xor_sync(kFull, dot, o);

                float km[KIND == Kind::Final ? S : 1];
                float dm = 0.f;
                if constexpr (KIND == Kind::Final) {
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const float4 t = KIO<KT_t>::load4(KMT, row4 + c * Q + q);
                        km[4 * c] = t.x; km[4 * c + 1] = t.y; km[4 * c + 2] = t.z; km[4 * c + 3] = t.w;
                    }
#pragma unroll
                    for (int s = 0; s < S; ++s) dm = fmaf(km[s], uu[s], dm);
#pragma unroll
                    for (int o = 1; o < Q; o <<= 1) dm += __shfl_xor_sync(kFull, dm, o);
                }

                // Guard: K^T u so small that FP32 products may have underflowed.  The
                // dots are recomputed in FP64 from the same (exactly widened) inputs.
                const bool tiny = valid && !(dot >= 0x1p-100f);
                double dot64 = 0.0, dm64 = 0.0;
                if (__any_sync(kFull, tiny)) {
                    SWMD_COLD_PATH();
#pragma unroll
                    for (int s = 0; s < S; ++s) dot64 = fma((double)kr[s], (double)uu[s], dot64);
#pragma unroll
                    for (int o = 1; o < Q; o <<= 1) dot64 += __shfl_xor_sync(kFull, dot64, o);
                    if constexpr (KIND == Kind::Final) {
#pragma unroll
                        for (int s = 0; s < S; ++s) dm64 = fma((double)km[s], (double)uu[s], dm64);
#pragma unroll
                        for (int o = 1; o < Q; o <<= 1) dm64 += __shfl_xor_sync(kFull, dm64, o);
                    }
                    if (tiny && q == 0) atomicOr(status, dot64 > 0.0 ? ST_GUARD : ST_NUMERIC);
                }

                if constexpr (KIND == Kind::Final) {
                    if (valid && q == 0) {
                        if (tiny) dist += (double)cval * (dm64 / dot64);
                        else dist += (double)(cval * (dm / dot));
                    }
                } else {
                    float tau = valid ? cval / dot : 0.f;
                    if (tiny) tau = (dot64 > 0.0) ? (float)((double)cval / dot64) : 0.f;
                    if constexpr (KIND == Kind::Sddmm) {
                        if (valid && q == 0) a.v[idx] = tau;
                    } else {
#pragma unroll
                        for (int s = 0; s < S; ++s) acc[s] = fmaf(tau, kr[s], acc[s]);
                    }
                }
            }
        }

        if constexpr (KIND == Kind::Fused || KIND == Kind::Spmm) {
#pragma unroll
            for (int o = Q; o < G; o <<= 1)
#pragma unroll
                for (int s = 0; s < S; ++s) acc[s] += __shfl_xor_sync(kFull, acc[s], o);
            if (has) {
                float4 *ur = reinterpret_cast<float4 *>(a.u + doc * VRP);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    if (c % P != p) continue;
                    const int k0 = 4 * (c * Q + q);
                    float o4[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int k = k0 + e;
                        float val = 0.f;
                        if (k < vr) {
                            val = __ldg(a.r + k) / acc[4 * c + e];
                            if (!(val < INFINITY)) atomicOr(status, ST_NUMERIC);
                        }
                        o4[e] = val;
                    }
                    ur[c * Q + q] = make_float4(o4[0], o4[1], o4[2], o4[3]);
                }
            }
        } else if constexpr (KIND == Kind::Final) {
#pragma unroll
            for (int o = Q; o < G; o <<= 1) dist += __shfl_xor_sync(kFull, dist, o);
            if (has && tl == 0) {
                if (!(fabs(dist) < INFINITY)) atomicOr(status, ST_NUMERIC);
                out[__ldg(a.doc_orig + doc)] = dist;
            }
        }
    }
}

// All t x-updates and the final step of each document in one launch.  Algorithm 1
// acts on every column of c independently, so a team can keep u_j in registers
// from the first x-update to the distance: u never travels to memory and c's
// nonzeros of the document are re-read from cache each iteration.  Per iteration
// the work is the Kind::Fused walk; at the end the Kind::Final walk.
template <int VRP, int Q, int P, class KT_t>
__global__ void __launch_bounds__(kWalkThreads) k_resident(ResidentArgs ra) {
    constexpr int G = P * Q;
    constexpr int S = VRP / Q;
    constexpr int C = S / 4;
    constexpr int TPW = 32 / G;
    static_assert(G <= 32 && (32 % G) == 0, "team must divide a warp");
    static_assert(VRP % (4 * Q) == 0, "VRP must be a multiple of 4Q");
    const IterArgs &a = ra.it;

    const int lane = threadIdx.x & 31;
    const int tl = lane & (G - 1);
    const int p = tl / Q;
    const int q = tl - p * Q;
    const int team_in_warp = lane / G;
    const long warp_global = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    const int vr = a.qp->vr;
    const float u0 = a.qp->u0;
    int *const status = a.qp->status;
    double *const out = a.out ? a.out : a.qp->out;
    const KT_t *KT = reinterpret_cast<const KT_t *>(a.KT);
    const KT_t *KMT = reinterpret_cast<const KT_t *>(a.KMT);

    float rr[S];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = 4 * (c * Q + q) + e;
            rr[4 * c + e] = (k < vr) ? __ldg(a.r + k) : 0.f;
        }

    for (long base = warp_global * TPW; base < a.N; base += nwarps * TPW) {
        const long doc = a.doc0 + base + team_in_warp;
        const bool has = base + team_in_warp < a.N;
        int beg = 0, end = 0;
        if (has) {
            beg = __ldg(a.doc_ptr + doc);
            end = __ldg(a.doc_ptr + doc + 1);
        }
        int rounds = (end - beg + P - 1) / P;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rounds = max(rounds, __shfl_xor_sync(kFull, rounds, o));

        float uu[S];
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                uu[4 * c + e] = (has && 4 * (c * Q + q) + e < vr) ? u0 : 0.f;

        for (int it = 0; it < ra.t; ++it) {
            float acc[S];
#pragma unroll
            for (int i = 0; i < S; ++i) acc[i] = 0.f;
            for (int i = 0; i < rounds; ++i) {
                const int idx = beg + i * P + p;
                const bool valid = idx < end;
                const int2 e = valid ? __ldg(a.nz + idx) : make_int2(0, 0);
                const float cval = __int_as_float(e.y);
                const long row4 = (long)e.x * (VRP / 4);
                float kr[S];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float4 t = KIO<KT_t>::load4(KT, row4 + c * Q + q);
                    kr[4 * c] = t.x; kr[4 * c + 1] = t.y; kr[4 * c + 2] = t.z; kr[4 * c + 3] = t.w;
                }
                float d4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int s = 0; s < S; ++s) d4[s & 3] = fmaf(kr[s], uu[s], d4[s & 3]);
                float dot = (d4[0] + d4[1]) + (d4[2] + d4[3]);
#pragma unroll
                for (int o = 1; o < Q; o <<= 1) dot += __shfl_xor_sync(kFull, dot, o);
                const bool tiny = valid && !(dot >= 0x1p-100f);
                float tau = valid ? cval / dot : 0.f;
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
#pragma unroll
            for (int o = Q; o < G; o <<= 1)
#pragma unroll
                for (int s = 0; s < S; ++s) acc[s] += __shfl_xor_sync(kFull, acc[s], o);
            bool bad = false;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const float nu = (rr[s] > 0.f) ? rr[s] / acc[s] : 0.f;
                bad |= !(nu < INFINITY);
                uu[s] = nu;
            }
            if (bad && has) atomicOr(status, ST_NUMERIC);
        }

        double dist = 0.0;
        for (int i = 0; i < rounds; ++i) {
            const int idx = beg + i * P + p;
            const bool valid = idx < end;
            const int2 e = valid ? __ldg(a.nz + idx) : make_int2(0, 0);
            const float cval = __int_as_float(e.y);
            const long row4 = (long)e.x * (VRP / 4);
            float kr[S], km[S];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float4 t = KIO<KT_t>::load4(KT, row4 + c * Q + q);
                kr[4 * c] = t.x; kr[4 * c + 1] = t.y; kr[4 * c + 2] = t.z; kr[4 * c + 3] = t.w;
                const float4 m = KIO<KT_t>::load4(KMT, row4 + c * Q + q);
                km[4 * c] = m.x; km[4 * c + 1] = m.y; km[4 * c + 2] = m.z; km[4 * c + 3] = m.w;
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
#pragma unroll
        for (int o = Q; o < G; o <<= 1) dist += __shfl_xor_sync(kFull, dist, o);
        if (has && tl == 0) {
            if (!(fabs(dist) < INFINITY)) atomicOr(status, ST_NUMERIC);
            out[__ldg(a.doc_orig + doc)] = dist;
        }
    }
}

// The mappings compiled for the walk kernels: (VRP, Q, P).
#define SWMD_WALK_MAPPINGS(X)                                                         \
    X(4, 1, 4) X(4, 1, 8) X(8, 1, 4) X(8, 1, 8) X(8, 2, 4) X(12, 1, 4) X(12, 1, 8)   \
    X(16, 1, 4) X(16, 1, 8) X(16, 2, 4) X(16, 4, 4) X(20, 1, 4) X(20, 1, 8)          \
    X(24, 1, 4) X(24, 1, 8) X(24, 2, 4) X(28, 1, 4) X(28, 1, 8) X(32, 1, 4)          \
    X(32, 1, 8) X(32, 2, 4) X(32, 4, 4) X(32, 8, 4) X(40, 2, 4) X(48, 2, 4)          \
    X(48, 4, 4) X(56, 2, 4) X(64, 2, 4) X(64, 4, 4) X(64, 8, 4) X(80, 4, 4)          \
    X(96, 4, 4) X(96, 8, 4) X(112, 4, 4) X(128, 4, 4) X(128, 8, 4)

template <class K>
int walk_blocks(K kernel, LaunchCache &cache, long N, int G, int sms) {
    int per_sm = 1;
    if (cache.blocks_per_sm(kernel, kWalkThreads, 0, -1, &per_sm) != cudaSuccess) per_sm = 1;
    const long need = (N * G + kWalkThreads - 1) / kWalkThreads;
    const long cap = (long)sms * per_sm;
    const long b = need < cap ? need : cap;
    return (int)(b < 1 ? 1 : b);
}

template <int VRP, int Q, int P, class KT_t, Kind KIND>
cudaError_t run_walk(const IterArgs &a, int sms, cudaStream_t s) {
    auto kern = k_walk<VRP, Q, P, KT_t, KIND>;
    static LaunchCache cache;
    const int blocks = walk_blocks(kern, cache, a.N, P * Q, sms);
    if (a.N > 0) kern<<<blocks, kWalkThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class KT_t, Kind KIND>
cudaError_t dispatch_walk(const IterArgs &a, Mapping m, int sms, cudaStream_t s) {
    const int key = m.vrp * 10000 + m.q * 100 + m.p;
    switch (key) {
#define SWMD_CASE(V, QQ, PP) \
    case V * 10000 + QQ * 100 + PP: return run_walk<V, QQ, PP, KT_t, KIND>(a, sms, s);
        SWMD_WALK_MAPPINGS(SWMD_CASE)
#undef SWMD_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <Kind KIND>
cudaError_t dispatch_walk_prec(const IterArgs &a, Mapping m, int kprec, int sms, cudaStream_t s) {
    switch (kprec) {
        case 0: return dispatch_walk<float, KIND>(a, m, sms, s);
        case 1: return dispatch_walk<__nv_bfloat16, KIND>(a, m, sms, s);
        case 2: return dispatch_walk<__half, KIND>(a, m, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int VRP, int Q, int P, class KT_t>
cudaError_t run_resident(const ResidentArgs &a, int sms, cudaStream_t s) {
    auto kern = k_resident<VRP, Q, P, KT_t>;
    static LaunchCache cache;
    const int blocks = walk_blocks(kern, cache, a.it.N, P * Q, sms);
    if (a.it.N > 0) kern<<<blocks, kWalkThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class KT_t>
cudaError_t dispatch_resident(const ResidentArgs &a, Mapping m, int sms, cudaStream_t s) {
    const int key = m.vrp * 10000 + m.q * 100 + m.p;
    switch (key) {
#define SWMD_CASE(V, QQ, PP) \
    case V * 10000 + QQ * 100 + PP: return run_resident<V, QQ, PP, KT_t>(a, sms, s);
        SWMD_WALK_MAPPINGS(SWMD_CASE)
#undef SWMD_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swmd
