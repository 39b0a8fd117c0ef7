// a3 x t + a4 in one launch with each document's K^T rows held in registers.
// (Templates; resident_regs_{fp32,bf16,fp16}.cu instantiate one K precision each.)
//
// Every column of c is an independent problem in Algorithm 1, and one x-update of
// document j only touches the rows K^T[w] of its own words: with A_j the
// len_j x v_r matrix of those rows, an iteration is s = A_j u, tau = c_j ./ s,
// acc = A_j^T tau, u = r ./ acc (the fused SDDMM_SpMM of Section III-C).  Here A_j
// is spread over a team of G lanes (lane p holds rows p, p + G, ... -- up to NPL
// of them -- in registers) and stays there for all t iterations, so an iteration
// is register FMAs plus one team reduction of acc.  The reduction goes through a
// per-warp shared-memory transpose: every lane stores its partial acc, lane p
// sums the entries k = p, p + G, ... over the team, divides r_k by it, and
// publishes u_k; the team then reads the new u back.  The final step (Algorithm 1
// last line) reloads the same positions with the KM^T rows.
//
// Documents longer than 32 * NPL use a whole warp; their remaining K^T rows are
// staged once into a per-warp shared-memory buffer (sized from the corpus's
// longest document, up to `ovf_cap` rows; any rows beyond that are read from L2
// each iteration).  Teams are formed from documents of one team size, so a
// document's arithmetic depends on its own length only.
#pragma once

#include "walk.cuh"

namespace swmd {
namespace {

constexpr int kRegThreads = 128;
constexpr int kWarps = kRegThreads / 32;

// Per-warp transpose buffer: lane l's partial row of acc starts at float 33 l
// (a row stride of 33 = 1 mod 32 banks), so a team's rows sit at 33 * (lane of
// its first member); storing one k across the warp, summing one column across a
// team, publishing u and reading it back are all free of bank conflicts.
constexpr int kRowStride = 33;

// Element k of a row held as pairs (k a compile-time index after unrolling).
template <int N>
__device__ __forceinline__ float row_at(const float2 (&r)[N], int k) {
    return (k & 1) ? r[k >> 1].y : r[k >> 1].x;
}

template <int VRP, int NPL, int G, class KT_t>
__device__ __forceinline__ void regs_task(const IterArgs &a, int t, int4 tk, int lane, float *wacc,
                                          float *wrow, float *wc, int ovf_cap) {
    constexpr int C = VRP / 4;
    constexpr int KS = (VRP + G - 1) / G;   // entries of u each lane finishes
    static_assert(VRP <= kRowStride, "row stride");
    const int vr = a.qp->vr;
    const float u0 = a.qp->u0;
    int *const status = a.qp->status;
    double *const out = a.out ? a.out : a.qp->out;
    const KT_t *KT = reinterpret_cast<const KT_t *>(a.KT);
    const KT_t *KMT = reinterpret_cast<const KT_t *>(a.KMT);

    const int d0 = tk.x, nd = tk.z;
    const int team = lane / G;
    const int p = lane - team * G;
    const bool has = team < nd;
    const int doc = d0 + team;
    int beg = 0, len = 0;
    if (has) {
        beg = __ldg(a.doc_ptr + doc);
        len = __ldg(a.doc_ptr + doc + 1) - beg;
    }
    float *tacc = wacc + team * G * kRowStride;   // this team's G partial accumulators

    // overflow rows (documents longer than G * NPL exist only with G = 32, one
    // document per warp): the first ovf_cap go to shared memory once
    int extra = 0, n_ovf = 0;
    if (G == 32) {
        extra = len > 32 * NPL ? (len - 32 * NPL + 31) / 32 : 0;
        if (extra > 0) {
            const int n_all = len - 32 * NPL;
            n_ovf = n_all < ovf_cap ? n_all : ovf_cap;
            for (int i = lane; i < n_ovf * C; i += 32) {
                const int row = i / C, c = i - row * C;
                const int2 e = __ldg(a.nz + beg + 32 * NPL + row);
                reinterpret_cast<float4 *>(wrow)[i] = KIO<KT_t>::load4(KT, (long)e.x * C + c);
                if (c == 0) wc[row] = __int_as_float(e.y);
            }
            __syncwarp();
        }
    }

    // rows as pairs: the operands of the packed f32x2 FMAs of the iteration
    float2 rows2[NPL][VRP / 2];
    float cv[NPL];
    int wid[NPL];
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        const int idx = p + G * j;
        const bool valid = idx < len;
        int2 e = make_int2(0, 0);
        if (valid) e = __ldg(a.nz + beg + idx);
        wid[j] = e.x;
        cv[j] = valid ? __int_as_float(e.y) : 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float4 v = valid ? KIO<KT_t>::load4(KT, (long)e.x * C + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            rows2[j][2 * c] = make_float2(v.x, v.y);
            rows2[j][2 * c + 1] = make_float2(v.z, v.w);
        }
    }
    // r for the entries of u this lane finishes (k = p + G i)
    float rk[KS];
#pragma unroll
    for (int i = 0; i < KS; ++i) {
        const int k = p + G * i;
        rk[i] = (has && k < VRP && k < vr) ? __ldg(a.r + k) : 0.f;
    }
    float uu[VRP];
#pragma unroll
    for (int k = 0; k < VRP; ++k) uu[k] = (has && k < vr) ? u0 : 0.f;

    for (int it = 0; it < t; ++it) {
        float acc[VRP];
        float2 acc2[VRP / 2];
#pragma unroll
        for (int k = 0; k < VRP / 2; ++k) acc2[k] = make_float2(0.f, 0.f);
        bool tiny_any = false;
#pragma unroll
        for (int j = 0; j < NPL; ++j) {
            float2 da = make_float2(0.f, 0.f), db = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < VRP / 2; k += 2) {
                da = __ffma2_rn(rows2[j][k], make_float2(uu[2 * k], uu[2 * k + 1]), da);
                if (k + 1 < VRP / 2)
                    db = __ffma2_rn(rows2[j][k + 1], make_float2(uu[2 * k + 2], uu[2 * k + 3]), db);
            }
            const float dot = (da.x + da.y) + (db.x + db.y);
            const bool valid = cv[j] > 0.f;
            tiny_any |= valid && !(dot >= 0x1p-100f);
            const float tau = valid ? __fdividef(cv[j], dot) : 0.f;
            const float2 t2 = make_float2(tau, tau);
#pragma unroll
            for (int k = 0; k < VRP / 2; ++k) acc2[k] = __ffma2_rn(t2, rows2[j][k], acc2[k]);
        }
#pragma unroll
        for (int k = 0; k < VRP / 2; ++k) {
            acc[2 * k] = acc2[k].x;
            acc[2 * k + 1] = acc2[k].y;
        }
        for (int x = 0; x < extra; ++x) {
            const int idx = p + G * (NPL + x);
            const int o = idx - 32 * NPL;
            const bool valid = idx < len;
            float kr[VRP];
            float cval;
            if (o < n_ovf) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float4 v = reinterpret_cast<const float4 *>(wrow + (size_t)o * VRP)[c];
                    kr[4 * c] = v.x; kr[4 * c + 1] = v.y; kr[4 * c + 2] = v.z; kr[4 * c + 3] = v.w;
                }
                cval = wc[o];
            } else {
                int2 e = make_int2(0, 0);
                if (valid) e = __ldg(a.nz + beg + idx);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float4 v = KIO<KT_t>::load4(KT, (long)e.x * C + c);
                    kr[4 * c] = v.x; kr[4 * c + 1] = v.y; kr[4 * c + 2] = v.z; kr[4 * c + 3] = v.w;
                }
                cval = __int_as_float(e.y);
            }
            float d4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < VRP; ++k) d4[k & 3] = fmaf(kr[k], uu[k], d4[k & 3]);
            const float dot = (d4[0] + d4[1]) + (d4[2] + d4[3]);
            tiny_any |= valid && !(dot >= 0x1p-100f);
            const float tau = valid ? __fdividef(cval, dot) : 0.f;
#pragma unroll
            for (int k = 0; k < VRP; ++k) acc[k] = fmaf(tau, kr[k], acc[k]);
        }
        if (__any_sync(kFull, tiny_any)) {
            SWMD_COLD_PATH();
            // some K^T u fell below 2^-100: redo this lane's accumulation with the
            // affected denominators in FP64 (rows held in registers; an overflow
            // row always comes with a full-warp team and is re-derived the same way)
#pragma unroll
            for (int k = 0; k < VRP; ++k) acc[k] = 0.f;
#pragma unroll
            for (int j = 0; j < NPL; ++j) {
                float d4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int k = 0; k < VRP; ++k) d4[k & 3] = fmaf(row_at(rows2[j], k), uu[k], d4[k & 3]);
                const float dot = (d4[0] + d4[1]) + (d4[2] + d4[3]);
                const bool valid = cv[j] > 0.f;
                float tau = valid ? __fdividef(cv[j], dot) : 0.f;
                if (valid && !(dot >= 0x1p-100f)) {
                    double s = 0.0;
#pragma unroll
                    for (int k = 0; k < VRP; ++k) s = fma((double)row_at(rows2[j], k), (double)uu[k], s);
                    tau = s > 0.0 ? (float)((double)cv[j] / s) : 0.f;
                    atomicOr(status, s > 0.0 ? ST_GUARD : ST_NUMERIC);
                }
#pragma unroll
                for (int k = 0; k < VRP; ++k) acc[k] = fmaf(tau, row_at(rows2[j], k), acc[k]);
            }
            for (int x = 0; x < extra; ++x) {
                const int idx = p + G * (NPL + x);
                const bool valid = idx < len;
                int2 e = make_int2(0, 0);
                if (valid) e = __ldg(a.nz + beg + idx);
                float kr[VRP];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float4 v = KIO<KT_t>::load4(KT, (long)e.x * C + c);
                    kr[4 * c] = v.x; kr[4 * c + 1] = v.y; kr[4 * c + 2] = v.z; kr[4 * c + 3] = v.w;
                }
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < VRP; ++k) s = fma((double)kr[k], (double)uu[k], s);
                float tau = 0.f;
                if (valid) {
                    tau = s > 0.0 ? (float)((double)__int_as_float(e.y) / s) : 0.f;
                    if (!(s > 0.0)) atomicOr(status, ST_NUMERIC);
                }
#pragma unroll
                for (int k = 0; k < VRP; ++k) acc[k] = fmaf(tau, kr[k], acc[k]);
            }
        }
        bool bad = false;
        if constexpr (G == 1) {
#pragma unroll
            for (int k = 0; k < VRP; ++k) {
                const float nu = rk[k] > 0.f ? __fdividef(rk[k], acc[k]) : 0.f;
                bad |= !(nu < INFINITY);
                uu[k] = nu;
            }
        } else {
            // team reduction of acc: store the partials, finish entries k = p + G i,
            // publish them in place of the first partial row, read the new u back
#pragma unroll
            for (int k = 0; k < VRP; ++k) tacc[p * kRowStride + k] = acc[k];
            __syncwarp();
            float nu[KS];
#pragma unroll
            for (int i = 0; i < KS; ++i) {
                const int k = p + G * i;
                float s = 0.f;
                if (k < VRP) {
#pragma unroll
                    for (int g = 0; g < G; ++g) s += tacc[g * kRowStride + k];
                }
                nu[i] = rk[i] > 0.f ? __fdividef(rk[i], s) : 0.f;
                bad |= !(nu[i] < INFINITY);
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < KS; ++i) {
                const int k = p + G * i;
                if (k < VRP) tacc[k] = nu[i];
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < VRP; ++k) uu[k] = tacc[k];
            __syncwarp();
        }
        if (bad) atomicOr(status, ST_NUMERIC);
    }

    // final step: s = K^T[w].u and m = KM^T[w].u per nonzero, WMD = sum c m / s
    double dist = 0.0;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
        float d4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < VRP; ++k) d4[k & 3] = fmaf(row_at(rows2[j], k), uu[k], d4[k & 3]);
        const float dot = (d4[0] + d4[1]) + (d4[2] + d4[3]);
        const bool valid = cv[j] > 0.f;
        float m4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float4 v = valid ? KIO<KT_t>::load4(KMT, (long)wid[j] * C + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            m4[0] = fmaf(v.x, uu[4 * c], m4[0]);
            m4[1] = fmaf(v.y, uu[4 * c + 1], m4[1]);
            m4[2] = fmaf(v.z, uu[4 * c + 2], m4[2]);
            m4[3] = fmaf(v.w, uu[4 * c + 3], m4[3]);
        }
        const float dm = (m4[0] + m4[1]) + (m4[2] + m4[3]);
        if (valid) {
            if (dot >= 0x1p-100f) {
                dist += (double)(cv[j] * (dm / dot));
            } else {
                SWMD_COLD_PATH();
                double s = 0.0, m = 0.0;
#pragma unroll
                for (int k = 0; k < VRP; ++k) s = fma((double)row_at(rows2[j], k), (double)uu[k], s);
                for (int c = 0; c < C; ++c) {
                    const float4 v = KIO<KT_t>::load4(KMT, (long)wid[j] * C + c);
                    m = fma((double)v.x, (double)uu[4 * c], m);
                    m = fma((double)v.y, (double)uu[4 * c + 1], m);
                    m = fma((double)v.z, (double)uu[4 * c + 2], m);
                    m = fma((double)v.w, (double)uu[4 * c + 3], m);
                }
                dist += (double)cv[j] * (m / s);
                atomicOr(status, s > 0.0 ? ST_GUARD : ST_NUMERIC);
            }
        }
    }
    for (int x = 0; x < extra; ++x) {
        const int idx = p + G * (NPL + x);
        const bool valid = idx < len;
        int2 e = make_int2(0, 0);
        if (valid) e = __ldg(a.nz + beg + idx);
        float d4[4] = {0.f, 0.f, 0.f, 0.f}, m4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float4 v = KIO<KT_t>::load4(KT, (long)e.x * C + c);
            const float4 m = KIO<KT_t>::load4(KMT, (long)e.x * C + c);
            d4[0] = fmaf(v.x, uu[4 * c], d4[0]); d4[1] = fmaf(v.y, uu[4 * c + 1], d4[1]);
            d4[2] = fmaf(v.z, uu[4 * c + 2], d4[2]); d4[3] = fmaf(v.w, uu[4 * c + 3], d4[3]);
            m4[0] = fmaf(m.x, uu[4 * c], m4[0]); m4[1] = fmaf(m.y, uu[4 * c + 1], m4[1]);
            m4[2] = fmaf(m.z, uu[4 * c + 2], m4[2]); m4[3] = fmaf(m.w, uu[4 * c + 3], m4[3]);
        }
        const float dot = (d4[0] + d4[1]) + (d4[2] + d4[3]);
        const float dm = (m4[0] + m4[1]) + (m4[2] + m4[3]);
        if (valid) {
            if (!(dot >= 0x1p-100f)) atomicOr(status, ST_NUMERIC);
            dist += (double)(__int_as_float(e.y) * (dm / dot));
        }
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) dist += __shfl_xor_sync(kFull, dist, o);
    if (has && p == 0) {
        if (!(fabs(dist) < INFINITY)) atomicOr(status, ST_NUMERIC);
        out[__ldg(a.doc_orig + doc)] = dist;
    }
    __syncwarp();   // the next task reuses the warp's shared buffers
}

template <int VRP, int NPL, class KT_t>
__device__ __noinline__ void k_resident_regs_body(const ResidentArgs &ra, const int4 *tasks, int n_tasks, int ovf_cap) {
    // one copy of the arguments (the fields are read in every task; through the
    // reference they were loaded again each time: 72 -> 63 us on the paper-shaped query)
    const IterArgs a = ra.it;
    // per warp: the transpose buffer (32 partial rows, stride kRowStride)
    constexpr int WACC = 32 * kRowStride;
    __shared__ __align__(16) float s_acc[kWarps][WACC];
    extern __shared__ __align__(16) float s_ovf[];   // per warp: overflow rows, then their counts
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float *wacc = s_acc[warp];
    float *wrow = s_ovf + (size_t)warp * ovf_cap * (VRP + 1);
    float *wc = wrow + (size_t)ovf_cap * VRP;
    const long gwarp = ((long)blockIdx.x * kRegThreads + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * kRegThreads) >> 5;
    for (long task = gwarp; task < n_tasks; task += nwarps) {
        const int4 tk = __ldg(tasks + task);   // first document, team size, documents
        switch (tk.y) {
            case 1: regs_task<VRP, NPL, 1, KT_t>(a, ra.t, tk, lane, wacc, wrow, wc, ovf_cap); break;
            case 2: regs_task<VRP, NPL, 2, KT_t>(a, ra.t, tk, lane, wacc, wrow, wc, ovf_cap); break;
            case 4: regs_task<VRP, NPL, 4, KT_t>(a, ra.t, tk, lane, wacc, wrow, wc, ovf_cap); break;
            case 8: regs_task<VRP, NPL, 8, KT_t>(a, ra.t, tk, lane, wacc, wrow, wc, ovf_cap); break;
            case 16: regs_task<VRP, NPL, 16, KT_t>(a, ra.t, tk, lane, wacc, wrow, wc, ovf_cap); break;
            default: regs_task<VRP, NPL, 32, KT_t>(a, ra.t, tk, lane, wacc, wrow, wc, ovf_cap); break;
        }
    }
}

template <int VRP, int NPL, class KT_t>
__global__ void __launch_bounds__(kRegThreads)
k_resident_regs(const __grid_constant__ ResidentArgs ra0, const ResidentArgs *batch, const int4 *tasks,
                int n_tasks, int ovf_cap) {
    // one query per grid row when batched (batch[blockIdx.y]), else the argument
    if (batch) k_resident_regs_body<VRP, NPL, KT_t>(batch[blockIdx.y], tasks, n_tasks, ovf_cap);
    else k_resident_regs_body<VRP, NPL, KT_t>(ra0, tasks, n_tasks, ovf_cap);
}

template <int VRP, int NPL, class KT_t>
cudaError_t run_regs(const ResidentArgs &a, const TaskSet &ts, int sms, cudaStream_t s, int nq,
                     const ResidentArgs *batch) {
    auto kern = k_resident_regs<VRP, NPL, KT_t>;
    // overflow buffer: rows beyond 32 * NPL of the longest document, at most 40 KB per warp
    int ovf = ts.max_len - 32 * NPL;
    const int cap_rows = (40 * 1024) / ((VRP + 1) * 4);
    if (ovf < 0) ovf = 0;
    if (ovf > cap_rows) ovf = cap_rows;
    ovf = (ovf + 3) / 4 * 4;   // keeps every warp's buffer 16-byte aligned
    const size_t smem = (size_t)kWarps * ovf * (VRP + 1) * sizeof(float);
    static LaunchCache cache;
    int per_sm = 1;
    cudaError_t e = cache.blocks_per_sm(kern, kRegThreads, smem, -1, &per_sm);
    if (e != cudaSuccess) return e;
    long blocks = ((long)ts.n_tasks + kWarps - 1) / kWarps;
    long cap = ((long)sms * per_sm * 2 + nq - 1) / nq;   // resident blocks shared by the queries
    if (cap < 1) cap = 1;
    if (nq == 1) cap = (long)sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks > 0)
        kern<<<dim3((unsigned)blocks, (unsigned)nq), kRegThreads, smem, s>>>(a, batch, ts.tasks,
                                                                           ts.n_tasks, ovf);
    return cudaGetLastError();
}

template <class KT_t>
cudaError_t dispatch_regs(const ResidentArgs &a, int vrp, const TaskSet &ts, int sms, cudaStream_t s,
                          int nq, const ResidentArgs *batch) {
    switch (vrp * 100 + ts.npl) {
#define SWMD_R(V, N) \
    case V * 100 + N: return run_regs<V, N, KT_t>(a, ts, sms, s, nq, batch);
        SWMD_R(4, 8) SWMD_R(8, 8) SWMD_R(12, 4) SWMD_R(16, 4) SWMD_R(20, 4) SWMD_R(24, 2)
        SWMD_R(28, 2) SWMD_R(32, 2) SWMD_R(12, 8) SWMD_R(16, 2) SWMD_R(20, 2) SWMD_R(20, 3)
        SWMD_R(24, 3) SWMD_R(32, 1) SWMD_R(24, 4)
#undef SWMD_R
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace swmd
