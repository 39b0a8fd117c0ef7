// The per-iteration walk with lanes over the query words (k), for the fused
// SDDMM-SpMM iteration, the unfused SDDMM / SpMM pair and the final step.
//
// Section III-C's SDDMM_SpMM reads, per nonzero (w, c_wj) of document j, the row
// K^T[w] twice: once for s = K^T[w].u_j (SDDMM) and once for acc += tau K^T[w]
// (SpMM).  A K^T row is VRP contiguous values; here a team of Q = VRP / 4 lanes
// owns a document and lane q holds the float4 slice q of every row, u_j and acc,
// so the team reads each row as one contiguous piece and the SpMM accumulation
// acc[k] is complete in the lane that owns k (no cross-lane reduction of acc).
// Only the dots need combining: rows are taken R at a time, the R partial dots
// are reduce-scattered across the Q lanes (each lane finishes R / Q of them and
// divides c by them), then the R values of tau are all-gathered.
#pragma once

#include "walk.cuh"

namespace swmd {

constexpr int kWalk2Threads = 256;

// v[0..R): per-lane partial sums of R values over a team of Q lanes (Q a power of
// two, lanes of a team consecutive).  On return v[0..R/Q) hold complete sums of
// values b*(R/Q) .. (b+1)*(R/Q)-1 where b = lane-in-team (R >= Q), or, if R < Q,
// v[0] holds the complete sum of value lane-in-team / (Q / R).
template <int R, int Q>
__device__ __forceinline__ void team_reduce_scatter(float (&v)[R], int tl) {
    int n = R;
#pragma unroll
    for (int o = Q / 2; o >= 1; o >>= 1) {
        if (n > 1) {
            const bool up = (tl & o) != 0;
#pragma unroll
            for (int i = 0; i < R / 2; ++i) {
                if (i < n / 2) {
                    const float keep = up ? v[i + n / 2] : v[i];
                    const float send = up ? v[i] : v[i + n / 2];
                    v[i] = keep + __shfl_xor_sync(kFull, send, o);
                }
            }
            n >>= 1;
        } else {
            v[0] += __shfl_xor_sync(kFull, v[0], o);
        }
    }
}

// Inverse of team_reduce_scatter's layout: every lane ends with all R values.
template <int R, int Q>
__device__ __forceinline__ void team_all_gather(float (&v)[R], int tl) {
    constexpr int M0 = R >= Q ? R / Q : 1;   // values per lane after the scatter
    constexpr int O0 = R >= Q ? 1 : Q / R;   // lanes that share one value
    int m = M0;
#pragma unroll
    for (int o = O0; o < Q; o <<= 1) {
        const bool up = (tl & o) != 0;
        float tmp[R];
#pragma unroll
        for (int i = 0; i < R; ++i) tmp[i] = 0.f;
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            if (i < m) {
                const float other = __shfl_xor_sync(kFull, v[i], o);
                tmp[i] = up ? other : v[i];        // lower block: the partner's if mine is upper
                tmp[i + m] = up ? v[i] : other;
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (i < 2 * m) v[i] = tmp[i];
        m <<= 1;
    }
}

// arr[idx] for a runtime idx without indexing a register array at run time
template <int R, class T>
__device__ __forceinline__ T pick(const T (&arr)[R], int idx) {
    T v = arr[0];
#pragma unroll
    for (int r = 1; r < R; ++r)
        if (r == idx) v = arr[r];
    return v;
}

template <int VRP, class KT_t, Kind KIND>
__global__ void __launch_bounds__(kWalk2Threads) k_walk2(IterArgs a) {
    constexpr int Q = VRP / 4;                 // lanes per document, one float4 each
    constexpr int R = Q >= 16 ? 16 : 8;        // rows per chunk
    constexpr int TPW = 32 / Q;                // documents per warp
    constexpr int RL = R >= Q ? R / Q : 1;     // finished dots per lane per chunk
    static_assert(VRP % 4 == 0 && (Q & (Q - 1)) == 0 && Q <= 32, "VRP / 4 must be a power of two");

    const int lane = threadIdx.x & 31;
    const int tl = lane & (Q - 1);
    const int team = lane / Q;
    const long warp_global = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    const int vr = a.qp->vr;
    const float u0 = a.qp->u0;
    int *const status = a.qp->status;
    double *const out = a.out ? a.out : a.qp->out;
    const KT_t *KT = reinterpret_cast<const KT_t *>(a.KT);
    const KT_t *KMT = reinterpret_cast<const KT_t *>(a.KMT);
    // the rows this lane finishes in a chunk: its block of the reduce-scatter
    const int my0 = R >= Q ? tl * RL : tl / (Q / R);

    for (long base = warp_global * TPW; base < a.N; base += nwarps * TPW) {
        const long doc = a.doc0 + base + team;
        const bool has = base + team < a.N;
        int beg = 0, len = 0;
        if (has) {
            beg = __ldg(a.doc_ptr + doc);
            len = __ldg(a.doc_ptr + doc + 1) - beg;
        }
        int chunks = (len + R - 1) / R;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) chunks = max(chunks, __shfl_xor_sync(kFull, chunks, o));

        float4 u4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (KIND != Kind::Spmm) {
            if (a.first) {
                const int k0 = 4 * tl;
                u4 = make_float4(has && k0 < vr ? u0 : 0.f, has && k0 + 1 < vr ? u0 : 0.f,
                                 has && k0 + 2 < vr ? u0 : 0.f, has && k0 + 3 < vr ? u0 : 0.f);
            } else if (has) {
                u4 = reinterpret_cast<const float4 *>(a.u + doc * VRP)[tl];
            }
        }
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        double dist = 0.0;

        for (int ch = 0; ch < chunks; ++ch) {
            const int i0 = ch * R;
            float cv[R];
            int wv[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bool valid = i0 + r < len;
                const int2 e = valid ? __ldg(a.nz + beg + i0 + r) : make_int2(0, 0);
                wv[r] = e.x;
                cv[r] = valid ? __int_as_float(e.y) : 0.f;
            }
            float4 ks[R];
#pragma unroll
            for (int r = 0; r < R; ++r)
                ks[r] = cv[r] > 0.f ? KIO<KT_t>::load4(KT, (long)wv[r] * Q + tl)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);

            if constexpr (KIND == Kind::Spmm) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float tau = cv[r] > 0.f ? __ldg(a.v + beg + i0 + r) : 0.f;
                    acc.x = fmaf(tau, ks[r].x, acc.x); acc.y = fmaf(tau, ks[r].y, acc.y);
                    acc.z = fmaf(tau, ks[r].z, acc.z); acc.w = fmaf(tau, ks[r].w, acc.w);
                }
                continue;
            }

            // partial dots s_r = K^T[w_r] . u over this lane's four k
            float d[R];
#pragma unroll
            for (int r = 0; r < R; ++r)
                d[r] = fmaf(ks[r].x, u4.x, fmaf(ks[r].y, u4.y, fmaf(ks[r].z, u4.z, ks[r].w * u4.w)));
            float dm[KIND == Kind::Final ? R : 1];
            if constexpr (KIND == Kind::Final) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float4 m = cv[r] > 0.f ? KIO<KT_t>::load4(KMT, (long)wv[r] * Q + tl)
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
                    dm[r] = fmaf(m.x, u4.x, fmaf(m.y, u4.y, fmaf(m.z, u4.z, m.w * u4.w)));
                }
                team_reduce_scatter<R, Q>(dm, tl);
            }
            team_reduce_scatter<R, Q>(d, tl);

            // this lane's finished rows: r = my0 + i (values picked without
            // run-time indexing of the register arrays)
            float cmine[RL];
#pragma unroll
            for (int i = 0; i < RL; ++i) cmine[i] = pick<R>(cv, my0 + i);
            bool tiny = false;
#pragma unroll
            for (int i = 0; i < RL; ++i) tiny |= cmine[i] > 0.f && !(d[i] >= 0x1p-100f);
            double fix[RL];       // FP64 replacement of a tiny row's tau (or contribution)
            unsigned fixed = 0;
            if (__any_sync(kFull, tiny)) {
                SWMD_COLD_PATH();
                // K^T u below 2^-100 somewhere in the warp: every dot of the chunk
                // again in FP64 from the same, exactly widened inputs
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    double s = (double)ks[r].x * u4.x + (double)ks[r].y * u4.y +
                               (double)ks[r].z * u4.z + (double)ks[r].w * u4.w;
                    double m = 0.0;
                    if constexpr (KIND == Kind::Final) {
                        const float4 km = cv[r] > 0.f ? KIO<KT_t>::load4(KMT, (long)wv[r] * Q + tl)
                                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                        m = (double)km.x * u4.x + (double)km.y * u4.y + (double)km.z * u4.z +
                            (double)km.w * u4.w;
                    }
#pragma unroll
                    for (int o = 1; o < Q; o <<= 1) {
                        s += __shfl_xor_sync(kFull, s, o);
                        if constexpr (KIND == Kind::Final) m += __shfl_xor_sync(kFull, m, o);
                    }
#pragma unroll
                    for (int i = 0; i < RL; ++i) {
                        if (r == my0 + i && cmine[i] > 0.f && !(d[i] >= 0x1p-100f)) {
                            if constexpr (KIND == Kind::Final) fix[i] = (double)cmine[i] * (m / s);
                            else fix[i] = s > 0.0 ? (double)cmine[i] / s : 0.0;
                            fixed |= 1u << i;
                            if (R >= Q || (tl % (Q / R)) == 0)
                                atomicOr(status, s > 0.0 ? ST_GUARD : ST_NUMERIC);
                        }
                    }
                }
            }

            if constexpr (KIND == Kind::Final) {
                // contributions of the finished rows; the team sum comes at the end
                if (R >= Q || (tl % (Q / R)) == 0) {
#pragma unroll
                    for (int i = 0; i < RL; ++i) {
                        if (cmine[i] > 0.f)
                            dist += (fixed >> i & 1u) ? fix[i] : (double)(cmine[i] * (dm[i] / d[i]));
                    }
                }
            } else {
                float tau[R];
#pragma unroll
                for (int i = 0; i < R; ++i) tau[i] = 0.f;
#pragma unroll
                for (int i = 0; i < RL; ++i) {
                    tau[i] = cmine[i] > 0.f ? __fdividef(cmine[i], d[i]) : 0.f;
                    if (fixed >> i & 1u) tau[i] = (float)fix[i];
                }
                if constexpr (KIND == Kind::Sddmm) {
                    if (R >= Q || (tl % (Q / R)) == 0) {
#pragma unroll
                        for (int i = 0; i < RL; ++i) {
                            const int r = my0 + i;
                            if (cmine[i] > 0.f) a.v[beg + i0 + r] = tau[i];
                        }
                    }
                } else {
                    team_all_gather<R, Q>(tau, tl);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        acc.x = fmaf(tau[r], ks[r].x, acc.x); acc.y = fmaf(tau[r], ks[r].y, acc.y);
                        acc.z = fmaf(tau[r], ks[r].z, acc.z); acc.w = fmaf(tau[r], ks[r].w, acc.w);
                    }
                }
            }
        }

        if constexpr (KIND == Kind::Fused || KIND == Kind::Spmm) {
            if (has) {
                const int k0 = 4 * tl;
                const float4 r4 = __ldg(reinterpret_cast<const float4 *>(a.r) + tl);
                float4 nu;
                nu.x = k0 < vr ? __fdividef(r4.x, acc.x) : 0.f;
                nu.y = k0 + 1 < vr ? __fdividef(r4.y, acc.y) : 0.f;
                nu.z = k0 + 2 < vr ? __fdividef(r4.z, acc.z) : 0.f;
                nu.w = k0 + 3 < vr ? __fdividef(r4.w, acc.w) : 0.f;
                if (!(nu.x < INFINITY && nu.y < INFINITY && nu.z < INFINITY && nu.w < INFINITY))
                    atomicOr(status, ST_NUMERIC);
                reinterpret_cast<float4 *>(a.u + doc * VRP)[tl] = nu;
            }
        } else if constexpr (KIND == Kind::Final) {
#pragma unroll
            for (int o = 1; o < Q; o <<= 1) dist += __shfl_xor_sync(kFull, dist, o);
            if (has && tl == 0) {
                if (!(fabs(dist) < INFINITY)) atomicOr(status, ST_NUMERIC);
                out[__ldg(a.doc_orig + doc)] = dist;
            }
        }
    }
}

template <int VRP, class KT_t, Kind KIND>
cudaError_t run_walk2(const IterArgs &a, int sms, cudaStream_t s) {
    auto kern = k_walk2<VRP, KT_t, KIND>;
    static int per_sm = 0;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWalk2Threads, 0) != cudaSuccess ||
            per_sm < 1) {
            (void)cudaGetLastError();
            per_sm = 1;
        }
    }
    constexpr int Q = VRP / 4;
    const long need = ((long)a.N * Q + kWalk2Threads - 1) / kWalk2Threads;
    long blocks = (long)sms * per_sm;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (a.N > 0) kern<<<(unsigned)blocks, kWalk2Threads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class KT_t, Kind KIND>
cudaError_t dispatch_walk2(const IterArgs &a, int vrp, int sms, cudaStream_t s) {
    switch (vrp) {
        case 4: return run_walk2<4, KT_t, KIND>(a, sms, s);
        case 8: return run_walk2<8, KT_t, KIND>(a, sms, s);
        case 16: return run_walk2<16, KT_t, KIND>(a, sms, s);
        case 32: return run_walk2<32, KT_t, KIND>(a, sms, s);
        case 64: return run_walk2<64, KT_t, KIND>(a, sms, s);
        case 128: return run_walk2<128, KT_t, KIND>(a, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

template <Kind KIND>
cudaError_t dispatch_walk2_prec(const IterArgs &a, int vrp, int kprec, int sms, cudaStream_t s) {
    switch (kprec) {
        case 0: return dispatch_walk2<float, KIND>(a, vrp, sms, s);
        case 1: return dispatch_walk2<__nv_bfloat16, KIND>(a, vrp, sms, s);
        case 2: return dispatch_walk2<__half, KIND>(a, vrp, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swmd
