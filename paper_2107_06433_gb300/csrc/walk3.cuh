// The per-iteration walk over the sliced nonzero layout: the fused SDDMM-SpMM
// iteration (Section III-C, SDDMM_SpMM type 1), the unfused SDDMM / SpMM pair
// (Algorithms 2 and 3) and the final step (type 2 and the distance).
//
// Layout.  Documents (internal order: decreasing length) are grouped in slices of
// 32; slice s stores its nonzeros row by row, entry (i, t) -- the i-th nonzero of
// the slice's t-th document -- at slice_ptr[s] + 32 i + t, with (0, c = 0) where
// a document has fewer than the slice's longest length.  A warp walking some
// documents of one slice reads their i-th nonzeros with one coalesced load.
//
// Lanes.  A K^T row is VRP values; lane tl of a team of Q = VRP / P lanes holds
// the P consecutive values [tl P, tl P + P) of every row, of u_j and of the SpMM
// accumulator, so a row is read by one wide load per lane (32 bytes for P = 8 in
// FP32 or P = 16 in 16-bit storage) and one load instruction of the warp covers
// whole rows.  The dot K^T[w].u_j is finished with a butterfly over the Q lanes
// (log2 Q shuffles); acc += tau K^T[w] needs no exchange.  A warp owns 32 / Q
// documents of one slice, so every lane of a warp walks the same number of rows.
// A document's arithmetic depends on its own nonzeros only, not on the other
// documents of its slice, launch or partition.
#pragma once

#include "walk.cuh"

namespace swmd {

constexpr int kWalk3Threads = 256;
constexpr int kSlice = kSliceDocs;

template <int VRP, class KT_t>
struct W3 {
    static constexpr int EB = (int)sizeof(KT_t);
    static constexpr int P = VRP * EB >= 32 ? 32 / EB : VRP;   // values per lane
    static constexpr int Q = VRP / P;                            // lanes per document
    static constexpr int WORDS = P * EB / 4;                     // 32-bit words per lane and row
    static constexpr int TPW = 32 / Q;                           // documents per warp
    static constexpr int RB = 4;                                 // rows per batch
    static constexpr int ROWS = Q > RB ? Q : RB;                 // rows per group
    static constexpr int EPL = ROWS / Q;                         // entries loaded per lane per group
    static_assert(P % 2 == 0 && WORDS >= 2 && WORDS <= 8, "lane slice of 8 to 32 bytes");
    static_assert((Q & (Q - 1)) == 0 && Q <= 32, "team must be a power of two");
};

// WORDS 32-bit words from global memory, read-only path, one vector load.
template <int WORDS>
__device__ __forceinline__ void load_words(const void *p, uint32_t (&w)[WORDS]) {
    if constexpr (WORDS == 8) {
        asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                       "=r"(w[6]), "=r"(w[7])
                     : "l"(p));
    } else if constexpr (WORDS == 4) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        w[0] = v.x; w[1] = v.y;
    }
}

// Values 2i and 2i+1 of a lane slice held as raw words.
template <class KT_t>
__device__ __forceinline__ float2 pair_of(const uint32_t *w, int i);
template <>
__device__ __forceinline__ float2 pair_of<float>(const uint32_t *w, int i) {
    return make_float2(__uint_as_float(w[2 * i]), __uint_as_float(w[2 * i + 1]));
}
template <>
__device__ __forceinline__ float2 pair_of<__nv_bfloat16>(const uint32_t *w, int i) {
    // a bfloat16 is the upper half of the float with the same value
    return make_float2(__uint_as_float(w[i] << 16), __uint_as_float(w[i] & 0xffff0000u));
}
template <>
__device__ __forceinline__ float2 pair_of<__half>(const uint32_t *w, int i) {
    __half2 h;
    memcpy(&h, &w[i], sizeof h);
    return __half22float2(h);
}

template <int P>
__device__ __forceinline__ void load_floats(const float *p, float (&v)[P]) {
#pragma unroll
    for (int i = 0; i < P / 4; ++i) {
        const float4 f = reinterpret_cast<const float4 *>(p)[i];
        v[4 * i] = f.x; v[4 * i + 1] = f.y; v[4 * i + 2] = f.z; v[4 * i + 3] = f.w;
    }
}

template <int VRP, class KT_t, Kind KIND>
__global__ void __launch_bounds__(kWalk3Threads) k_walk3(IterArgs a) {
    using C = W3<VRP, KT_t>;
    constexpr int P = C::P, Q = C::Q, WORDS = C::WORDS, TPW = C::TPW, RB = C::RB;
    constexpr int ROWS = C::ROWS, EPL = C::EPL;
    constexpr bool kDots = KIND != Kind::Spmm;

    const int lane = threadIdx.x & 31;
    const int tl = lane & (Q - 1);
    const int team = lane / Q;
    const int lead = lane & ~(Q - 1);
    const long warp_global = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    const int vr = a.qp->vr;
    const float u0 = a.qp->u0;
    int *const status = a.qp->status;
    double *const out = a.out ? a.out : a.qp->out;
    const char *KT = reinterpret_cast<const char *>(a.KT);
    const char *KMT = reinterpret_cast<const char *>(a.KMT);
    constexpr long kRowBytes = (long)VRP * C::EB;
    const long lane_off = (long)tl * P * C::EB;
    const long n_groups = (long)a.n_slices * Q;

    for (long g = warp_global; g < n_groups; g += nwarps) {
        const int s = (int)(g / Q);
        const int t = (int)(g - (long)s * Q) * TPW + team;   // document within the slice
        const long ld = (long)s * kSlice + t;                  // local document
        const bool has = ld < a.N;
        const int sbeg = __ldg(a.slice_ptr + s);
        const int Ls = (__ldg(a.slice_ptr + s + 1) - sbeg) / kSlice;
        const int2 *ent = a.slice_nz + sbeg + t;

        float u[P];
        if constexpr (kDots) {
            if (a.first) {
#pragma unroll
                for (int p = 0; p < P; ++p) u[p] = has && tl * P + p < vr ? u0 : 0.f;
            } else if (has) {
                load_floats<P>(a.u + ld * VRP + tl * P, u);
            } else {
#pragma unroll
                for (int p = 0; p < P; ++p) u[p] = 0.f;
            }
        }
        float2 acc[P / 2];
#pragma unroll
        for (int p = 0; p < P / 2; ++p) acc[p] = make_float2(0.f, 0.f);
        double dist = 0.0;

        // entries of the first group; the next group's are fetched while this one runs
        int2 e[EPL];
        float ev[EPL];
#pragma unroll
        for (int j = 0; j < EPL; ++j) {
            const int i = j * Q + tl;
            e[j] = i < Ls ? __ldg(ent + (long)i * kSlice) : make_int2(0, 0);
            if constexpr (KIND == Kind::Spmm) ev[j] = i < Ls ? __ldg(a.v + sbeg + (long)i * kSlice + t) : 0.f;
        }
        for (int i0 = 0; i0 < Ls; i0 += ROWS) {
            int2 en[EPL];
            float evn[EPL];
#pragma unroll
            for (int j = 0; j < EPL; ++j) {
                const int i = i0 + ROWS + j * Q + tl;
                en[j] = i < Ls ? __ldg(ent + (long)i * kSlice) : make_int2(0, 0);
                if constexpr (KIND == Kind::Spmm)
                    evn[j] = i < Ls ? __ldg(a.v + sbeg + (long)i * kSlice + t) : 0.f;
            }
#pragma unroll
            for (int b = 0; b < ROWS / RB; ++b) {
                int wv[RB];
                float cv[RB], tv[RB];
#pragma unroll
                for (int rr = 0; rr < RB; ++rr) {
                    const int ri = b * RB + rr, j = ri / Q, q = ri % Q;
                    if constexpr (Q == 1) {
                        wv[rr] = e[j].x;
                        cv[rr] = __int_as_float(e[j].y);
                        if constexpr (KIND == Kind::Spmm) tv[rr] = ev[j];
                    } else {
                        wv[rr] = __shfl_sync(kFull, e[j].x, lead + q);
                        cv[rr] = __shfl_sync(kFull, __int_as_float(e[j].y), lead + q);
                        if constexpr (KIND == Kind::Spmm) tv[rr] = __shfl_sync(kFull, ev[j], lead + q);
                    }
                }
                uint32_t kw[RB][WORDS];
#pragma unroll
                for (int rr = 0; rr < RB; ++rr) {
                    if (cv[rr] != 0.f) {
                        load_words<WORDS>(KT + (long)wv[rr] * kRowBytes + lane_off, kw[rr]);
                    } else {
#pragma unroll
                        for (int x = 0; x < WORDS; ++x) kw[rr][x] = 0u;
                    }
                }
                float tau[RB];
                if constexpr (KIND == Kind::Spmm) {
#pragma unroll
                    for (int rr = 0; rr < RB; ++rr) tau[rr] = cv[rr] != 0.f ? tv[rr] : 0.f;
                } else {
                    float d[RB];
#pragma unroll
                    for (int rr = 0; rr < RB; ++rr) {
                        float2 d2 = make_float2(0.f, 0.f);
#pragma unroll
                        for (int p = 0; p < P / 2; ++p)
                            d2 = __ffma2_rn(pair_of<KT_t>(kw[rr], p), make_float2(u[2 * p], u[2 * p + 1]), d2);
                        d[rr] = d2.x + d2.y;
                    }
                    float dm[KIND == Kind::Final ? RB : 1];
                    uint32_t mw[KIND == Kind::Final ? RB : 1][WORDS];
                    if constexpr (KIND == Kind::Final) {
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) {
                            if (cv[rr] != 0.f) {
                                load_words<WORDS>(KMT + (long)wv[rr] * kRowBytes + lane_off, mw[rr]);
                            } else {
#pragma unroll
                                for (int x = 0; x < WORDS; ++x) mw[rr][x] = 0u;
                            }
                            float2 m2 = make_float2(0.f, 0.f);
#pragma unroll
                            for (int p = 0; p < P / 2; ++p)
                                m2 = __ffma2_rn(pair_of<KT_t>(mw[rr], p), make_float2(u[2 * p], u[2 * p + 1]), m2);
                            dm[rr] = m2.x + m2.y;
                        }
                    }
#pragma unroll
                    for (int o = 1; o < Q; o <<= 1) {
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) {
                            d[rr] += __shfl_xor_sync(kFull, d[rr], o);
                            if constexpr (KIND == Kind::Final) dm[rr] += __shfl_xor_sync(kFull, dm[rr], o);
                        }
                    }
                    bool tiny = false;
#pragma unroll
                    for (int rr = 0; rr < RB; ++rr) tiny |= cv[rr] != 0.f && !(d[rr] >= 0x1p-100f);
                    double fix[RB];
                    unsigned fixed = 0;
                    if (__any_sync(kFull, tiny)) {
                        SWMD_COLD_PATH();
                        // K^T u below 2^-100 somewhere in the warp: this batch's dots
                        // again in FP64 from the same, exactly widened values
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) {
                            double sd = 0.0, md = 0.0;
#pragma unroll
                            for (int p = 0; p < P / 2; ++p) {
                                const float2 k2 = pair_of<KT_t>(kw[rr], p);
                                sd += (double)k2.x * u[2 * p] + (double)k2.y * u[2 * p + 1];
                                if constexpr (KIND == Kind::Final) {
                                    const float2 m2 = pair_of<KT_t>(mw[rr], p);
                                    md += (double)m2.x * u[2 * p] + (double)m2.y * u[2 * p + 1];
                                }
                            }
#pragma unroll
                            for (int o = 1; o < Q; o <<= 1) {
                                sd += __shfl_xor_sync(kFull, sd, o);
                                if constexpr (KIND == Kind::Final) md += __shfl_xor_sync(kFull, md, o);
                            }
                            if (cv[rr] != 0.f && !(d[rr] >= 0x1p-100f)) {
                                if constexpr (KIND == Kind::Final) fix[rr] = (double)cv[rr] * (md / sd);
                                else fix[rr] = sd > 0.0 ? (double)cv[rr] / sd : 0.0;
                                fixed |= 1u << rr;
                                if (tl == 0) atomicOr(status, sd > 0.0 ? ST_GUARD : ST_NUMERIC);
                            }
                        }
                    }
                    if constexpr (KIND == Kind::Final) {
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr)
                            if (cv[rr] != 0.f)
                                dist += (fixed >> rr & 1u) ? fix[rr] : (double)(cv[rr] * (dm[rr] / d[rr]));
                        continue;
                    } else {
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) {
                            tau[rr] = cv[rr] != 0.f ? __fdividef(cv[rr], d[rr]) : 0.f;
                            if (fixed >> rr & 1u) tau[rr] = (float)fix[rr];
                        }
                    }
                    if constexpr (KIND == Kind::Sddmm) {
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) {
                            const int ri = b * RB + rr, q = ri % Q;
                            const int i = i0 + ri;
                            if (tl == q && cv[rr] != 0.f) a.v[sbeg + (long)i * kSlice + t] = tau[rr];
                        }
                        continue;
                    }
                }
                // acc += tau K^T[w] over this lane's P values
#pragma unroll
                for (int rr = 0; rr < RB; ++rr) {
                    const float2 t2 = make_float2(tau[rr], tau[rr]);
#pragma unroll
                    for (int p = 0; p < P / 2; ++p) acc[p] = __ffma2_rn(t2, pair_of<KT_t>(kw[rr], p), acc[p]);
                }
            }
#pragma unroll
            for (int j = 0; j < EPL; ++j) {
                e[j] = en[j];
                if constexpr (KIND == Kind::Spmm) ev[j] = evn[j];
            }
        }

        if constexpr (KIND == Kind::Fused || KIND == Kind::Spmm) {
            if (has) {
                float rr[P], nu[P];
                load_floats<P>(a.r + tl * P, rr);
                bool bad = false;
#pragma unroll
                for (int p = 0; p < P / 2; ++p) {
                    const int k = tl * P + 2 * p;
                    nu[2 * p] = k < vr ? __fdividef(rr[2 * p], acc[p].x) : 0.f;
                    nu[2 * p + 1] = k + 1 < vr ? __fdividef(rr[2 * p + 1], acc[p].y) : 0.f;
                    bad |= !(nu[2 * p] < INFINITY) || !(nu[2 * p + 1] < INFINITY);
                }
                if (bad) atomicOr(status, ST_NUMERIC);
                float *dst = a.u + ld * VRP + tl * P;
#pragma unroll
                for (int i = 0; i < P / 4; ++i)
                    reinterpret_cast<float4 *>(dst)[i] =
                        make_float4(nu[4 * i], nu[4 * i + 1], nu[4 * i + 2], nu[4 * i + 3]);
            }
        } else if constexpr (KIND == Kind::Final) {
            // every lane of the team holds the same sum (the dots were all-reduced)
            if (has && tl == 0) {
                if (!(fabs(dist) < INFINITY)) atomicOr(status, ST_NUMERIC);
                out[__ldg(a.doc_orig + ld)] = dist;
            }
        }
    }
}

template <int VRP, class KT_t, Kind KIND>
cudaError_t run_walk3(const IterArgs &a, int sms, cudaStream_t s) {
    auto kern = k_walk3<VRP, KT_t, KIND>;
    static int per_sm = 0;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWalk3Threads, 0) != cudaSuccess ||
            per_sm < 1) {
            (void)cudaGetLastError();
            per_sm = 1;
        }
    }
    constexpr int Q = W3<VRP, KT_t>::Q;
    const long groups = (long)a.n_slices * Q;
    const long need = (groups * 32 + kWalk3Threads - 1) / kWalk3Threads;
    long blocks = (long)sms * per_sm;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (a.N > 0) kern<<<(unsigned)blocks, kWalk3Threads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class KT_t, Kind KIND>
cudaError_t dispatch_walk3(const IterArgs &a, int vrp, int sms, cudaStream_t s) {
    switch (vrp) {
        case 4: return run_walk3<4, KT_t, KIND>(a, sms, s);
        case 8: return run_walk3<8, KT_t, KIND>(a, sms, s);
        case 16: return run_walk3<16, KT_t, KIND>(a, sms, s);
        case 32: return run_walk3<32, KT_t, KIND>(a, sms, s);
        case 64: return run_walk3<64, KT_t, KIND>(a, sms, s);
        case 128: return run_walk3<128, KT_t, KIND>(a, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

template <Kind KIND>
cudaError_t dispatch_walk3_prec(const IterArgs &a, int vrp, int kprec, int sms, cudaStream_t s) {
    switch (kprec) {
        case 0: return dispatch_walk3<float, KIND>(a, vrp, sms, s);
        case 1: return dispatch_walk3<__nv_bfloat16, KIND>(a, vrp, sms, s);
        case 2: return dispatch_walk3<__half, KIND>(a, vrp, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace swmd
