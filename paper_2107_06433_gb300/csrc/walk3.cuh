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

#include <cfloat>
#include <type_traits>

#include "walk.cuh"

namespace swmd {

constexpr int kSlice = kSliceDocs;

template <int VRP, class KT_t>
struct W3 {
    static constexpr int EB = (int)sizeof(KT_t);
    static constexpr int P = VRP * EB >= 32 ? 32 / EB : VRP;   // values per lane
    static constexpr int Q = VRP / P;                            // lanes per document
    static constexpr int WORDS = P * EB / 4;                     // 32-bit words per lane and row
    static constexpr int TPW = 32 / Q;                           // documents per warp
    static constexpr int RB = 4;                                 // rows per batch
    static_assert(P % 2 == 0 && WORDS >= 2 && WORDS <= 8, "lane slice of 8 to 32 bytes");
    static_assert((Q & (Q - 1)) == 0 && Q <= 32, "team must be a power of two");
};

// L2 cache policies: the streamed arrays (c's entries, u) are read once per launch
// and would push the gathered K^T rows (re-read by every document that holds the
// word) out of L2; they are loaded evict-first and skip L1, K^T rows evict-last.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int2 ld_stream(const int2 *p, uint64_t pol) {
    int2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.s32 {%0, %1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *p, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_stream4(const float *p, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_stream4(float *p, float4 v, uint64_t pol) {
    asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
                 ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
}

// WORDS 32-bit words of a K^T row slice, read-only path, one vector load, kept in L2.
template <int WORDS>
__device__ __forceinline__ void load_words(const void *p, uint32_t (&w)[WORDS], uint64_t pol) {
    if constexpr (WORDS == 8) {
        asm volatile("ld.global.nc.L1::evict_last.L2::cache_hint.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                     : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                       "=r"(w[6]), "=r"(w[7])
                     : "l"(p), "l"(pol));
    } else if constexpr (WORDS == 4) {
        asm volatile("ld.global.nc.L1::evict_last.L2::cache_hint.v4.b32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                     : "l"(p), "l"(pol));
    } else {
        asm volatile("ld.global.nc.L1::evict_last.L2::cache_hint.v2.b32 {%0,%1}, [%2], %3;"
                     : "=r"(w[0]), "=r"(w[1])
                     : "l"(p), "l"(pol));
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

// The same widening as pair_of, written so the compiler cannot reuse (and keep
// live) the values pair_of produced earlier: for 16-bit rows that would hold
// twice the registers of the raw row across the whole batch.
template <class KT_t>
__device__ __forceinline__ float2 pair_again(const uint32_t *w, int i) {
    return pair_of<KT_t>(w, i);
}
template <>
__device__ __forceinline__ float2 pair_again<__nv_bfloat16>(const uint32_t *w, int i) {
    uint32_t lo, hi;
    asm volatile("shl.b32 %0, %2, 16;\n\tand.b32 %1, %2, 0xffff0000;" : "=r"(lo), "=r"(hi) : "r"(w[i]));
    return make_float2(__uint_as_float(lo), __uint_as_float(hi));
}
template <>
__device__ __forceinline__ float2 pair_again<__half>(const uint32_t *w, int i) {
    float x, y;
    asm volatile("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
                 : "=f"(x), "=f"(y) : "r"(w[i]));
    return make_float2(x, y);
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// 1/x from the SFU's approximate reciprocal (relative error about 2^-23;
// subnormal x flushes to zero, so 1/x is then infinite).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int P>
__device__ __forceinline__ void load_floats(const float *p, float (&v)[P]) {
#pragma unroll
    for (int i = 0; i < P / 4; ++i) {
        const float4 f = reinterpret_cast<const float4 *>(p)[i];
        v[4 * i] = f.x; v[4 * i + 1] = f.y; v[4 * i + 2] = f.z; v[4 * i + 3] = f.w;
    }
}

template <int VRP, class KT_t, Kind KIND, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_walk3(IterArgs a) {
    using C = W3<VRP, KT_t>;
    constexpr int P = C::P, Q = C::Q, WORDS = C::WORDS, TPW = C::TPW;
    constexpr int RB = C::RB;
    constexpr bool kDots = KIND != Kind::Spmm;

    const int lane = threadIdx.x & 31;
    const int tl = lane & (Q - 1);
    const int team = lane / Q;
    const long warp_global = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    const int vr = a.qp->vr;
    const float u0 = a.qp->u0;
    int *const status = a.qp->status;
    double *const out = a.out ? a.out : a.qp->out;
    constexpr long kRowBytes = (long)VRP * C::EB;
    const long lane_off = (long)tl * P * C::EB;
    const char *KTl = reinterpret_cast<const char *>(a.KT) + lane_off;
    const char *KMTl = reinterpret_cast<const char *>(a.KMT) + lane_off;
    const long n_groups = (long)a.n_slices * Q;
    const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
    // convergence mode: nothing to do once the previous iteration came below tol
    // (the same decision in every thread of the grid)
    if (KIND == Kind::Fused && a.tol > 0.f && a.it > 0 && __uint_as_float(a.conv[a.it]) < a.tol) return;
    float errmax = 0.f;   // convergence mode: largest |u (K v) - r| this lane saw

    // slice bounds of the warp's next group, loaded one group ahead
    int nb = 0, ne = 0;
    if (warp_global < n_groups) {
        const int s0 = (int)(warp_global / Q);
        nb = __ldg(a.slice_ptr + s0);
        ne = __ldg(a.slice_ptr + s0 + 1);
    }
    for (long g = warp_global; g < n_groups; g += nwarps) {
        const int s = (int)(g / Q);
        const int t = (int)(g - (long)s * Q) * TPW + team;   // document within the slice
        const long ld = (long)s * kSlice + t;                  // local document
        const bool has = ld < a.N;
        const int sbeg = nb;
        const int Ls = (ne - nb) / kSlice;
        const int2 *ent = a.slice_nz + sbeg + t;
        static_assert(kSliceRows % C::RB == 0, "slices hold whole batches");
        // The next group: its bounds now, its u_j (and, below, its first entries)
        // into L2 while this group runs.
        const long g2 = g + nwarps;
        const int s2 = (int)(g2 / Q);
        const int t2 = (int)(g2 - (long)s2 * Q) * TPW;
        if (g2 < n_groups) {
            nb = __ldg(a.slice_ptr + s2);
            ne = __ldg(a.slice_ptr + s2 + 1);
            const long ld2 = (long)s2 * kSlice + t2 + team;
            if (kDots && !a.first && ld2 < a.N) prefetch_l2(a.u + ld2 * VRP + tl * P);
        }

        // u_j's values of this lane as pairs (the operands of the packed FMA)
        float2 u[P / 2];
        if constexpr (kDots) {
            if (a.first) {
#pragma unroll
                for (int p = 0; p < P / 2; ++p)
                    u[p] = make_float2(has && tl * P + 2 * p < vr ? u0 : 0.f, has && tl * P + 2 * p + 1 < vr ? u0 : 0.f);
            } else if (has) {
                const float *src = a.u + ld * VRP + tl * P;
#pragma unroll
                for (int i = 0; i < P / 4; ++i) {
                    const float4 f = ld_stream4(src + 4 * i, pol_stream);
                    u[2 * i] = make_float2(f.x, f.y);
                    u[2 * i + 1] = make_float2(f.z, f.w);
                }
            } else {
#pragma unroll
                for (int p = 0; p < P / 2; ++p) u[p] = make_float2(0.f, 0.f);
            }
        }
        float2 acc[P / 2];
#pragma unroll
        for (int p = 0; p < P / 2; ++p) acc[p] = make_float2(0.f, 0.f);
        double dist = 0.0;

        // Every lane reads its document's entries itself: the teams of a warp walk
        // consecutive documents of the slice, so their i-th entries are adjacent
        // and one load instruction serves the warp.  The next batch's entries are
        // fetched while this one runs.
        // (a slice's row count is a multiple of RB: whole batches, no bounds checks)
        const float *vent = a.v + sbeg + t;
        int2 e[RB], en[RB];
        float ev[RB], evn[RB];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            e[rr] = ld_stream(ent + rr * kSlice, pol_stream);
            if constexpr (KIND == Kind::Spmm) ev[rr] = ld_stream(vent + rr * kSlice, pol_stream);
        }
        for (int i0 = 0; i0 < Ls; i0 += RB) {
            if (i0 + RB < Ls) {
                ent += RB * kSlice;
                if constexpr (KIND == Kind::Spmm) vent += RB * kSlice;
#pragma unroll
                for (int rr = 0; rr < RB; ++rr) {
                    en[rr] = ld_stream(ent + rr * kSlice, pol_stream);
                    if constexpr (KIND == Kind::Spmm) evn[rr] = ld_stream(vent + rr * kSlice, pol_stream);
                }
            }
#pragma unroll 1
            for (int once = 0; once < 1; ++once) {   // `continue` ends the batch early
                float cv[RB], tv[RB];
#pragma unroll
                for (int rr = 0; rr < RB; ++rr) {
                    cv[rr] = __int_as_float(e[rr].y);
                    if constexpr (KIND == Kind::Spmm) tv[rr] = ev[rr];
                }
                // padding entries (c = 0) read row 0, always valid: no zero fill, and
                // their tau is 0
                uint32_t kw[RB][WORDS];
#pragma unroll
                for (int rr = 0; rr < RB; ++rr) {
                    e[rr].x = checked_index(e[rr].x, a.Vu, status);
                    load_words<WORDS>(KTl + (long)e[rr].x * kRowBytes, kw[rr], pol_keep);
                }
                float tau[RB];
                if constexpr (KIND == Kind::Spmm) {
#pragma unroll
                    for (int rr = 0; rr < RB; ++rr) tau[rr] = cv[rr] != 0.f ? tv[rr] : 0.f;
                } else {
                    float d[RB];
#pragma unroll
                    for (int rr = 0; rr < RB; ++rr) {
                        float2 d2 = __fmul2_rn(pair_of<KT_t>(kw[rr], 0), u[0]);
#pragma unroll
                        for (int p = 1; p < P / 2; ++p)
                            d2 = __ffma2_rn(pair_of<KT_t>(kw[rr], p), u[p], d2);
                        d[rr] = d2.x + d2.y;
                    }
                    float dm[KIND == Kind::Final ? RB : 1];
                    uint32_t mw[KIND == Kind::Final ? RB : 1][WORDS];
                    if constexpr (KIND == Kind::Final) {
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) {
                            load_words<WORDS>(KMTl + (long)e[rr].x * kRowBytes, mw[rr], pol_keep);
                            float2 m2 = __fmul2_rn(pair_of<KT_t>(mw[rr], 0), u[0]);
#pragma unroll
                            for (int p = 1; p < P / 2; ++p)
                                m2 = __ffma2_rn(pair_of<KT_t>(mw[rr], p), u[p], m2);
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
                    if constexpr (KIND == Kind::Final) {
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) tau[rr] = cv[rr] * (dm[rr] * rcp_approx(d[rr]));
                    } else {
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) tau[rr] = cv[rr] * rcp_approx(d[rr]);
                    }
                    bool tiny = false;
#pragma unroll
                    for (int rr = 0; rr < RB; ++rr) tiny |= cv[rr] != 0.f && !(d[rr] >= 0x1p-100f);
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
                                sd += (double)k2.x * u[p].x + (double)k2.y * u[p].y;
                                if constexpr (KIND == Kind::Final) {
                                    const float2 m2 = pair_of<KT_t>(mw[rr], p);
                                    md += (double)m2.x * u[p].x + (double)m2.y * u[p].y;
                                }
                            }
#pragma unroll
                            for (int o = 1; o < Q; o <<= 1) {
                                sd += __shfl_xor_sync(kFull, sd, o);
                                if constexpr (KIND == Kind::Final) md += __shfl_xor_sync(kFull, md, o);
                            }
                            if (cv[rr] != 0.f && !(d[rr] >= 0x1p-100f)) {
                                if constexpr (KIND == Kind::Final) {
                                    if (tl == (rr & (Q - 1))) dist += (double)cv[rr] * (md / sd);
                                }
                                else tau[rr] = sd > 0.0 ? (float)((double)cv[rr] / sd) : 0.f;
                                fixed |= 1u << rr;
                                if (tl == 0) atomicOr(status, sd > 0.0 ? ST_GUARD : ST_NUMERIC);
                            }
                        }
                    }
                    if constexpr (KIND == Kind::Final) {
                        // Every lane holds every row's contribution; lane tl adds rows
                        // tl, tl + Q, ... in FP64, one FP64 add per row and warp (the
                        // FP64 pipe is narrow), and the team's sums are combined at the end.
#pragma unroll
                        for (int r0 = 0; r0 < RB; r0 += Q) {
                            float mine = 0.f;
#pragma unroll
                            for (int q = 0; q < Q && r0 + q < RB; ++q) {
                                const int rr = r0 + q;
                                const float c_rr = cv[rr] != 0.f && !(fixed >> rr & 1u) ? tau[rr] : 0.f;
                                mine = tl == q ? c_rr : mine;
                            }
                            dist += (double)mine;
                        }
                        continue;
                    } else {
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) tau[rr] = cv[rr] != 0.f ? tau[rr] : 0.f;
                    }
                    if constexpr (KIND == Kind::Sddmm) {
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) {
                            const int i = i0 + rr;
                            if (tl == (rr & (Q - 1)) && cv[rr] != 0.f) a.v[sbeg + (long)i * kSlice + t] = tau[rr];
                        }
                        continue;
                    }
                }
                // acc += tau K^T[w] over this lane's P values (16-bit rows are widened
                // again here rather than kept widened across the batch)
                if constexpr (KIND == Kind::Fused || KIND == Kind::Spmm) {
#pragma unroll
                    for (int rr = 0; rr < RB; ++rr) {
                        const float2 t2 = make_float2(tau[rr], tau[rr]);
#pragma unroll
                        for (int p = 0; p < P / 2; ++p) acc[p] = __ffma2_rn(t2, pair_again<KT_t>(kw[rr], p), acc[p]);
                    }
                }
            }
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) {
                e[rr] = en[rr];
                if constexpr (KIND == Kind::Spmm) ev[rr] = evn[rr];
            }
            if (i0 == 0 && g2 < n_groups && lane < (ne - nb) / kSlice)
                prefetch_l2(a.slice_nz + nb + (long)lane * kSlice + t2);   // the next group's row `lane`
        }

        if constexpr (KIND == Kind::Fused || KIND == Kind::Spmm) {
            if (has) {
                float rr[P], nu[P];
                load_floats<P>(a.r + tl * P, rr);
                bool bad = false;
                if (KIND == Kind::Fused && a.tol > 0.f) {
                    // the row marginal of P = diag(u) K diag(v) against r, with this
                    // iteration's u and v (a NaN counts as not converged)
#pragma unroll
                    for (int p = 0; p < P / 2; ++p) {
                        const int k = tl * P + 2 * p;
                        const float e0 = k < vr ? fabsf(u[p].x * acc[p].x - rr[2 * p]) : 0.f;
                        const float e1 = k + 1 < vr ? fabsf(u[p].y * acc[p].y - rr[2 * p + 1]) : 0.f;
                        errmax = fmaxf(errmax, e0 <= FLT_MAX ? e0 : INFINITY);
                        errmax = fmaxf(errmax, e1 <= FLT_MAX ? e1 : INFINITY);
                    }
                }
#pragma unroll
                for (int p = 0; p < P / 2; ++p) {
                    const int k = tl * P + 2 * p;
                    nu[2 * p] = k < vr ? rr[2 * p] * rcp_approx(acc[p].x) : 0.f;
                    nu[2 * p + 1] = k + 1 < vr ? rr[2 * p + 1] * rcp_approx(acc[p].y) : 0.f;
                    bad |= !(nu[2 * p] < INFINITY) || !(nu[2 * p + 1] < INFINITY);
                }
                if (bad) atomicOr(status, ST_NUMERIC);
                float *dst = a.u + ld * VRP + tl * P;
#pragma unroll
                for (int i = 0; i < P / 4; ++i)
                    st_stream4(dst + 4 * i, make_float4(nu[4 * i], nu[4 * i + 1], nu[4 * i + 2], nu[4 * i + 3]),
                               pol_stream);
            }
        } else if constexpr (KIND == Kind::Final) {
#pragma unroll
            for (int o = 1; o < Q; o <<= 1) dist += __shfl_xor_sync(kFull, dist, o);
            if (has && tl == 0) {
                if (!(fabs(dist) < INFINITY)) atomicOr(status, ST_NUMERIC);
                out[__ldg(a.doc_orig + ld)] = dist;
            }
        }
    }
    if constexpr (KIND == Kind::Fused) {
        if (a.tol > 0.f) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) errmax = fmaxf(errmax, __shfl_xor_sync(kFull, errmax, o));
            if (lane == 0) atomicMax(a.conv + 1 + a.it, __float_as_uint(errmax));
        }
    }
    if constexpr (KIND == Kind::Final) {
        // the x-updates applied: all of them, or up to the one that came below tol
        if (a.conv && blockIdx.x == 0 && threadIdx.x == 0) {
            int applied = a.it;
            if (a.tol > 0.f)
                for (int i = 0; i < a.it; ++i)
                    if (__uint_as_float(a.conv[1 + i]) < a.tol) {
                        applied = i + 1;
                        break;
                    }
            a.conv[0] = (unsigned)applied;
        }
    }
}

template <int VRP, class KT_t, Kind KIND, int NT, int MINB>
cudaError_t run_walk3_v(const IterArgs &a, int sms, cudaStream_t s) {
    auto kern = k_walk3<VRP, KT_t, KIND, NT, MINB>;
    static LaunchCache cache;
    int per_sm = 1;
    // no shared memory: all of the SM's L1 for the gathered K^T rows (carveout 0)
    cudaError_t e = cache.blocks_per_sm(kern, NT, 0, 0, &per_sm);
    if (e != cudaSuccess) return e;
    constexpr int Q = W3<VRP, KT_t>::Q;
    const long groups = (long)a.n_slices * Q;
    const long need = (groups * 32 + NT - 1) / NT;
    long blocks = (long)sms * per_sm;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (a.N > 0) kern<<<(unsigned)blocks, NT, 0, s>>>(a);
    return cudaGetLastError();
}

// Launch shape: 128-thread blocks with a register cap that lets 4 blocks share an
// SM (3 for FP16 rows, whose widening takes more registers); the final step, with a
// second row per nonzero, 3 (FP32) or 2.
template <int VRP, class KT_t, Kind KIND>
cudaError_t run_walk3(const IterArgs &a, int sms, cudaStream_t s) {
    constexpr bool f32 = sizeof(KT_t) == 4, bf = std::is_same<KT_t, __nv_bfloat16>::value;
    constexpr int MINB = KIND == Kind::Final ? (f32 ? 3 : 2) : (f32 || bf ? 4 : 3);
    return run_walk3_v<VRP, KT_t, KIND, 128, MINB>(a, sms, s);
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
