// a3 x t + a4 in one launch, each document's K^T rows held in registers and split
// by columns across a team of lanes.
//
// Every column of c is an independent problem in Algorithm 1.  With A_j the
// len_j x v_r matrix of the K^T rows of document j's words, one x-update is
// s = A_j u_j, tau = c_j ./ s, acc = A_j^T tau, u_j = r ./ acc (the fused
// SDDMM_SpMM of Section III-C, type 1), and the final step is
// WMD_j = sum_w c_wj (KM^T[w] . u_j) / (K^T[w] . u_j) (type 2).  A_j does not
// change between iterations, so it is gathered once and kept in registers.
//
// Lanes.  A document of LMAX rows (its length rounded up to its bucket; rows past
// the end are masked) is held by a team of G row groups of Q = VRP / 8 lanes (G = 1,
// 2, 4 or 8); group g holds rows [g RL, g RL + RL), RL = LMAX / G (at most 12, 16 in
// 128-column layouts), and lane q of a group holds columns [P q, P q + P), P = 8, of
// each of them.  acc = A_j^T tau is then partial over the groups only, the dots s = A_j u_j
// partial over the Q lanes of a group.
//
// Rows.  The dots are finished by a reduce-scatter over the group's Q lanes: after
// it lane q holds the full dots of rows [qR, qR + R), R = RL / Q, computes their tau,
// and an all-gather gives every lane of the group all of tau.  Both are log2(Q)
// butterfly steps that move half of the remaining values each.  For the butterfly
// to need no selects, lane q stores row block b ^ q (blocks of R rows) in register
// block b: then at every step all lanes keep the same register blocks and send the
// same others.  The lane reads its word ids in that order (its own R ids,
// all-gathered the same way), so its gathers fill the register blocks directly.
//
// Columns, likewise over the G groups: group g stores column block c ^ g (blocks of
// P / G columns of the lane's slice) in register block c, the partial acc go through
// a reduce-scatter over the groups (group g ends with column block g), each group
// takes u = r / acc for its P / G columns only, and an all-gather hands u back to
// every group.  The final step reads KM^T in natural column order and puts u back
// in that order once.
//
// Packed f32x2 FMAs work on column pairs of a row: a row's dot is P / 2 of them
// plus one add, its contribution to acc another P / 2.
//
// A document's arithmetic depends on its own nonzeros and on its bucket (a
// function of its length) only, so it gives the same bits alone, batched, served
// or in any document range.
#pragma once

#include "walk3.cuh"

namespace swmd {
namespace {

constexpr int kColThreads = 128;

// Four K^T values [4 idx4, 4 idx4 + 4) of the word-major layout, widened to float.
__device__ __forceinline__ float4 load_slice(const void *base, int kprec, long idx4) {
    if (kprec == 0) return __ldg(reinterpret_cast<const float4 *>(base) + idx4);
    const uint2 raw = __ldg(reinterpret_cast<const uint2 *>(base) + idx4);
    if (kprec == 1)
        return make_float4(__uint_as_float(raw.x << 16), __uint_as_float(raw.x & 0xffff0000u),
                           __uint_as_float(raw.y << 16), __uint_as_float(raw.y & 0xffff0000u));
    __half2 a, b;
    memcpy(&a, &raw.x, sizeof a);
    memcpy(&b, &raw.y, sizeof b);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

// The 32-bit words of a stored 16-bit pair, widened (x: the lower element).
__device__ __forceinline__ float2 widen2(uint32_t w, int kprec) {
    if (kprec == 1) return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    __half2 h;
    memcpy(&h, &w, sizeof h);
    return __half22float2(h);
}

// P consecutive 32-bit words (P = 1, 2, 4 or 8) of the read-only path, one vector load.
template <int P>
__device__ __forceinline__ void ldg_words(const void *p, uint32_t (&w)[P]) {
    if constexpr (P == 8) {
        asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
            : "l"(p));
    } else if constexpr (P == 4) {
        asm("ld.global.nc.v4.b32 {%0,%1,%2,%3}, [%4];" : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
    } else if constexpr (P == 2) {
        asm("ld.global.nc.v2.b32 {%0,%1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "l"(p));
    } else {
        asm("ld.global.nc.b32 %0, [%1];" : "=r"(w[0]) : "l"(p));
    }
}

// Swaps register blocks kb and kb ^ bit (blocks of P / G values) for every bit below
// 2^H set in g (H = log2 G: every bit): natural column order <-> the XOR block order
// of group g, or the rest of it after a load that placed the higher bits.
template <int P, int G, int H = 31 - __builtin_clz(G)>
__device__ __forceinline__ void swap_blocks(float (&x)[P], int g) {
    constexpr int B = P / G;
#pragma unroll
    for (int bit = 1; bit < G && bit < (1 << H); bit <<= 1) {
        const bool sw = (g & bit) != 0;
#pragma unroll
        for (int kb = 0; kb < G; ++kb) {
            if (kb & bit) continue;
#pragma unroll
            for (int e = 0; e < B; ++e) {
                const float lo = x[kb * B + e], hi = x[(kb ^ bit) * B + e];
                x[kb * B + e] = sw ? hi : lo;
                x[(kb ^ bit) * B + e] = sw ? lo : hi;
            }
        }
    }
}

// How a lane puts its slice of a K^T row into the XOR column-block order of its
// group g (blocks of P / G values): G >> H vector loads of 2^H blocks each, placed
// by the high bits of g, then conditional swaps for the low H bits.  H = 0: one load
// per block, no swap; H = log2 G: one whole-slice load, every bit swapped (fewer L1
// requests, more registers).  Timed per layout and group count on the
// 1,000,000-document workload: whole slices at 16 and 64 columns; at 32 columns two
// half-slice loads and one swap for four groups (solver 1.489 ms, against 1.513 ms
// with four block loads; swapping for two groups too spilled more and took 1.536 ms),
// block loads for two; block loads at 128 columns.
__host__ __device__ constexpr int cols_gather_h(int vrp, int g) {
    return (vrp == 16 || vrp == 64 || g >= 8) ? (g >= 8 ? 3 : g >= 4 ? 2 : g >= 2 ? 1 : 0)
                                              : vrp == 32 ? (g >= 4 ? 1 : 0) : 0;
}

// Columns [P ql, P ql + P) of the rows of words wv[i] (word-major layout of VRP
// columns), widened to float; PERM: in group g's column order (register block kb of
// B = P / G columns holds column block kb ^ g), else in natural order.  Rows past the
// document's end (wv[i] < 0) are not loaded: zeros, whose tau is masked to 0.  One
// unrolled loop per storage type, so all loads of a lane are in flight together.
template <int VRP, int P, int G, int RL, bool PERM = true>
__device__ __forceinline__ void gather_rows(float (&rv)[RL][P], const void *base, int kprec, const int (&wv)[RL],
                                            int ql, int g) {
    constexpr int LG2G = 31 - __builtin_clz(G);
    constexpr int H = PERM ? cols_gather_h(VRP, G) : LG2G;   // natural order: whole-slice loads
    constexpr int L = (P / G) << H;                          // values per load
    constexpr int NL = P / L;                                // loads per row
    static_assert(H <= LG2G && NL * L == P, "load shape");
    const int ghi = PERM ? (g >> H) : 0;                     // the load-placed bits of g
    if (kprec == 0) {
        const float *b = reinterpret_cast<const float *>(base) + ql * P;
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            uint32_t w[P] = {};
            if (wv[i] >= 0) {
#pragma unroll
                for (int kl = 0; kl < NL; ++kl) {
                    uint32_t wb[L];
                    ldg_words<L>(b + (long)wv[i] * VRP + (NL > 1 ? (kl ^ ghi) * L : 0), wb);
#pragma unroll
                    for (int e = 0; e < L; ++e) w[kl * L + e] = wb[e];
                }
            }
#pragma unroll
            for (int k = 0; k < P; ++k) rv[i][k] = __uint_as_float(w[k]);
            if constexpr (PERM && H > 0) swap_blocks<P, G, H>(rv[i], g);
        }
    } else {
        const unsigned short *b = reinterpret_cast<const unsigned short *>(base) + ql * P;
        uint32_t raw[RL][P / 2] = {};
#pragma unroll
        for (int i = 0; i < RL; ++i)
            if (wv[i] >= 0) {
#pragma unroll
                for (int kl = 0; kl < NL; ++kl) {
                    uint32_t wb[L / 2];
                    ldg_words<L / 2>(b + (long)wv[i] * VRP + (NL > 1 ? (kl ^ ghi) * L : 0), wb);
#pragma unroll
                    for (int e = 0; e < L / 2; ++e) raw[i][kl * (L / 2) + e] = wb[e];
                }
            }
#pragma unroll
        for (int i = 0; i < RL; ++i)
#pragma unroll
            for (int k = 0; k < P / 2; ++k) {
                const float2 f = widen2(raw[i][k], kprec);
                rv[i][2 * k] = f.x;
                rv[i][2 * k + 1] = f.y;
            }
        if constexpr (PERM && H > 0)
#pragma unroll
            for (int i = 0; i < RL; ++i) swap_blocks<P, G, H>(rv[i], g);
    }
}

// Partial dots of every register row with the lane's slice of u.
template <int RL, int P>
__device__ __forceinline__ void partial_dots(const float (&rv)[RL][P], const float (&u)[P], float (&s)[RL]) {
#pragma unroll
    for (int i = 0; i < RL; ++i) {
        float2 d = __fmul2_rn(make_float2(rv[i][0], rv[i][1]), make_float2(u[0], u[1]));
#pragma unroll
        for (int k = 2; k < P; k += 2)
            d = __ffma2_rn(make_float2(rv[i][k], rv[i][k + 1]), make_float2(u[k], u[k + 1]), d);
        s[i] = d.x + d.y;
    }
}

// Reduce-scatter over the Q lanes of a row group: afterwards s[0..R) hold the
// group's full sums of the lane's own rows (register block 0).
template <class T, int RL, int Q, int R>
__device__ __forceinline__ void reduce_scatter(T (&s)[RL]) {
#pragma unroll
    for (int m = Q / 2; m >= 1; m >>= 1)
#pragma unroll
        for (int i = 0; i < m * R; ++i) s[i] += __shfl_xor_sync(kFull, s[i + m * R], m);
}

// All-gather over the Q lanes: tv[0..R) of every lane -> tv[i] for every register
// row (block b of lane ql from lane ql ^ b: the register-block order).
template <class T, int RL, int Q, int R>
__device__ __forceinline__ void all_gather(T (&tv)[RL]) {
#pragma unroll
    for (int m = 1; m < Q; m <<= 1)
#pragma unroll
        for (int i = 0; i < m * R; ++i) tv[m * R + i] = __shfl_xor_sync(kFull, tv[i], m);
}

// The FP64 guard for a K^T u below 2^-100 (rare, entered by the whole warp):
// the lane's u slice is published in the warp's shared buffer `su` (lane l's P
// values at P l), and the dot of an own row is recomputed in FP64 from the stored
// row (the same, exactly widened values) and the team's whole u.
template <int P>
__device__ __forceinline__ void publish_u(float *su, int lane, const float (&u)[P]) {
    __syncwarp();
#pragma unroll
    for (int k = 0; k < P; ++k) su[P * lane + k] = u[k];
    __syncwarp();
}
template <int VRP>
__device__ __forceinline__ double dot_fp64(const void *base, int kprec, int w, const float *su_team) {
    double s = 0.0;
#pragma unroll 4
    for (int c = 0; c < VRP / 4; ++c) {
        const float4 k4 = load_slice(base, kprec, (long)w * (VRP / 4) + c);
        s = fma((double)k4.x, (double)su_team[4 * c], s);
        s = fma((double)k4.y, (double)su_team[4 * c + 1], s);
        s = fma((double)k4.z, (double)su_team[4 * c + 2], s);
        s = fma((double)k4.w, (double)su_team[4 * c + 3], s);
    }
    return s;
}

// One task: up to 32 / (G Q) documents of one bucket (LMAX = G RL rows).  A team of
// G row groups of Q lanes owns a document; group g holds rows [g RL, g RL + RL).
// su: this warp's shared buffer (32 P floats) for the FP64 guard.
template <int VRP, int G, int RL>
__device__ __forceinline__ void cols_task(const ColArgs &a, const ResidentArgs &q, int4 tk, int lane,
                                          float *su) {
    constexpr int P = cols_p(VRP), Q = VRP / P, R = RL / Q, TEAM = G * Q, B = P / G;
    static_assert(Q >= 1 && Q <= 32 && (Q & (Q - 1)) == 0, "row groups of a power of two lanes");
    static_assert(RL % Q == 0 && R >= 1 && TEAM <= 32 && (G & (G - 1)) == 0, "whole row blocks");
    static_assert(B >= 1 && B * G == P, "whole column blocks");
    const int team = lane / TEAM, g = (lane / Q) % G, ql = lane % Q;
    // the column of the lane's slice held in register k: block k / B holds block (k / B) ^ g
    auto col_of = [g](int k) { return (((k / B) ^ g) * B) + k % B; };
    const bool has = team < tk.y;
    const int doc = tk.x + team;
    int beg = 0, len = 0;
    const QParams *qp = q.it.qp;
    const int vr = qp->vr;
    const float u0 = qp->u0;
    int *const status = qp->status;
    if (has) {
        beg = checked_index(__ldg(a.doc_ptr + doc), a.nnz + 1, status);
        len = checked_index(__ldg(a.doc_ptr + doc + 1), a.nnz + 1, status) - beg;
#if SWMD_DEBUG_CHECKS
        if (len < 0) {
            atomicOr(status, ST_BOUNDS);
            len = 0;
        }
#endif
    }
    const int2 *ent = a.nz + beg;
    const int row0 = g * RL;                          // the group's first row
    const float *su_team = su + P * (team * TEAM);    // the team's u, column-ordered (guard only)

    // the nonzeros (word id, c) of the rows this lane finishes, row block ql of the
    // group; past the end: word -1 (not loaded) and c = 0 (tau 0)
    float cown[R];
    int wown[R];
#pragma unroll
    for (int o = 0; o < R; ++o) {
        const int row = row0 + ql * R + o;
        int2 e = make_int2(-1, 0);
        if (row < len) {
            e = __ldg(&ent[row]);
            e.x = checked_index(e.x, a.Vu, status);
        }
        wown[o] = e.x;
        cown[o] = __int_as_float(e.y);
    }
    // u in the lane's column order (register k: column ql P + col_of(k)); r of the B
    // columns whose u this lane computes (column block g of its slice)
    float rr[B], u[P];
#pragma unroll
    for (int k = 0; k < P; ++k) u[k] = has && ql * P + col_of(k) < vr ? u0 : 0.f;
#pragma unroll
    for (int e = 0; e < B; ++e) rr[e] = __ldg(q.it.r + ql * P + g * B + e);
    // the group's rows of K^T in register-block order, all loads in flight at once
    float rv[RL][P];
    {
        int wv[RL];   // word ids in register-block order: the team's own ids, all-gathered
#pragma unroll
        for (int o = 0; o < R; ++o) wv[o] = wown[o];
        all_gather<int, RL, Q, R>(wv);
        gather_rows<VRP, P, G, RL>(rv, q.it.KT, a.kprec, wv, ql, g);
    }

    bool bad = false;
    for (int it = 0; it < q.t; ++it) {
        float tv[RL];
        partial_dots<RL, P>(rv, u, tv);
        reduce_scatter<float, RL, Q, R>(tv);
        bool tiny = false;
        float s_own[R];
#pragma unroll
        for (int o = 0; o < R; ++o) {
            s_own[o] = tv[o];
            const bool valid = cown[o] != 0.f;
            tiny |= valid && !(tv[o] >= 0x1p-100f);
            tv[o] = valid ? cown[o] * rcp_approx(tv[o]) : 0.f;
        }
        if (__any_sync(kFull, tiny)) {
            SWMD_COLD_PATH();
            publish_u<P>(su, lane, u);
#pragma unroll
            for (int o = 0; o < R; ++o) {
                if (cown[o] != 0.f && !(s_own[o] >= 0x1p-100f)) {
                    const int w = checked_index(__ldg(&ent[row0 + ql * R + o].x), a.Vu, status);
                    const double sd = dot_fp64<VRP>(q.it.KT, a.kprec, w, su_team);
                    tv[o] = sd > 0.0 ? (float)((double)cown[o] / sd) : 0.f;
                    atomicOr(status, sd > 0.0 ? ST_GUARD : ST_NUMERIC);
                }
            }
        }
        all_gather<float, RL, Q, R>(tv);
        float2 acc[P / 2];
#pragma unroll
        for (int k = 0; k < P / 2; ++k) acc[k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            const float2 t2 = make_float2(tv[i], tv[i]);
#pragma unroll
            for (int k = 0; k < P / 2; ++k)
                acc[k] = __ffma2_rn(make_float2(rv[i][2 * k], rv[i][2 * k + 1]), t2, acc[k]);
        }
        // the row groups' partial sums: a reduce-scatter over the G groups leaves
        // group g the full acc of column block g (register block 0) ...
#pragma unroll
        for (int m = G / 2; m >= 1; m >>= 1)
#pragma unroll
            for (int k = 0; k < m * B / 2; ++k) {
                acc[k].x += __shfl_xor_sync(kFull, acc[k + m * B / 2].x, m * Q);
                acc[k].y += __shfl_xor_sync(kFull, acc[k + m * B / 2].y, m * Q);
            }
        // (blocks of one column, eight groups: the last step splits a pair)
        if constexpr (B == 1) acc[0].x += __shfl_xor_sync(kFull, acc[0].y, Q);
        // ... whose u it computes ...
#pragma unroll
        for (int e = 0; e < B; ++e) {
            const bool live = has && ql * P + g * B + e < vr;
            const float nu = live ? rr[e] * rcp_approx((e & 1) ? acc[e / 2].y : acc[e / 2].x) : 0.f;
            bad |= live && !(nu < INFINITY);
            u[e] = nu;
        }
        // ... and an all-gather gives every group all P (register block b from group g ^ b)
#pragma unroll
        for (int m = 1; m < G; m <<= 1)
#pragma unroll
            for (int e = 0; e < m * B; ++e) u[m * B + e] = __shfl_xor_sync(kFull, u[e], m * Q);
    }

    // final step: s = K^T[w].u and m = KM^T[w].u per nonzero, WMD = sum c m / s
    float s_own[R];
    bool tiny = false;
    {
        float tv[RL];
        partial_dots<RL, P>(rv, u, tv);
        reduce_scatter<float, RL, Q, R>(tv);
#pragma unroll
        for (int o = 0; o < R; ++o) {
            s_own[o] = tv[o];
            tiny |= cown[o] != 0.f && !(tv[o] >= 0x1p-100f);
        }
    }
    {
        int wv[RL];   // the word ids again
#pragma unroll
        for (int o = 0; o < R; ++o) wv[o] = wown[o];
        all_gather<int, RL, Q, R>(wv);
        gather_rows<VRP, P, G, RL, false>(rv, q.it.KMT, a.kprec, wv, ql, g);   // natural order
    }
    swap_blocks<P, G>(u, g);   // u back to natural column order, like the KM^T rows
    double dist = 0.0;
    {
        float tv[RL];
        partial_dots<RL, P>(rv, u, tv);
        reduce_scatter<float, RL, Q, R>(tv);
#pragma unroll
        for (int o = 0; o < R; ++o)
            if (cown[o] != 0.f && s_own[o] >= 0x1p-100f) dist += (double)(cown[o] * (tv[o] * rcp_approx(s_own[o])));
    }
    if (__any_sync(kFull, tiny)) {
        SWMD_COLD_PATH();
        publish_u<P>(su, lane, u);
#pragma unroll
        for (int o = 0; o < R; ++o) {
            if (cown[o] != 0.f && !(s_own[o] >= 0x1p-100f)) {
                const int w = checked_index(__ldg(&ent[row0 + ql * R + o].x), a.Vu, status);
                const double sd = dot_fp64<VRP>(q.it.KT, a.kprec, w, su_team);
                const double md = dot_fp64<VRP>(q.it.KMT, a.kprec, w, su_team);
                dist += (double)cown[o] * (md / sd);
                atomicOr(status, sd > 0.0 ? ST_GUARD : ST_NUMERIC);
            }
        }
    }
#pragma unroll
    for (int m = 1; m < TEAM; m <<= 1) dist += __shfl_xor_sync(kFull, dist, m);
    if (bad) atomicOr(status, ST_NUMERIC);
    if (has && g == 0 && ql == 0) {
        if (!(fabs(dist) < INFINITY)) atomicOr(status, ST_NUMERIC);
        double *const out = q.it.out ? q.it.out : qp->out;
        out[__ldg(a.doc_orig + doc)] = dist;
    }
}

// One document task for one query: the bucket's instantiation.  LONG: the task list
// also holds the buckets of 48, 64 and 96 rows (a separate kernel, so that the
// buckets of up to 32 rows keep the registers they have without them).
template <int VRP, bool LONG>
__device__ __forceinline__ void cols_dispatch(const ColArgs &a, const ResidentArgs &q, int4 tk, int lane, float *su) {
    switch (tk.z) {
        case 8:
            if constexpr (cols_fits(8, VRP)) cols_task<VRP, cols_groups(8, VRP), 8 / cols_groups(8, VRP)>(a, q, tk, lane, su);
            break;
        case 16:
            if constexpr (cols_fits(16, VRP)) cols_task<VRP, cols_groups(16, VRP), 16 / cols_groups(16, VRP)>(a, q, tk, lane, su);
            break;
        case 24:
            if constexpr (cols_fits(24, VRP)) cols_task<VRP, cols_groups(24, VRP), 24 / cols_groups(24, VRP)>(a, q, tk, lane, su);
            break;
        case 48:
            if constexpr (LONG && cols_fits(48, VRP)) cols_task<VRP, cols_groups(48, VRP), 48 / cols_groups(48, VRP)>(a, q, tk, lane, su);
            break;
        case 64:
            if constexpr (LONG && cols_fits(64, VRP)) cols_task<VRP, cols_groups(64, VRP), 64 / cols_groups(64, VRP)>(a, q, tk, lane, su);
            break;
        case 96:
            if constexpr (LONG && cols_fits(96, VRP)) cols_task<VRP, cols_groups(96, VRP), 96 / cols_groups(96, VRP)>(a, q, tk, lane, su);
            break;
        default:
            cols_task<VRP, cols_groups(32, VRP), 32 / cols_groups(32, VRP)>(a, q, tk, lane, su);
            break;
    }
}

// Four blocks of 128 threads per SM (at most 128 registers a thread): the gathers
// of one warp's rows are hidden by the arithmetic of the others, which measured
// faster than fewer, spill-free warps.  128-column layouts hold 16 rows of eight
// columns per lane and take three blocks (168 registers).
constexpr int cols_min_blocks(int vrp) { return vrp >= 128 ? 3 : 4; }

// One query (the kernel argument a.q0): warps walk the document tasks.
template <int VRP, bool LONG>
__global__ void __launch_bounds__(kColThreads, cols_min_blocks(VRP)) k_resident_cols(const __grid_constant__ ColArgs a) {
    constexpr int P = cols_p(VRP);
    __shared__ __align__(16) float s_u[kColThreads * P];   // per warp: 32 lanes x P values of u
    const int lane = threadIdx.x & 31;
    float *su = s_u + P * (threadIdx.x & ~31);
    const long gwarp = ((long)blockIdx.x * kColThreads + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * kColThreads) >> 5;
    for (long task = gwarp; task < a.n_tasks; task += nwarps)
        cols_dispatch<VRP, LONG>(a, a.q0, __ldg(a.tasks + task), lane, su);
}

// Many queries of one layout in one persistent launch: warps walk the tiles
// (query group, document task) in group-major order -- the whole GPU works on one
// group's K^T at a time (it stays in L2) and the next group starts while the last
// tiles of this one finish.  A tile runs its task for every query of the group in
// turn, so the task's nonzeros come from DRAM once for the group (later queries
// re-read them from L1).  Each (query, document) computes exactly what the single
// query does: the same bits.
template <int VRP, bool LONG>
__global__ void __launch_bounds__(kColThreads, cols_min_blocks(VRP)) k_resident_cols_multi(const __grid_constant__ ColArgs a) {
    constexpr int P = cols_p(VRP);
    __shared__ __align__(16) float s_u[kColThreads * P];
    const int lane = threadIdx.x & 31;
    float *su = s_u + P * (threadIdx.x & ~31);
    const long gwarp = ((long)blockIdx.x * kColThreads + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * kColThreads) >> 5;
    const long groups = (a.nq + a.q_per_group - 1) / a.q_per_group;
    const long tiles = groups * a.n_tasks;
    for (long tile = gwarp; tile < tiles; tile += nwarps) {
        const long grp = tile / a.n_tasks;
        const int4 tk = __ldg(a.tasks + (tile - grp * a.n_tasks));
        const int q0 = (int)grp * a.q_per_group;
        const int q1 = min(q0 + a.q_per_group, a.nq);
        for (int qi = q0; qi < q1; ++qi) cols_dispatch<VRP, LONG>(a, a.queries[qi], tk, lane, su);
    }
}

template <int VRP, bool LONG>
cudaError_t run_cols(const ColArgs &a, int sms, int nq, cudaStream_t s) {
    static LaunchCache cache, cache_multi;
    int per_sm = 1;
    if (!a.queries) {
        auto kern = k_resident_cols<VRP, LONG>;
        cudaError_t e = cache.blocks_per_sm(kern, kColThreads, 0, -1, &per_sm);
        if (e != cudaSuccess) return e;
        long blocks = ((long)a.n_tasks + kColThreads / 32 - 1) / (kColThreads / 32);
        if (blocks > (long)sms * per_sm) blocks = (long)sms * per_sm;
        if (blocks > 0) kern<<<(unsigned)blocks, kColThreads, 0, s>>>(a);
        return cudaGetLastError();
    }
    if (a.nq != nq || a.q_per_group < 1) return cudaErrorInvalidValue;
    auto kern = k_resident_cols_multi<VRP, LONG>;
    cudaError_t e = cache_multi.blocks_per_sm(kern, kColThreads, 0, -1, &per_sm);
    if (e != cudaSuccess) return e;
    const long tiles = (long)((nq + a.q_per_group - 1) / a.q_per_group) * a.n_tasks;
    long blocks = (tiles + kColThreads / 32 - 1) / (kColThreads / 32);
    if (blocks > (long)sms * per_sm) blocks = (long)sms * per_sm;
    if (blocks > 0) kern<<<(unsigned)blocks, kColThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace
}  // namespace swmd
