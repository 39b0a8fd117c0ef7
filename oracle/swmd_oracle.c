/*
 * swmd_oracle.c -- plain, slow, FP64 CPU oracle of Sinkhorn Word Mover's Distance
 * for one query document against many target documents (arXiv 2107.06433).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  The CUDA product path never links,
 * loads or calls it, and it shares no code, header or table with that path.
 *
 * What it follows:
 *   - Algorithm 1 (Section III-A): I = (r > 0); r = r(I); M = M(I,:);
 *     K = exp(-lambda M); x = ones / length(r); repeat x = diag(1./r) K
 *     (c .* (1 ./ (K^T (1./x)))); then u = 1./x; v = c .* (1 ./ (K^T u));
 *     d = sum(u .* ((K .* M) v)), a per-document (column) sum.
 *   - Section III-B1 and Table I: the same steps as the paper's Python code runs
 *     them (M = cdist(vecs[sel], vecs); K_over_r = (1/r) * K; x = K_over_r @ v).
 *   - Algorithms 2 and 3 (Section III-B4): the sparse reformulation, an SDDMM
 *     that evaluates K^T u only at the nonzeros of c, followed by the transpose
 *     to CSC and the SpMM x = K_over_r v.
 *   - Section III-E, Table II (right column): the 1-to-1 variant, one (query,
 *     target) pair with the cost built over the target's words only.
 *
 * Readings of the paper taken here (each is listed with its reason in the design
 * notes of the repository):
 *   - K = exp(-lambda M) with lambda > 0 (Algorithm 1; Table I negates lambda).
 *   - M is the plain Euclidean distance, not its square (Section II-A, Table I
 *     "cdist"), computed here in the direct difference form.
 *   - "while x changes" is run as exactly t = max_iter updates of x (Table I),
 *     t = 0 allowed; a separate convergence mode stops on the row marginal.
 *   - The SDDMM listing's garbled indices are read as Algorithm 1 states them:
 *     v_wj = c_wj / sum_k K[k,w] u[k,j].
 *   - The final sum is per document: the result is a length-N vector.
 *   - Duplicate query ids are summed, zero weights dropped (I = r > 0), and r
 *     is normalised to sum 1 (Section III-B1); negative or NaN weights and ids
 *     outside [0, V) are errors.
 *   - Columns of c are normalised to sum 1 (Section III-B1); a non-positive value
 *     or an empty column is an error.
 *
 * Everything is FP64 (inputs that arrive as float are widened).  Loops that
 * OpenMP runs in parallel write disjoint outputs, each computed in a fixed
 * order, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Section III-B1 / Algorithm 1 first line: r is a length-V histogram; keep its
 * positive entries (I = r > 0) in increasing word order and normalise to sum 1.
 * The query arrives as (id, weight) pairs; repeated ids add up.
 * Returns v_r > 0, or ORACLE_EINVAL. */
int64_t oracle_select(int64_t V, int64_t n, const int32_t *ids, const double *w,
                      int32_t *out_ids, double *out_r)
{
    if (V <= 0 || n < 0) return ORACLE_EINVAL;
    double *r = (double *)calloc((size_t)V, sizeof(double));
    if (!r) return ORACLE_ENOMEM;
    for (int64_t i = 0; i < n; ++i) {
        if (ids[i] < 0 || ids[i] >= V || !(w[i] >= 0.0) || isinf(w[i])) {
            free(r);
            return ORACLE_EINVAL;
        }
        r[ids[i]] += w[i];
    }
    double total = 0.0;
    int64_t vr = 0;
    for (int64_t i = 0; i < V; ++i)
        if (r[i] > 0.0) { total += r[i]; ++vr; }
    if (vr == 0) { free(r); return ORACLE_EINVAL; }
    int64_t k = 0;
    for (int64_t i = 0; i < V; ++i)
        if (r[i] > 0.0) { out_ids[k] = (int32_t)i; out_r[k] = r[i] / total; ++k; }
    free(r);
    return vr;
}

/* Section II-A: m(i,j) = sqrt(sum_d (emb[i,d] - emb[j,d])^2); Table I computes
 * M = cdist(vecs[sel], vecs), a v_r x V matrix (row k = query word q[k]).
 * M is row-major [v_r][V]. */
void oracle_cdist(int64_t V, int32_t d, const float *E, int32_t vr, const int32_t *q, double *M)
{
    int64_t w;
#pragma omp parallel for schedule(static)
    for (w = 0; w < V; ++w) {
        const float *ew = E + (size_t)w * d;
        for (int32_t k = 0; k < vr; ++k) {
            const float *eq = E + (size_t)q[k] * d;
            double acc = 0.0;
            for (int32_t j = 0; j < d; ++j) {
                double diff = (double)eq[j] - (double)ew[j];
                acc += diff * diff;
            }
            M[(size_t)k * V + w] = sqrt(acc);
        }
    }
}

/* Algorithm 1 / Table I: K = exp(-lambda M) and K .* M, elementwise. */
void oracle_kernel(int64_t n, const double *M, double lambda, double *K, double *KM)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        K[i] = exp(-lambda * M[i]);
        KM[i] = K[i] * M[i];
    }
}

/* Section III-B1: each column of c sums to 1.  c is V x N CSR (row = word,
 * column = document).  Returns ORACLE_EINVAL on a malformed matrix, a
 * non-positive value or an empty column. */
int oracle_normalize_columns(int64_t V, int64_t N, const int64_t *row_ptr, const int32_t *col,
                             const double *val_in, double *val_out)
{
    if (row_ptr[0] != 0) return ORACLE_EINVAL;
    double *colsum = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    if (!colsum) return ORACLE_ENOMEM;
    for (int64_t w = 0; w < V; ++w) {
        if (row_ptr[w + 1] < row_ptr[w]) { free(colsum); return ORACLE_EINVAL; }
        for (int64_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p) {
            if (col[p] < 0 || col[p] >= N || !(val_in[p] > 0.0) || isinf(val_in[p])) {
                free(colsum);
                return ORACLE_EINVAL;
            }
            colsum[col[p]] += val_in[p];
        }
    }
    for (int64_t j = 0; j < N; ++j)
        if (!(colsum[j] > 0.0)) { free(colsum); return ORACLE_EINVAL; }
    for (int64_t p = 0; p < row_ptr[V]; ++p) val_out[p] = val_in[p] / colsum[col[p]];
    free(colsum);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Dense mode: Algorithm 1 with dense matrices, as Table I's NumPy lines do it.
 * Every step of Algorithm 1 acts column by column (document by document), so
 * the documents are processed in blocks of nb columns to bound memory; within a
 * block nothing is reordered.
 *
 * K, KM: [v_r][V] row-major.  r: [v_r] (sums to 1).  c: V x N CSR, columns
 * normalised.  wmd: [N].  x_out (optional): final x as [N][v_r]. */
int oracle_sinkhorn_dense(int32_t vr, int64_t V, int64_t N, const double *K, const double *KM,
                          const double *r, const int64_t *row_ptr, const int32_t *col,
                          const double *cval, int32_t t, int64_t nb, double *wmd, double *x_out)
{
    if (vr <= 0 || V <= 0 || N < 0 || t < 0) return ORACLE_EINVAL;
    if (nb <= 0) nb = 64;
    /* K_over_r = (1 / r) * K  (Table I) */
    double *Kr = (double *)malloc(sizeof(double) * (size_t)vr * V);
    if (!Kr) return ORACLE_ENOMEM;
    for (int32_t k = 0; k < vr; ++k)
        for (int64_t w = 0; w < V; ++w) Kr[(size_t)k * V + w] = (1.0 / r[k]) * K[(size_t)k * V + w];

    int rc = ORACLE_OK;
    int64_t j0;
    for (j0 = 0; j0 < N; j0 += nb) {
        int64_t b = (N - j0 < nb) ? (N - j0) : nb;
        double *cd = (double *)calloc((size_t)V * b, sizeof(double));   /* dense c block  [V][b] */
        double *x = (double *)malloc(sizeof(double) * (size_t)vr * b);  /* [v_r][b] */
        double *u = (double *)malloc(sizeof(double) * (size_t)vr * b);
        double *KTu = (double *)malloc(sizeof(double) * (size_t)V * b); /* [V][b] */
        double *v = (double *)malloc(sizeof(double) * (size_t)V * b);   /* [V][b] */
        if (!cd || !x || !u || !KTu || !v) {
            free(cd); free(x); free(u); free(KTu); free(v);
            rc = ORACLE_ENOMEM;
            break;
        }
        for (int64_t w = 0; w < V; ++w)
            for (int64_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p)
                if (col[p] >= j0 && col[p] < j0 + b) cd[(size_t)w * b + (col[p] - j0)] = cval[p];

        /* x = ones(length(r), size(c,2)) / length(r) */
        for (int64_t i = 0; i < (int64_t)vr * b; ++i) x[i] = 1.0 / vr;

        for (int32_t it = 0; it <= t; ++it) {
            /* u = 1 ./ x */
            for (int64_t i = 0; i < (int64_t)vr * b; ++i) u[i] = 1.0 / x[i];
            /* KT @ u : [V][b], dense over every word and document */
            int64_t w;
#pragma omp parallel for schedule(static)
            for (w = 0; w < V; ++w)
                for (int64_t jj = 0; jj < b; ++jj) {
                    double s = 0.0;
                    for (int32_t k = 0; k < vr; ++k) s += K[(size_t)k * V + w] * u[(size_t)k * b + jj];
                    KTu[(size_t)w * b + jj] = s;
                }
            /* v = c .* (1 ./ (KT @ u)) */
            for (int64_t i = 0; i < V * b; ++i) v[i] = cd[i] * (1.0 / KTu[i]);
            if (it == t) break;
            /* x = K_over_r @ v */
            int32_t k;
#pragma omp parallel for schedule(static)
            for (k = 0; k < vr; ++k)
                for (int64_t jj = 0; jj < b; ++jj) {
                    double s = 0.0;
                    for (int64_t ww = 0; ww < V; ++ww) s += Kr[(size_t)k * V + ww] * v[(size_t)ww * b + jj];
                    x[(size_t)k * b + jj] = s;
                }
        }
        /* d = sum(u .* ((K .* M) @ v), axis=0); u and v are those of the last pass */
        for (int64_t jj = 0; jj < b; ++jj) {
            double d = 0.0;
            for (int32_t k = 0; k < vr; ++k) {
                double y = 0.0;
                for (int64_t ww = 0; ww < V; ++ww) y += KM[(size_t)k * V + ww] * v[(size_t)ww * b + jj];
                d += u[(size_t)k * b + jj] * y;
            }
            wmd[j0 + jj] = d;
        }
        if (x_out)
            for (int64_t jj = 0; jj < b; ++jj)
                for (int32_t k = 0; k < vr; ++k) x_out[(size_t)(j0 + jj) * vr + k] = x[(size_t)k * b + jj];
        free(cd); free(x); free(u); free(KTu); free(v);
    }
    free(Kr);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sparse mode: the reformulation of Section III-B4.
 *   SDDMM (Algorithm 2): for every nonzero (w, j) of the V x N CSR c,
 *       v_wj = c_wj * (1 / sum_k KT[w][k] u[j][k])
 *   v.tocsc(): the same values in document-major (CSC) order;
 *   SpMM (Algorithm 3 on v_csc): x[j][k] = sum_{w in doc j} K_over_r[w][k] v_wj.
 * Layouts follow Section III-B4: KT[V][v_r] (word-major), u and x [N][v_r]
 * (document-major).  Unfused, in the paper's order.
 *
 * Optional outputs: x_out [N][v_r] (last x), u_out [N][v_r] (final u),
 * v_out [nnz] (final v in CSR order). */
typedef struct {
    int64_t *csc_ptr;  /* [N+1] */
    int64_t *csc_src;  /* [nnz] CSR position of each CSC entry */
    int32_t *csc_row;  /* [nnz] word of each CSC entry */
} csc_map;

static int build_csc(int64_t V, int64_t N, const int64_t *row_ptr, const int32_t *col, csc_map *m)
{
    int64_t nnz = row_ptr[V];
    m->csc_ptr = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    m->csc_src = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    m->csc_row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t *fill = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    if (!m->csc_ptr || !m->csc_src || !m->csc_row || !fill) {
        free(fill);
        return ORACLE_ENOMEM;
    }
    for (int64_t p = 0; p < nnz; ++p) m->csc_ptr[col[p] + 1]++;
    for (int64_t j = 0; j < N; ++j) m->csc_ptr[j + 1] += m->csc_ptr[j];
    /* rows are visited in increasing order, so each column lists its words ascending */
    for (int64_t w = 0; w < V; ++w)
        for (int64_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p) {
            int64_t q = m->csc_ptr[col[p]] + fill[col[p]]++;
            m->csc_src[q] = p;
            m->csc_row[q] = (int32_t)w;
        }
    free(fill);
    return ORACLE_OK;
}

static void free_csc(csc_map *m)
{
    free(m->csc_ptr);
    free(m->csc_src);
    free(m->csc_row);
}

/* Algorithm 2 with 1/dot, as Algorithm 1 defines v. */
static void sddmm(int32_t vr, int64_t V, const double *KT, const double *u, const int64_t *row_ptr,
                  const int32_t *col, const double *cval, double *v)
{
    int64_t w;
#pragma omp parallel for schedule(dynamic, 256)
    for (w = 0; w < V; ++w)
        for (int64_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p) {
            const double *kt = KT + (size_t)w * vr;
            const double *uj = u + (size_t)col[p] * vr;
            double s = 0.0;
            for (int32_t k = 0; k < vr; ++k) s += kt[k] * uj[k];
            v[p] = cval[p] * (1.0 / s);
        }
}

/* Algorithm 3 over v_csc: y[j][k] = sum over doc j's words of A[w][k] * v_wj. */
static void spmm(int32_t vr, int64_t N, const double *A, const csc_map *m, const double *v, double *y)
{
    int64_t j;
#pragma omp parallel for schedule(dynamic, 64)
    for (j = 0; j < N; ++j) {
        double *yj = y + (size_t)j * vr;
        for (int32_t k = 0; k < vr; ++k) yj[k] = 0.0;
        for (int64_t q = m->csc_ptr[j]; q < m->csc_ptr[j + 1]; ++q) {
            const double *a = A + (size_t)m->csc_row[q] * vr;
            double vv = v[m->csc_src[q]];
            for (int32_t k = 0; k < vr; ++k) yj[k] += a[k] * vv;
        }
    }
}

static int sinkhorn_sparse_impl(int32_t vr, int64_t V, int64_t N, const double *K, const double *KM,
                                const double *r, const int64_t *row_ptr, const int32_t *col,
                                const double *cval, int32_t t, double tol, int32_t *iters,
                                double *wmd, double *x_out, double *u_out, double *v_out)
{
    if (vr <= 0 || V <= 0 || N < 0 || t < 0) return ORACLE_EINVAL;
    int64_t nnz = row_ptr[V];
    csc_map m;
    int rc = build_csc(V, N, row_ptr, col, &m);
    double *KT = (double *)malloc(sizeof(double) * (size_t)V * vr);   /* KT = K.T */
    double *KrT = (double *)malloc(sizeof(double) * (size_t)V * vr);  /* K_over_r, word-major */
    double *KMT = (double *)malloc(sizeof(double) * (size_t)V * vr);
    double *x = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * vr);
    double *u = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * vr);
    double *v = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * vr);
    if (rc != ORACLE_OK || !KT || !KrT || !KMT || !x || !u || !v || !y) {
        rc = ORACLE_ENOMEM;
        goto done;
    }
    for (int32_t k = 0; k < vr; ++k)
        for (int64_t w = 0; w < V; ++w) {
            KT[(size_t)w * vr + k] = K[(size_t)k * V + w];
            KrT[(size_t)w * vr + k] = (1.0 / r[k]) * K[(size_t)k * V + w];
            KMT[(size_t)w * vr + k] = KM[(size_t)k * V + w];
        }
    for (int64_t i = 0; i < N * vr; ++i) x[i] = 1.0 / vr;

    int32_t done_it = 0;
    for (;;) {
        for (int64_t i = 0; i < N * vr; ++i) u[i] = 1.0 / x[i];         /* u = 1./x      */
        sddmm(vr, V, KT, u, row_ptr, col, cval, v);                      /* SDDMM         */
        if (tol > 0.0) {
            /* convergence mode: row sums of P = diag(u) K diag(v) against r */
            spmm(vr, N, KT, &m, v, y);
            double err = 0.0;
            for (int64_t j = 0; j < N; ++j)
                for (int32_t k = 0; k < vr; ++k) {
                    double e = fabs(u[(size_t)j * vr + k] * y[(size_t)j * vr + k] - r[k]);
                    if (e > err) err = e;
                }
            if (err < tol || done_it >= t) break;
        } else if (done_it >= t) {
            break;
        }
        spmm(vr, N, KrT, &m, v, x);                                      /* x = K_over_r v */
        ++done_it;
    }
    if (iters) *iters = done_it;
    /* d = sum(u .* ((K .* M) v)) per document */
    spmm(vr, N, KMT, &m, v, y);
    for (int64_t j = 0; j < N; ++j) {
        double d = 0.0;
        for (int32_t k = 0; k < vr; ++k) d += u[(size_t)j * vr + k] * y[(size_t)j * vr + k];
        wmd[j] = d;
    }
    if (x_out) memcpy(x_out, x, sizeof(double) * (size_t)N * vr);
    if (u_out) memcpy(u_out, u, sizeof(double) * (size_t)N * vr);
    if (v_out) memcpy(v_out, v, sizeof(double) * (size_t)nnz);
done:
    free_csc(&m);
    free(KT); free(KrT); free(KMT); free(x); free(u); free(v); free(y);
    return rc;
}

int oracle_sinkhorn_sparse(int32_t vr, int64_t V, int64_t N, const double *K, const double *KM,
                           const double *r, const int64_t *row_ptr, const int32_t *col,
                           const double *cval, int32_t t, double *wmd, double *x_out,
                           double *u_out, double *v_out)
{
    return sinkhorn_sparse_impl(vr, V, N, K, KM, r, row_ptr, col, cval, t, 0.0, NULL, wmd, x_out,
                                u_out, v_out);
}

/* Convergence mode ("while x changes", Algorithm 1): iterate until every row sum
 * of the plan is within tol of r, or max_iter updates have run. */
int oracle_sinkhorn_converge(int32_t vr, int64_t V, int64_t N, const double *K, const double *KM,
                             const double *r, const int64_t *row_ptr, const int32_t *col,
                             const double *cval, int32_t max_iter, double tol, int32_t *iters,
                             double *wmd, double *u_out, double *v_out)
{
    if (!(tol > 0.0)) return ORACLE_EINVAL;
    return sinkhorn_sparse_impl(vr, V, N, K, KM, r, row_ptr, col, cval, max_iter, tol, iters, wmd,
                                NULL, u_out, v_out);
}

/* The whole problem statement (Section III-B1): sinkhorn_wmd(r, c, vecs, lambda,
 * max_iter) with r given as (id, weight) pairs and c as a V x N CSR.
 * mode 0 = sparse, 1 = dense.  Returns 0 or ORACLE_EINVAL / ORACLE_ENOMEM. */
int oracle_wmd(int64_t V, int32_t d, const float *E, int64_t N, const int64_t *row_ptr,
               const int32_t *col, const float *cval_in, int64_t nq, const int32_t *q_ids,
               const float *q_w, double lambda, int32_t t, int32_t mode, double *wmd)
{
    if (!(lambda > 0.0) || isinf(lambda) || t < 0 || d <= 0) return ORACLE_EINVAL;
    int64_t nnz = row_ptr[V];
    int rc = ORACLE_OK;
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nq > 0 ? nq : 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(nq > 0 ? nq : 1));
    double *w = (double *)malloc(sizeof(double) * (size_t)(nq > 0 ? nq : 1));
    double *craw = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double *c = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double *M = NULL, *K = NULL, *KM = NULL;
    if (!sel || !r || !w || !craw || !c) { rc = ORACLE_ENOMEM; goto out; }
    for (int64_t i = 0; i < nq; ++i) w[i] = (double)q_w[i];
    int64_t vr = oracle_select(V, nq, q_ids, w, sel, r);
    if (vr <= 0) { rc = (int)(vr < 0 ? vr : ORACLE_EINVAL); goto out; }
    for (int64_t p = 0; p < nnz; ++p) craw[p] = (double)cval_in[p];
    rc = oracle_normalize_columns(V, N, row_ptr, col, craw, c);
    if (rc != ORACLE_OK) goto out;
    M = (double *)malloc(sizeof(double) * (size_t)vr * V);
    K = (double *)malloc(sizeof(double) * (size_t)vr * V);
    KM = (double *)malloc(sizeof(double) * (size_t)vr * V);
    if (!M || !K || !KM) { rc = ORACLE_ENOMEM; goto out; }
    oracle_cdist(V, d, E, (int32_t)vr, sel, M);
    oracle_kernel(vr * V, M, lambda, K, KM);
    if (mode == 1)
        rc = oracle_sinkhorn_dense((int32_t)vr, V, N, K, KM, r, row_ptr, col, c, t, 64, wmd, NULL);
    else
        rc = oracle_sinkhorn_sparse((int32_t)vr, V, N, K, KM, r, row_ptr, col, c, t, wmd, NULL, NULL,
                                    NULL);
out:
    free(sel); free(r); free(w); free(craw); free(c); free(M); free(K); free(KM);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* 1-to-1 WMD (Section III-E, Table II, right column): the distance of one query
 * histogram to ONE target histogram, with the cost matrix built only over the
 * target's v_x distinct words (v_r x v_x) instead of the whole vocabulary.
 * Algorithm 1 with a single column c: every word outside the target has c = 0,
 * so its v entry is 0 and it adds nothing to x = K_over_r v or to the final sum;
 * dropping those words is the restriction that gives Table II's per-pair cost.
 *
 * Both sides are selected and normalised as Section III-B1 does for r and for a
 * column of c (repeated ids add up, zero weights dropped, sum 1).  The target's
 * words become the vocabulary of a one-column problem solved by the dense
 * routine above (tol == 0: exactly t x-updates) or by the convergence mode
 * (tol > 0).
 *
 * Pair p: query (q_ids, q_w)[q_ptr[p] .. q_ptr[p+1]), target (x_ids, x_w)
 * [x_ptr[p] .. x_ptr[p+1]).  wmd[n_pairs]; iters[n_pairs] (optional) receives
 * the x-updates run.  Returns 0 or the first failing pair's error code. */
static int wmd_pair_one(int64_t V, int32_t d, const float *E, int64_t nq, const int32_t *qi,
                        const float *qw, int64_t nx, const int32_t *xi, const float *xw,
                        double lambda, int32_t t, double tol, double *wmd, int32_t *iters)
{
    int rc = ORACLE_OK;
    int64_t nmax = nq > nx ? nq : nx;
    if (nmax < 1) nmax = 1;
    int32_t *sq = (int32_t *)malloc(sizeof(int32_t) * (size_t)nmax);
    int32_t *sx = (int32_t *)malloc(sizeof(int32_t) * (size_t)nmax);
    double *r = (double *)malloc(sizeof(double) * (size_t)nmax);
    double *cx = (double *)malloc(sizeof(double) * (size_t)nmax);
    double *w = (double *)malloc(sizeof(double) * (size_t)nmax);
    double *M = NULL, *K = NULL, *KM = NULL;
    int64_t *rp = NULL;
    int32_t *col = NULL;
    if (!sq || !sx || !r || !cx || !w) { rc = ORACLE_ENOMEM; goto out; }
    for (int64_t i = 0; i < nq; ++i) w[i] = (double)qw[i];
    int64_t vr = oracle_select(V, nq, qi, w, sq, r);
    if (vr <= 0) { rc = (int)(vr < 0 ? vr : ORACLE_EINVAL); goto out; }
    for (int64_t i = 0; i < nx; ++i) w[i] = (double)xw[i];
    int64_t vx = oracle_select(V, nx, xi, w, sx, cx);
    if (vx <= 0) { rc = (int)(vx < 0 ? vx : ORACLE_EINVAL); goto out; }

    /* M[k][j] = ||E[q_k] - E[x_j]||_2 over the target's words only (Section II-A) */
    M = (double *)malloc(sizeof(double) * (size_t)(vr * vx));
    K = (double *)malloc(sizeof(double) * (size_t)(vr * vx));
    KM = (double *)malloc(sizeof(double) * (size_t)(vr * vx));
    rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(vx + 1));
    col = (int32_t *)calloc((size_t)vx, sizeof(int32_t));
    if (!M || !K || !KM || !rp || !col) { rc = ORACLE_ENOMEM; goto out; }
    for (int64_t k = 0; k < vr; ++k)
        for (int64_t j = 0; j < vx; ++j) {
            const float *a = E + (size_t)sq[k] * d;
            const float *b = E + (size_t)sx[j] * d;
            double acc = 0.0;
            for (int32_t e = 0; e < d; ++e) {
                double diff = (double)a[e] - (double)b[e];
                acc += diff * diff;
            }
            M[(size_t)k * vx + j] = sqrt(acc);
        }
    oracle_kernel(vr * vx, M, lambda, K, KM);
    /* c as a vx x 1 CSR: target word j is row j, one nonzero in column 0 */
    for (int64_t j = 0; j <= vx; ++j) rp[j] = j;
    if (tol > 0.0) {
        rc = oracle_sinkhorn_converge((int32_t)vr, vx, 1, K, KM, r, rp, col, cx, t, tol, iters,
                                      wmd, NULL, NULL);
    } else {
        rc = oracle_sinkhorn_dense((int32_t)vr, vx, 1, K, KM, r, rp, col, cx, t, 1, wmd, NULL);
        if (iters) *iters = t;
    }
out:
    free(sq); free(sx); free(r); free(cx); free(w);
    free(M); free(K); free(KM); free(rp); free(col);
    return rc;
}

int oracle_wmd_pairs(int64_t V, int32_t d, const float *E, int64_t n_pairs, const int64_t *q_ptr,
                     const int32_t *q_ids, const float *q_w, const int64_t *x_ptr,
                     const int32_t *x_ids, const float *x_w, double lambda, int32_t t, double tol,
                     double *wmd, int32_t *iters)
{
    if (!(lambda > 0.0) || isinf(lambda) || t < 0 || d <= 0 || n_pairs < 0 || !(tol >= 0.0))
        return ORACLE_EINVAL;
    int rc = ORACLE_OK;
    int64_t p;
    /* pairs are independent; each writes only its own outputs */
#pragma omp parallel for schedule(dynamic, 1)
    for (p = 0; p < n_pairs; ++p) {
        int32_t it = 0;
        int e = wmd_pair_one(V, d, E, q_ptr[p + 1] - q_ptr[p], q_ids + q_ptr[p], q_w + q_ptr[p],
                             x_ptr[p + 1] - x_ptr[p], x_ids + x_ptr[p], x_w + x_ptr[p], lambda, t,
                             tol, wmd + p, &it);
        if (iters) iters[p] = it;
        if (e != ORACLE_OK) {
#pragma omp critical
            if (rc == ORACLE_OK) rc = e;
        }
    }
    return rc;
}
