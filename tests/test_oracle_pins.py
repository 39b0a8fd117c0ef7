"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test fixes the oracle to something the paper or the mathematics determines:
library routines (scipy cdist, scipy linprog), closed forms of Algorithm 1 for
degenerate inputs, marginal invariants of the Sinkhorn plan, brute-force exact
EMD on tiny equal-mass instances, exact invariances, and agreement of the dense
(Algorithm 1 / Table I) and sparse (Algorithms 2-3) formulations.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2107_06433_gb300 import synth


def _unit_rows(rng, V, d):
    E = rng.standard_normal((V, d)).astype(np.float32)
    return E / np.linalg.norm(E, axis=1, keepdims=True)


def _direct_dist(E, a, b):
    """Euclidean distance of two embedding rows, written out in numpy."""
    diff = E[a].astype(np.float64) - E[b].astype(np.float64)
    return float(np.sqrt(np.sum(diff * diff)))


def _csr_from_docs(V, docs):
    """docs: list of {word: weight}.  Returns V x N CSR (row_ptr, col, val)."""
    rows = [[] for _ in range(V)]
    for j, doc in enumerate(docs):
        for w, x in doc.items():
            rows[w].append((j, x))
    row_ptr = [0]
    col, val = [], []
    for w in range(V):
        for j, x in sorted(rows[w]):
            col.append(j)
            val.append(x)
        row_ptr.append(len(col))
    return (np.array(row_ptr, np.int64), np.array(col, np.int32), np.array(val, np.float64))


# --------------------------------------------------------------------------- basics

def test_cdist_matches_scipy(tiny):
    from scipy.spatial.distance import cdist as sp_cdist
    E, C, (qi, qw) = tiny
    M = oracle.cdist(E, qi)
    ref = sp_cdist(E[qi].astype(np.float64), E.astype(np.float64))
    np.testing.assert_allclose(M, ref, rtol=1e-12, atol=1e-14)
    assert np.all(M[np.arange(len(qi)), qi] == 0.0)


def test_kernel_is_exp_of_minus_lambda_m():
    M = np.linspace(0.0, 2.0, 101).reshape(1, -1)
    for lam in (0.5, 1.0, 10.0):
        K, KM = oracle.kernel(M, lam)
        np.testing.assert_allclose(K, np.exp(-lam * M), rtol=1e-15)
        np.testing.assert_allclose(KM, np.exp(-lam * M) * M, rtol=1e-15)
        assert np.all(K <= 1.0)          # lambda > 0: exp(-lambda M) never exceeds 1


def test_select_merges_drops_normalises():
    ids, r = oracle.select(10, [7, 3, 7, 5, 1], [1.0, 2.0, 3.0, 0.0, 2.0])
    assert ids.tolist() == [1, 3, 7]      # zero weight dropped, ascending, merged
    np.testing.assert_allclose(r, [2 / 8, 2 / 8, 4 / 8], rtol=1e-15)
    for bad_ids, bad_w in (([10], [1.0]), ([-1], [1.0]), ([2], [-1.0]), ([2], [np.nan]),
                           ([2], [0.0])):
        with pytest.raises(oracle.OracleError):
            oracle.select(10, bad_ids, bad_w)


def test_normalize_columns_and_rejections():
    rp, col, val = _csr_from_docs(4, [{0: 2.0, 3: 6.0}, {1: 1.0}])
    out = oracle.normalize_columns(4, 2, rp, col, val)
    np.testing.assert_allclose(out, [0.25, 1.0, 0.75])
    with pytest.raises(oracle.OracleError):          # empty third column
        oracle.normalize_columns(4, 3, rp, col, val)
    with pytest.raises(oracle.OracleError):          # non-positive value
        oracle.normalize_columns(4, 2, rp, col, np.array([2.0, 0.0, 6.0]))


# --------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("t", [0, 1, 7])
@pytest.mark.parametrize("lam", [0.3, 1.0, 10.0])
@pytest.mark.parametrize("mode", ["sparse", "dense"])
def test_single_word_query_is_transport_to_every_word(t, lam, mode):
    """v_r = 1: the plan has one row and its column sums are c, so
    WMD_j = sum_w c_wj M[q, w] exactly, for any lambda and any t."""
    rng = np.random.default_rng(11)
    V, N = 40, 12
    E = _unit_rows(rng, V, 7)
    docs = []
    for j in range(N):
        ws = rng.choice(V, size=rng.integers(1, 8), replace=False)
        docs.append({int(w): float(rng.integers(1, 5)) for w in ws})
    rp, col, val = _csr_from_docs(V, docs)
    q = 5
    got = oracle.wmd(E, rp, col, val.astype(np.float32), N, [q], [1.0], lam, t, mode)
    for j, doc in enumerate(docs):
        tot = sum(doc.values())
        expect = sum(x / tot * _direct_dist(E, q, w) for w, x in doc.items())
        assert got[j] == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("t", [1, 2, 15])
@pytest.mark.parametrize("lam", [0.5, 1.0, 10.0])
def test_single_word_document_is_mean_distance_from_query(t, lam):
    """A document of one word w: one x-update reaches the fixed point and
    WMD = sum_i r_i M[q_i, w] for t >= 1."""
    rng = np.random.default_rng(12)
    V = 30
    E = _unit_rows(rng, V, 6)
    qi = [2, 9, 17, 23]
    qw = [1.0, 3.0, 2.0, 2.0]
    docs = [{w: 1.0} for w in (0, 9, 29, 14)]
    rp, col, val = _csr_from_docs(V, docs)
    got = oracle.wmd(E, rp, col, val.astype(np.float32), len(docs), qi, qw, lam, t)
    tot = sum(qw)
    for j, doc in enumerate(docs):
        (w,) = doc.keys()
        expect = sum(wi / tot * _direct_dist(E, i, w) for i, wi in zip(qi, qw))
        assert got[j] == pytest.approx(expect, rel=1e-12)


def test_both_single_is_the_word_distance():
    rng = np.random.default_rng(13)
    E = _unit_rows(rng, 8, 5)
    rp, col, val = _csr_from_docs(8, [{6: 1.0}, {3: 2.0}])
    got = oracle.wmd(E, rp, col, val.astype(np.float32), 2, [3], [1.0], 1.0, 15)
    assert got[0] == pytest.approx(_direct_dist(E, 3, 6), rel=1e-13)
    assert got[1] == 0.0


@pytest.mark.parametrize("lam", [0.5, 1.0, 10.0])
def test_zero_iterations_is_softmin_average(lam):
    """t = 0: x keeps its initial value 1/v_r, so u is uniform and the final step
    gives WMD_j = sum_w c_wj sum_k softmax_k(-lambda M[k,w]) M[k,w]."""
    E, C, (qi, qw) = synth.make("tiny", N=30)
    rp, col, val = C.csr()
    got = oracle.wmd(E, rp, col, val, C.N, qi, qw, lam, 0)
    for j in range(C.N):
        words = C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]]
        cv = C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]].astype(np.float64)
        cv /= cv.sum()
        tot = 0.0
        for w, cw in zip(words, cv):
            m = np.array([_direct_dist(E, k, w) for k in qi])
            a = np.exp(-lam * (m - m.min()))
            tot += cw * float(np.sum(a * m) / np.sum(a))
        assert got[j] == pytest.approx(tot, rel=1e-12)


# --------------------------------------------------------------------------- marginals

def _plans(K, u, v, rp, col, N):
    """Per document, P = diag(u_j) K[:, words] diag(v_j) as {j: (words, P)}."""
    V = len(rp) - 1
    per = {j: ([], []) for j in range(N)}
    for w in range(V):
        for p in range(rp[w], rp[w + 1]):
            per[int(col[p])][0].append(w)
            per[int(col[p])][1].append(v[p])
    out = {}
    for j, (ws, vs) in per.items():
        ws = np.array(ws)
        out[j] = (ws, u[j][:, None] * K[:, ws] * np.array(vs)[None, :])
    return out


@pytest.mark.parametrize("t", [0, 3, 15])
def test_column_marginal_is_c_after_final_step(tiny, t):
    E, C, (qi, qw) = tiny
    rp, col, val = C.csr()
    ids, r = oracle.select(C.V, qi, qw)
    K, KM = oracle.kernel(oracle.cdist(E, ids), 1.0)
    c = oracle.normalize_columns(C.V, C.N, rp, col, val)
    wmd, x, u, v = oracle.sinkhorn_sparse(K, KM, r, C.N, rp, col, c, t, want_state=True)
    M = oracle.cdist(E, ids)
    for j, (ws, P) in _plans(K, u, v, rp, col, C.N).items():
        cj = {int(w): 0.0 for w in ws}
        for w in range(C.V):
            for p in range(rp[w], rp[w + 1]):
                if col[p] == j:
                    cj[w] = c[p]
        np.testing.assert_allclose(P.sum(axis=0), [cj[int(w)] for w in ws], rtol=1e-12)
        # the reported distance is <P, M> (transport cost without the entropy term)
        assert wmd[j] == pytest.approx(float(np.sum(P * M[:, ws])), rel=1e-12)


def test_row_marginal_converges_to_r(tiny):
    E, C, (qi, qw) = tiny
    rp, col, val = C.csr()
    ids, r = oracle.select(C.V, qi, qw)
    K, KM = oracle.kernel(oracle.cdist(E, ids), 1.0)
    c = oracle.normalize_columns(C.V, C.N, rp, col, val)
    errs = []
    for t in (1, 4, 16, 64):
        _, _, u, v = oracle.sinkhorn_sparse(K, KM, r, C.N, rp, col, c, t, want_state=True)
        errs.append(max(np.max(np.abs(P.sum(axis=1) - r))
                        for _, P in _plans(K, u, v, rp, col, C.N).values()))
    assert errs[-1] < errs[0]
    wmd, it, u, v = oracle.sinkhorn_converge(K, KM, r, C.N, rp, col, c, tol=1e-12)
    assert it < 100000
    for _, P in _plans(K, u, v, rp, col, C.N).values():
        np.testing.assert_allclose(P.sum(axis=1), r, atol=1e-12)


# --------------------------------------------------------------------------- lambda limit

def _entropy(p):
    p = np.asarray(p, dtype=np.float64)
    p = p[p > 0]
    return float(-np.sum(p * np.log(p)))


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_lambda_limit_against_brute_force_emd(n):
    """Equal-mass uniform n x n: the exact EMD is a permutation (Birkhoff), found by
    enumerating all n! of them.  Converged Sinkhorn cost S_lambda = <P_lambda, M>
    satisfies 0 <= S - EMD <= (H(P_lambda) - H(P*))/lambda <= ln(n)/lambda and is
    non-increasing in lambda."""
    rng = np.random.default_rng(100 + n)
    V = 2 * n
    E = _unit_rows(rng, V, 4)
    Mq = np.array([[_direct_dist(E, i, n + j) for j in range(n)] for i in range(n)])
    emd = min(sum(Mq[i, p[i]] for i in range(n)) / n
              for p in itertools.permutations(range(n)))
    rp, col, val = _csr_from_docs(V, [{n + j: 1.0 for j in range(n)}])
    ids, r = oracle.select(V, list(range(n)), [1.0] * n)
    M = oracle.cdist(E, ids)
    c = oracle.normalize_columns(V, 1, rp, col, val)
    prev = None
    for lam in (1.0, 2.0, 5.0, 10.0, 20.0, 50.0):
        K, KM = oracle.kernel(M, lam)
        wmd, it, u, v = oracle.sinkhorn_converge(K, KM, r, 1, rp, col, c, tol=1e-11,
                                                 max_iter=400000)
        (ws, P), = _plans(K, u, v, rp, col, 1).values()
        slack = 2 * 2.0 * float(np.sum(np.abs(P.sum(axis=1) - r))) + 1e-12
        S = wmd[0]
        assert S >= emd - slack
        assert S - emd <= math.log(n) / lam + slack
        if prev is not None:
            assert S <= prev + slack
        prev = S


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lambda_limit_against_linear_program(seed):
    """Unequal masses: exact EMD from scipy's LP solver; the entropic gap is at most
    min(H(r), H(c)) / lambda."""
    from scipy.optimize import linprog
    rng = np.random.default_rng(200 + seed)
    nq, nd = 4, 5
    V = nq + nd
    E = _unit_rows(rng, V, 3)
    qw = rng.integers(1, 6, size=nq).astype(np.float64)
    cw = rng.integers(1, 6, size=nd).astype(np.float64)
    rp, col, val = _csr_from_docs(V, [{nq + j: float(cw[j]) for j in range(nd)}])
    ids, r = oracle.select(V, list(range(nq)), qw)
    c = oracle.normalize_columns(V, 1, rp, col, val)
    M = oracle.cdist(E, ids)
    Msub = M[:, nq:]
    A_eq = []
    for i in range(nq):
        row = np.zeros((nq, nd)); row[i, :] = 1; A_eq.append(row.ravel())
    for j in range(nd):
        row = np.zeros((nq, nd)); row[:, j] = 1; A_eq.append(row.ravel())
    b_eq = np.concatenate([r, c])
    lp = linprog(Msub.ravel(), A_eq=np.array(A_eq), b_eq=b_eq, bounds=(0, None),
                 method="highs")
    assert lp.status == 0
    emd = lp.fun
    gap_bound = min(_entropy(r), _entropy(c))
    for lam in (2.0, 10.0, 40.0):
        K, KM = oracle.kernel(M, lam)
        wmd, it, u, v = oracle.sinkhorn_converge(K, KM, r, 1, rp, col, c, tol=1e-11,
                                                 max_iter=400000)
        (ws, P), = _plans(K, u, v, rp, col, 1).values()
        slack = 2 * 2.0 * float(np.sum(np.abs(P.sum(axis=1) - r))) + 1e-9
        assert emd - slack <= wmd[0] <= emd + gap_bound / lam + slack


# --------------------------------------------------------------------------- invariances

def test_dense_equals_sparse(tiny):
    E, C, (qi, qw) = tiny
    rp, col, val = C.csr()
    for t in (0, 1, 15):
        a = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, t, "sparse")
        b = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, t, "dense")
        np.testing.assert_allclose(a, b, rtol=1e-13)


def test_dense_equals_sparse_paper_shaped_subset():
    E, C, (qi, qw) = synth.make("paper", N=120)
    rp, col, val = C.csr()
    a = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, 15, "sparse")
    b = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, 15, "dense")
    np.testing.assert_allclose(a, b, rtol=1e-13)


def test_document_permutation_and_subset(tiny):
    E, C, (qi, qw) = tiny
    rp, col, val = C.csr()
    full = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, 15)
    perm = np.random.default_rng(5).permutation(C.N)
    inv = np.empty_like(perm); inv[perm] = np.arange(C.N)
    col_p = inv[col].astype(np.int32)           # document j moves to column inv[j]
    order = np.lexsort((col_p, np.repeat(np.arange(C.V), np.diff(rp))))
    permuted = oracle.wmd(E, rp, col_p[order], val[order], C.N, qi, qw, 1.0, 15)
    np.testing.assert_array_equal(permuted[inv], full)
    keep = np.arange(0, C.N, 3)
    sub = np.isin(col, keep)
    remap = np.full(C.N, -1); remap[keep] = np.arange(len(keep))
    rows = np.repeat(np.arange(C.V), np.diff(rp))[sub]
    rp_s = np.zeros(C.V + 1, np.int64); np.cumsum(np.bincount(rows, minlength=C.V), out=rp_s[1:])
    part = oracle.wmd(E, rp_s, remap[col[sub]].astype(np.int32), val[sub], len(keep), qi, qw,
                      1.0, 15)
    np.testing.assert_array_equal(part, full[keep])


@pytest.mark.parametrize("t", [0, 5, 15])
def test_column_rescaling_of_k_is_exact(tiny, t):
    """K' = K diag(b) gives v' = v / b and the same x at every step, so the
    distance is unchanged for every t (the column shift a GPU path may use)."""
    E, C, (qi, qw) = tiny
    rp, col, val = C.csr()
    ids, r = oracle.select(C.V, qi, qw)
    M = oracle.cdist(E, ids)
    K, KM = oracle.kernel(M, 3.0)
    c = oracle.normalize_columns(C.V, C.N, rp, col, val)
    base = oracle.sinkhorn_sparse(K, KM, r, C.N, rp, col, c, t)
    b = np.exp(3.0 * M.min(axis=0))              # makes every column's largest K equal 1
    alt = oracle.sinkhorn_sparse(K * b, KM * b, r, C.N, rp, col, c, t)
    np.testing.assert_allclose(alt, base, rtol=1e-12)


def test_row_rescaling_only_at_convergence(tiny):
    E, C, (qi, qw) = tiny
    rp, col, val = C.csr()
    ids, r = oracle.select(C.V, qi, qw)
    M = oracle.cdist(E, ids)
    K, KM = oracle.kernel(M, 1.0)
    c = oracle.normalize_columns(C.V, C.N, rp, col, val)
    a = np.linspace(0.5, 2.0, len(ids))[:, None]
    base, _, _, _ = oracle.sinkhorn_converge(K, KM, r, C.N, rp, col, c, tol=1e-13)
    alt, _, _, _ = oracle.sinkhorn_converge(K * a, KM * a, r, C.N, rp, col, c, tol=1e-13)
    np.testing.assert_allclose(alt, base, rtol=1e-10)
    two = oracle.sinkhorn_sparse(K, KM, r, C.N, rp, col, c, 2)
    two_alt = oracle.sinkhorn_sparse(K * a, KM * a, r, C.N, rp, col, c, 2)
    assert np.max(np.abs(two - two_alt)) > 1e-9


def test_per_nonzero_form_of_the_final_step(tiny):
    """sum_k u_k ((K.*M) v)_k = sum_w c_w (KM^T u)_w / (K^T u)_w, the form the
    final fused reduction evaluates."""
    E, C, (qi, qw) = tiny
    rp, col, val = C.csr()
    ids, r = oracle.select(C.V, qi, qw)
    K, KM = oracle.kernel(oracle.cdist(E, ids), 1.0)
    c = oracle.normalize_columns(C.V, C.N, rp, col, val)
    wmd, x, u, v = oracle.sinkhorn_sparse(K, KM, r, C.N, rp, col, c, 15, want_state=True)
    alt = np.zeros(C.N)
    for w in range(C.V):
        for p in range(rp[w], rp[w + 1]):
            j = col[p]
            alt[j] += c[p] * float(KM[:, w] @ u[j]) / float(K[:, w] @ u[j])
    np.testing.assert_allclose(alt, wmd, rtol=1e-13)


def test_thread_count_does_not_change_results(tiny):
    E, C, (qi, qw) = tiny
    rp, col, val = C.csr()
    n0 = oracle.get_threads()
    try:
        oracle.set_threads(1)
        one = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, 15)
        oracle.set_threads(max(2, n0))
        many = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, 15)
    finally:
        oracle.set_threads(n0)
    np.testing.assert_array_equal(one, many)


def test_golden_tiny_values(tiny):
    """Regression against the stored oracle output for the tiny workload."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_wmd.txt")
    ref = np.loadtxt(path)
    E, C, (qi, qw) = tiny
    rp, col, val = C.csr()
    got = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, 15)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


# --------------------------------------------------------------------------- 1-to-1 WMD

def _doc_side(C, j):
    lo, hi = C.doc_ptr[j], C.doc_ptr[j + 1]
    return C.word_ids[lo:hi], C.vals[lo:hi]


@pytest.mark.parametrize("t", [0, 1, 15])
@pytest.mark.parametrize("lam", [1.0, 10.0])
@pytest.mark.parametrize("workload", ["tiny", "paper"])
def test_pair_equals_column_of_the_one_to_many_problem(t, lam, workload):
    """Table II's 1-to-1 problem builds the cost only over the target's words.  Every
    other word has c = 0 in Algorithm 1, so v = 0 there and it adds nothing: the pair
    distance equals that document's entry of the 1-to-N result."""
    E, C, (qi, qw) = synth.make(workload, N=40) if workload == "paper" else synth.make("tiny")
    rp, col, val = C.csr()
    full = oracle.wmd(E, rp, col, val, C.N, qi, qw, lam, t)
    pairs = oracle.wmd_pairs(E, [(qi, qw)] * C.N, [_doc_side(C, j) for j in range(C.N)], lam, t)
    np.testing.assert_allclose(pairs, full, rtol=1e-12)


@pytest.mark.parametrize("t", [0, 3, 15])
def test_pair_single_word_sides_are_closed_forms(t):
    """One query word: WMD = sum_j c_j M[q, x_j] (any t).  One target word, t >= 1:
    WMD = sum_k r_k M[q_k, x].  Both: the word distance."""
    rng = np.random.default_rng(21)
    V = 50
    E = _unit_rows(rng, V, 9)
    xs, xw = [3, 17, 40, 41], [2.0, 1.0, 4.0, 1.0]
    qs, qw = [0, 5, 17, 33, 49], [1.0, 1.0, 3.0, 2.0, 1.0]
    got = oracle.wmd_pairs(E, [([7], [1.0]), (qs, qw), ([7], [2.0])],
                           [(xs, xw), ([11], [1.0]), ([30], [5.0])], 2.0, t)
    expect0 = sum(w / sum(xw) * _direct_dist(E, 7, x) for x, w in zip(xs, xw))
    assert got[0] == pytest.approx(expect0, rel=1e-12)
    if t >= 1:
        expect1 = sum(w / sum(qw) * _direct_dist(E, q, 11) for q, w in zip(qs, qw))
        assert got[1] == pytest.approx(expect1, rel=1e-12)
    assert got[2] == pytest.approx(_direct_dist(E, 7, 30), rel=1e-13)


@pytest.mark.parametrize("lam", [0.5, 4.0])
def test_pair_zero_iterations_is_softmin_average(lam):
    """t = 0: u stays uniform and WMD = sum_j c_j sum_k softmax_k(-lam M[k,j]) M[k,j]."""
    rng = np.random.default_rng(22)
    V = 60
    E = _unit_rows(rng, V, 8)
    qs, qw = [1, 9, 22, 37], [3.0, 1.0, 1.0, 2.0]
    xs, xw = [4, 9, 50], [1.0, 2.0, 2.0]
    got = oracle.wmd_pairs(E, [(qs, qw)], [(xs, xw)], lam, 0)[0]
    tot = 0.0
    for x, w in zip(xs, xw):
        m = np.array([_direct_dist(E, q, x) for q in qs])
        a = np.exp(-lam * (m - m.min()))
        tot += w / sum(xw) * float(np.sum(a * m) / np.sum(a))
    assert got == pytest.approx(tot, rel=1e-12)


def test_pair_is_symmetric_at_convergence():
    """The entropic plan is the unique minimiser whichever side Sinkhorn starts from,
    so converged distances satisfy WMD(a, b) = WMD(b, a); after a fixed small t they
    do not (the iteration starts from the query side)."""
    rng = np.random.default_rng(23)
    V = 80
    E = _unit_rows(rng, V, 6)
    A, B = [], []
    for _ in range(6):
        na, nb = int(rng.integers(2, 9)), int(rng.integers(2, 9))
        A.append((rng.choice(V, na, replace=False), rng.integers(1, 6, na).astype(np.float32)))
        B.append((rng.choice(V, nb, replace=False), rng.integers(1, 6, nb).astype(np.float32)))
    ab, it_ab = oracle.wmd_pairs(E, A, B, 3.0, 200000, tol=1e-14, want_iters=True)
    ba, it_ba = oracle.wmd_pairs(E, B, A, 3.0, 200000, tol=1e-14, want_iters=True)
    assert np.all(it_ab < 200000) and np.all(it_ba < 200000)
    np.testing.assert_allclose(ab, ba, rtol=1e-10)
    ab2 = oracle.wmd_pairs(E, A, B, 3.0, 1)
    ba2 = oracle.wmd_pairs(E, B, A, 3.0, 1)
    assert np.max(np.abs(ab2 - ba2)) > 1e-6


@pytest.mark.parametrize("seed", [0, 1])
def test_pair_lambda_limit_against_linear_program(seed):
    """Unequal masses: exact EMD from scipy's LP; the converged entropic cost lies
    within min(H(r), H(c)) / lambda above it and falls as lambda grows."""
    from scipy.optimize import linprog
    rng = np.random.default_rng(300 + seed)
    V = 40
    E = _unit_rows(rng, V, 3)
    qs = rng.choice(V, 4, replace=False)
    xs = rng.choice(V, 5, replace=False)
    qw = rng.integers(1, 6, 4).astype(np.float64)
    xw = rng.integers(1, 6, 5).astype(np.float64)
    r, c = qw / qw.sum(), xw / xw.sum()
    M = np.array([[_direct_dist(E, a, b) for b in xs] for a in qs])
    A_eq = np.zeros((4 + 5, 20))
    for i in range(4):
        A_eq[i, i * 5:(i + 1) * 5] = 1.0
    for j in range(5):
        A_eq[4 + j, j::5] = 1.0
    lp = linprog(M.ravel(), A_eq=A_eq, b_eq=np.concatenate([r, c]), bounds=(0, None),
                 method="highs")
    emd = lp.fun
    prev = None
    for lam in (2.0, 8.0, 32.0, 128.0):
        S = oracle.wmd_pairs(E, [(qs, qw.astype(np.float32))], [(xs, xw.astype(np.float32))],
                             lam, 400000, tol=1e-12)[0]
        assert S >= emd - 1e-9
        assert S - emd <= min(_entropy(r), _entropy(c)) / lam + 1e-9
        if prev is not None:
            assert S <= prev + 1e-9
        prev = S


def test_pair_merges_duplicates_and_drops_zeros():
    rng = np.random.default_rng(24)
    E = _unit_rows(rng, 30, 5)
    merged = oracle.wmd_pairs(E, [([2, 8], [1.0, 3.0])], [([4, 20, 21], [2.0, 1.0, 1.0])], 1.0, 9)
    split = oracle.wmd_pairs(E, [([8, 2, 8, 11], [1.0, 1.0, 2.0, 0.0])],
                             [([21, 4, 20, 4, 6], [1.0, 1.5, 1.0, 0.5, 0.0])], 1.0, 9)
    np.testing.assert_array_equal(merged, split)


def test_pair_rejects_invalid_sides():
    rng = np.random.default_rng(25)
    E = _unit_rows(rng, 10, 3)
    ok = ([1, 2], [1.0, 1.0])
    for bad in (([1, 10], [1.0, 1.0]), ([1, -1], [1.0, 1.0]), ([1, 2], [1.0, -1.0]),
                ([1, 2], [0.0, 0.0]), ([], [])):
        with pytest.raises(oracle.OracleError):
            oracle.wmd_pairs(E, [ok], [bad], 1.0, 3)
        with pytest.raises(oracle.OracleError):
            oracle.wmd_pairs(E, [bad], [ok], 1.0, 3)
    with pytest.raises(oracle.OracleError):
        oracle.wmd_pairs(E, [ok], [ok], 0.0, 3)


def test_pair_equals_column_on_random_instances():
    """Property form of the Table II restriction: random vocabularies, embeddings,
    histograms with repeated ids and zero weights, lambda and t."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=40, deadline=None, derandomize=True)
    @hyp.given(seed=st.integers(0, 2**31 - 1), lam=st.sampled_from([0.5, 1.0, 4.0, 20.0]),
               t=st.integers(0, 12))
    def check(seed, lam, t):
        rng = np.random.default_rng(seed)
        V = int(rng.integers(6, 40))
        E = _unit_rows(rng, V, int(rng.integers(2, 9)))
        nq, nx = int(rng.integers(1, 8)), int(rng.integers(1, 8))
        qi = rng.integers(0, V, nq)
        qw = rng.integers(0, 4, nq).astype(np.float32)
        qw[0] = max(qw[0], 1.0)
        xi = rng.integers(0, V, nx)
        xw = rng.integers(0, 4, nx).astype(np.float32)
        xw[0] = max(xw[0], 1.0)
        doc = {}
        for w_, c_ in zip(xi, xw):
            if c_ > 0:
                doc[int(w_)] = doc.get(int(w_), 0.0) + float(c_)
        rp, col, val = _csr_from_docs(V, [doc])
        full = oracle.wmd(E, rp, col, val.astype(np.float32), 1, qi, qw, lam, t)
        pair = oracle.wmd_pairs(E, [(qi, qw)], [(xi, xw)], lam, t)
        np.testing.assert_allclose(pair, full, rtol=1e-12)

    check()


def test_golden_tiny_pairs(tiny):
    """Regression against the stored oracle output of 50 document-to-document pairs."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_pairs.txt")
    ref = np.loadtxt(path)
    E, C, _ = tiny
    docs = [(C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]], C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]])
            for j in range(51)]
    got = oracle.wmd_pairs(E, docs[:50], docs[1:51], 2.0, 10)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


@pytest.mark.parametrize("t", [0, 1, 6])
def test_pair_convergence_mode_capped_at_t_is_the_fixed_t_result(t):
    """With a tolerance no iteration reaches, the convergence mode runs exactly its cap
    of t x-updates (through the sparse routine) and must equal the fixed-t result
    (through the dense routine)."""
    rng = np.random.default_rng(31)
    V = 50
    E = _unit_rows(rng, V, 7)
    # two or more words on each side: a single-word side meets its marginal exactly
    # after one update, which would stop the convergence mode early (correctly)
    A = [(rng.choice(V, n, replace=False), rng.integers(1, 5, n).astype(np.float32)) for n in (2, 3, 6)]
    B = [(rng.choice(V, n, replace=False), rng.integers(1, 5, n).astype(np.float32)) for n in (4, 2, 9)]
    fixed = oracle.wmd_pairs(E, A, B, 2.0, t)
    capped, its = oracle.wmd_pairs(E, A, B, 2.0, t, tol=1e-300, want_iters=True)
    assert np.all(its == t)
    np.testing.assert_allclose(capped, fixed, rtol=1e-13)
