"""Parity of the 1-to-1 pair path (Section III-E, Table II) with the FP64 oracle.

The pair kernel builds each pair's cost over the target's words only and runs all
of Algorithm 1 for it in one block.  FP32 tolerance as for the 1-to-N path: 1e-5
relative per distance.
"""
import numpy as np
import pytest

import oracle
import paper_2107_06433_gb300 as swmd
from paper_2107_06433_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2107_06433_gb300 import build
    build.build()
    oracle.build()


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)))


@pytest.fixture(scope="module")
def paper():
    E, C, (qi, qw) = synth.make("paper", N=600)
    corpus = swmd.corpus_from_synth(E, C)
    yield E, C, (qi, qw), corpus
    corpus.close()


def doc(C, j):
    lo, hi = C.doc_ptr[j], C.doc_ptr[j + 1]
    return C.word_ids[lo:hi], C.vals[lo:hi]


def random_side(rng, V, n):
    ids = rng.choice(V, size=n, replace=False).astype(np.int32)
    return ids, rng.integers(1, 10, size=n).astype(np.float32)


@pytest.mark.parametrize("t", [0, 1, 15])
@pytest.mark.parametrize("lam", [1.0, 10.0])
def test_query_against_documents_matches_oracle(paper, t, lam):
    E, C, (qi, qw), corpus = paper
    docs = [doc(C, j) for j in range(200)]
    got = swmd.swmd_wmd_pairs(corpus, [(qi, qw)] * len(docs), docs, lam, t)
    ref = oracle.wmd_pairs(E, [(qi, qw)] * len(docs), docs, lam, t)
    assert rel_err(got, ref) <= RTOL


def test_pairs_equal_the_one_to_many_column(paper):
    """A pair's distance is that document's entry of the 1-to-N query (both within
    1e-5 of the oracle, so within 2e-5 of each other)."""
    E, C, (qi, qw), corpus = paper
    full = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
    got = swmd.swmd_wmd_pairs(corpus, [(qi, qw)] * C.N, [doc(C, j) for j in range(C.N)], 1.0, 15)
    assert rel_err(got, full) <= 2 * RTOL


@pytest.mark.parametrize("vr_set", [[1, 2, 5, 8], [9, 13, 16], [17, 19, 24], [25, 32, 33, 64, 65, 128],
                                    [129, 300]])
def test_ragged_sizes_span_tiles(paper, vr_set):
    """Query sizes in every cost-tile shape (4 KPT query words per tile), target sizes
    around the 32-word tile and beyond, pairs whose K and K.*M exceed shared memory."""
    E, C, _, corpus = paper
    rng = np.random.default_rng(sum(vr_set))
    queries, targets = [], []
    for vr in vr_set:
        for vx in (1, 3, 31, 32, 33, 100, 300):
            queries.append(random_side(rng, C.V, vr))
            targets.append(random_side(rng, C.V, vx))
    got = swmd.swmd_wmd_pairs(corpus, queries, targets, 1.0, 15)
    ref = oracle.wmd_pairs(E, queries, targets, 1.0, 15)
    assert rel_err(got, ref) <= RTOL


def test_large_lambda_uses_the_column_shift(paper):
    E, C, (qi, qw), corpus = paper
    docs = [doc(C, j) for j in range(0, 600, 7)]
    got = swmd.swmd_wmd_pairs(corpus, [(qi, qw)] * len(docs), docs, 30.0, 15)
    ref = oracle.wmd_pairs(E, [(qi, qw)] * len(docs), docs, 30.0, 15)
    assert rel_err(got, ref) <= RTOL


def test_single_word_sides_are_closed_forms(paper):
    E, C, _, corpus = paper
    a, b, c = 17, 4242, 99_000
    Ed = E.astype(np.float64)
    got = swmd.swmd_wmd_pairs(corpus, [([a], [1.0]), ([a, b], [1.0, 3.0])], [([c], [2.0]), ([c], [1.0])],
                              1.0, 5)
    dac, dbc = np.linalg.norm(Ed[a] - Ed[c]), np.linalg.norm(Ed[b] - Ed[c])
    assert got[0] == pytest.approx(dac, rel=RTOL)
    assert got[1] == pytest.approx(0.25 * dac + 0.75 * dbc, rel=RTOL)


def test_each_pair_is_independent_of_the_batch_and_launch(paper):
    """Bitwise: a pair alone, among others (other tile shapes and shared-memory
    placement chosen from the batch's largest pair), and through the device entry
    point with loose size bounds."""
    torch = pytest.importorskip("torch")
    E, C, (qi, qw), corpus = paper
    rng = np.random.default_rng(5)
    queries = [(qi, qw)] + [random_side(rng, C.V, n) for n in (3, 40, 128)]
    targets = [doc(C, 3)] + [random_side(rng, C.V, n) for n in (7, 200, 60)]
    together = swmd.swmd_wmd_pairs(corpus, queries, targets, 1.0, 15)
    for p in range(len(queries)):
        alone = swmd.swmd_wmd_pairs(corpus, [queries[p]], [targets[p]], 1.0, 15)
        assert alone[0] == together[p]
    # device entry point on selected, normalised sides
    sel_q = [swmd.swmd_select(C.V, *q) for q in queries]
    sel_x = [swmd.swmd_select(C.V, *x) for x in targets]
    qp, qi_, qr = swmd._ragged(sel_q)
    xp, xi_, xc = swmd._ragged(sel_x)
    dev = lambda a: torch.from_numpy(a).cuda()
    out = torch.empty(len(queries), dtype=torch.float64, device="cuda")
    its = torch.empty(len(queries), dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for bounds in ((128, 200), (4096, 4096), (1000, 300)):
        status.zero_()
        swmd.swmd_wmd_pairs_device(corpus, len(queries), dev(qp), dev(qi_), dev(qr), dev(xp), dev(xi_),
                                   dev(xc), bounds[0], bounds[1], 1.0, 15, out, status, d_iters=its)
        torch.cuda.synchronize()
        assert (int(status.item()) & ~4) == 0
        np.testing.assert_array_equal(out.cpu().numpy(), together)
        assert np.all(its.cpu().numpy() == 15)


def test_convergence_mode_matches_the_converged_oracle(paper):
    E, C, (qi, qw), corpus = paper
    docs = [doc(C, j) for j in range(0, 600, 31)]
    got, its = swmd.swmd_wmd_pairs(corpus, [(qi, qw)] * len(docs), docs, 1.0, 2000, tol=1e-6,
                                   want_iters=True)
    ref, ref_its = oracle.wmd_pairs(E, [(qi, qw)] * len(docs), docs, 1.0, 100000, tol=1e-12,
                                    want_iters=True)
    assert np.all(its < 2000) and np.all(its >= 1)
    # each pair's distance is the one of exactly the x-updates it applied (FP32 bound)
    for p, x in enumerate(docs):
        exact = oracle.wmd_pairs(E, [(qi, qw)], [x], 1.0, int(its[p]))
        assert rel_err(got[p:p + 1], exact) <= 1e-5, (p, int(its[p]))
    assert rel_err(got, ref) <= 1e-4
    # the rule stops where the oracle's does at the same tolerance, give or take rounding
    _, o_its = oracle.wmd_pairs(E, [(qi, qw)] * len(docs), docs, 1.0, 100000, tol=1e-6,
                                want_iters=True)
    assert np.all(np.abs(its - o_its) <= np.maximum(2, o_its // 5))
    # converged distances are symmetric in the pair
    back = swmd.swmd_wmd_pairs(corpus, docs, [(qi, qw)] * len(docs), 1.0, 2000, tol=1e-6)
    assert rel_err(back, got) <= 1e-4


def test_zero_pairs_and_invalid_sides(paper):
    E, C, (qi, qw), corpus = paper
    assert swmd.swmd_wmd_pairs(corpus, [], [], 1.0, 15).shape == (0,)
    ok = (qi, qw)
    for bad in (([0, C.V], [1.0, 1.0]), ([1, 2], [1.0, -1.0]), ([1, 2], [0.0, 0.0]), ([], []),
                (np.arange(4097), np.ones(4097))):
        for q, x in ((ok, bad), (bad, ok)):
            with pytest.raises(swmd.SwmdError) as e:
                swmd.swmd_wmd_pairs(corpus, [ok, q], [ok, x], 1.0, 15)
            assert e.value.code == swmd.SWMD_EINVAL
            assert "pair 1" in str(e.value)
    for lam, t, tol in ((0.0, 15, 0.0), (float("inf"), 15, 0.0), (1.0, -1, 0.0), (1.0, 15, -1.0)):
        with pytest.raises(swmd.SwmdError):
            swmd.swmd_wmd_pairs(corpus, [ok], [ok], lam, t, tol=tol)


def test_device_entry_flags_bad_pairs_without_stopping_the_rest(paper):
    torch = pytest.importorskip("torch")
    E, C, (qi, qw), corpus = paper
    ids, r = swmd.swmd_select(C.V, qi, qw)
    x_ids, x_c = swmd.swmd_select(C.V, *doc(C, 0))
    bad_ids = x_ids.copy()
    bad_ids[0] = C.V + 5
    qp, qi_, qr = swmd._ragged([(ids, r)] * 3)
    xp, xi_, xc = swmd._ragged([(x_ids, x_c), (bad_ids, x_c), (x_ids, x_c)])
    dev = lambda a: torch.from_numpy(a).cuda()
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    swmd.swmd_wmd_pairs_device(corpus, 3, dev(qp), dev(qi_), dev(qr), dev(xp), dev(xi_), dev(xc),
                               len(ids), len(x_ids), 1.0, 15, out, status)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert int(status.item()) & 1            # an id outside [0, V)
    assert np.isnan(o[1]) and np.isfinite(o[0]) and o[0] == o[2]
    # a side above its declared bound
    status.zero_()
    swmd.swmd_wmd_pairs_device(corpus, 3, dev(qp), dev(qi_), dev(qr), dev(xp), dev(xi_), dev(xc),
                               len(ids) - 1, len(x_ids), 1.0, 15, out, status)
    torch.cuda.synchronize()
    assert int(status.item()) & 16
    assert np.all(np.isnan(out.cpu().numpy()))


def test_full_size_paper_workload_sampled(paper):
    """The benchmark's launch: the paper-shaped query against all 5,000 documents of
    the paper workload, sampled outputs checked against the oracle."""
    E, C, (qi, qw) = synth.make("paper")
    corpus = swmd.corpus_from_synth(E, C)
    try:
        docs = [doc(C, j) for j in range(C.N)]
        got = swmd.swmd_wmd_pairs(corpus, [(qi, qw)] * C.N, docs, 1.0, 15)
        pick = np.random.default_rng(7).choice(C.N, 64, replace=False)
        ref = oracle.wmd_pairs(E, [(qi, qw)] * len(pick), [docs[j] for j in pick], 1.0, 15)
        assert rel_err(got[pick], ref) <= RTOL
        assert np.all(np.isfinite(got))
    finally:
        corpus.close()
