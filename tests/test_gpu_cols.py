"""The column-split register solver against the FP64 oracle, through the C ABI.

The solver keeps each document's K^T rows in registers for all t iterations, split
by columns over a team of VRP / 8 lanes, 4 for 128 columns (resident_cols.cu).  Query
layouts of 16, 32, 64 and 128 columns; buckets of 8, 16, 24 and 32 rows in every
layout, and of 48, 64 and 96 rows (four and eight row groups) at 16 and 32 columns.
Documents longer than a layout's largest bucket run on the register solver in a
launch before the column-split one (16 and 32 columns), else the query falls back
to the other resident solvers.  These tests cover every bucket and team size, ragged
buckets (every document length 1..32, and 1..300 for the long buckets), the
iteration counts 0, 1 and 15, lambda 1 and 10, and the invariances the other solvers
have (document ranges, batches and the server give the same bits).  Tolerance: 1e-5
relative on every distance (FP32), the stated bounds for BF16 / FP16 K.
"""
import numpy as np
import pytest

import oracle
import paper_2107_06433_gb300 as swmd
from paper_2107_06433_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5
BOUND = {"fp32": 1e-5, "bf16": 1e-2, "fp16": 2e-3}
SOLVER_COLS = 4


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
def short_docs():
    """300 documents: every length 1..32 five times, the rest uniform in 1..32 (so
    warps of one bucket hold documents of different lengths)."""
    rng = np.random.default_rng(31)
    V, d = 3000, 48
    E = synth.embeddings(rng, V, d)
    lens = np.concatenate([np.repeat(np.arange(1, 33), 5), rng.integers(1, 33, size=140)])
    rng.shuffle(lens)
    C = synth.corpus(rng, V, len(lens), lens, 10)
    return E, C


def oracle_wmd(E, C, qi, qw, lam, t):
    rp, col, val = C.csr()
    return oracle.wmd(E, rp, col, val, C.N, qi, qw, lam, t)


@pytest.mark.parametrize("vr", [1, 4, 15, 16, 17, 31, 32, 33, 63, 64, 65, 100, 128])
@pytest.mark.parametrize("t", [0, 1, 15])
def test_every_width_and_bucket(short_docs, vr, t):
    E, C = short_docs
    qi, qw = synth.query(np.random.default_rng(100 + vr), C.V, vr)
    corpus = swmd.corpus_from_synth(E, C, path="resident", solver=SOLVER_COLS)
    for lam in (1.0, 10.0):
        got = swmd.swmd_query(corpus, qi, qw, lam, t)
        assert rel_err(got, oracle_wmd(E, C, qi, qw, lam, t)) <= RTOL, (vr, t, lam)


def test_layout_is_a_power_of_two_of_16_or_more(short_docs):
    E, C = short_docs
    corpus = swmd.corpus_from_synth(E, C, path="resident", solver=SOLVER_COLS)
    for vr, vrp in ((1, 16), (16, 16), (17, 32), (32, 32), (33, 64), (100, 128)):
        assert swmd.swmd_get_mapping(corpus, vr, "resident")[0] == vrp


@pytest.mark.parametrize("kprec", ["bf16", "fp16"])
@pytest.mark.parametrize("lam", [1.0, 10.0])
def test_reduced_precision_bounds(short_docs, kprec, lam):
    E, C = short_docs
    corpus = swmd.corpus_from_synth(E, C, path="resident", solver=SOLVER_COLS, k_precision=kprec)
    for vr in (8, 32, 64):
        qi, qw = synth.query(np.random.default_rng(vr), C.V, vr)
        err = rel_err(swmd.swmd_query(corpus, qi, qw, lam, 15), oracle_wmd(E, C, qi, qw, lam, 15))
        assert err <= BOUND[kprec], (kprec, lam, vr, err)


def test_agrees_with_the_row_register_solver(short_docs):
    """The column-split and the row-per-lane register solvers compute the same
    iteration in different orders: equal within the FP32 tolerance."""
    E, C = short_docs
    qi, qw = synth.query(np.random.default_rng(5), C.V, 24)
    a = swmd.swmd_query(swmd.corpus_from_synth(E, C, path="resident", solver=SOLVER_COLS), qi, qw, 1.0, 15)
    b = swmd.swmd_query(swmd.corpus_from_synth(E, C, path="resident", solver=1), qi, qw, 1.0, 15)
    assert rel_err(a, b) <= RTOL


def test_document_ranges_give_the_same_bits(short_docs):
    E, C = short_docs
    rp, col, val = C.csr()
    qi, qw = synth.query(np.random.default_rng(7), C.V, 40)
    whole = swmd.swmd_query(swmd.swmd_create_corpus(C.V, C.N, rp, col, val, E), qi, qw, 1.0, 15)
    cut = [0, 77, 150, C.N]
    parts = [swmd.swmd_query(swmd.swmd_create_corpus(C.V, C.N, rp, col, val, E, doc_begin=a, doc_end=b),
                             qi, qw, 1.0, 15) for a, b in zip(cut[:-1], cut[1:])]
    np.testing.assert_array_equal(np.concatenate(parts), whole)


def test_default_solver_on_short_documents(short_docs):
    """On a corpus of documents up to 32 words the automatic resident solver is the
    column-split one: same bits as asking for it."""
    E, C = short_docs
    qi, qw = synth.query(np.random.default_rng(8), C.V, 19)
    a = swmd.swmd_query(swmd.corpus_from_synth(E, C, path="resident"), qi, qw, 1.0, 15)
    b = swmd.swmd_query(swmd.corpus_from_synth(E, C, path="resident", solver=SOLVER_COLS), qi, qw, 1.0, 15)
    np.testing.assert_array_equal(a, b)


def test_falls_back_on_long_documents():
    """Asking for the column-split solver on a corpus with documents above 32 words
    runs, at 64 columns (buckets up to 32 rows), the other resident solvers in their
    own layout (still within the tolerance)."""
    rng = np.random.default_rng(12)
    V = 2000
    E = synth.embeddings(rng, V, 32)
    C = synth.corpus(rng, V, 80, rng.integers(1, 60, size=80), 5)
    qi, qw = synth.query(rng, V, 40)
    corpus = swmd.corpus_from_synth(E, C, path="resident", solver=SOLVER_COLS)
    assert swmd.swmd_get_mapping(corpus, 40, "resident")[0] == 40   # the tight layout
    assert rel_err(swmd.swmd_query(corpus, qi, qw, 1.0, 15), oracle_wmd(E, C, qi, qw, 1.0, 15)) <= RTOL


@pytest.fixture(scope="module")
def long_docs():
    """250 documents: lengths spread over 1..300 (every bucket from 8 to 96 rows,
    and 60 documents above 96 words for the register solver), shuffled."""
    rng = np.random.default_rng(33)
    V, d = 6000, 48
    E = synth.embeddings(rng, V, d)
    lens = np.concatenate([rng.integers(1, 33, size=60), rng.integers(33, 49, size=40),
                           rng.integers(49, 65, size=40), rng.integers(65, 97, size=50),
                           rng.integers(97, 301, size=60)])
    rng.shuffle(lens)
    C = synth.corpus(rng, V, len(lens), lens, 10)
    return E, C


@pytest.mark.parametrize("vr", [1, 8, 16, 19, 32])
@pytest.mark.parametrize("t", [0, 1, 15])
def test_long_buckets_and_register_prefix(long_docs, vr, t):
    """Documents of 33-96 words in the buckets of 48, 64 and 96 rows, longer ones on
    the register solver in the same query: every distance against the oracle."""
    E, C = long_docs
    qi, qw = synth.query(np.random.default_rng(200 + vr), C.V, vr)
    corpus = swmd.corpus_from_synth(E, C, path="resident", solver=SOLVER_COLS)
    assert swmd.swmd_get_mapping(corpus, vr, "resident")[0] == (16 if vr <= 16 else 32)
    for lam in (1.0, 10.0):
        got = swmd.swmd_query(corpus, qi, qw, lam, t)
        assert rel_err(got, oracle_wmd(E, C, qi, qw, lam, t)) <= RTOL, (vr, t, lam)


@pytest.mark.parametrize("kprec", ["bf16", "fp16"])
def test_long_buckets_reduced_precision(long_docs, kprec):
    E, C = long_docs
    corpus = swmd.corpus_from_synth(E, C, path="resident", solver=SOLVER_COLS, k_precision=kprec)
    for vr in (12, 30):
        qi, qw = synth.query(np.random.default_rng(vr), C.V, vr)
        for lam in (1.0, 10.0):
            err = rel_err(swmd.swmd_query(corpus, qi, qw, lam, 15), oracle_wmd(E, C, qi, qw, lam, 15))
            assert err <= BOUND[kprec], (kprec, vr, lam, err)


def test_long_buckets_invariances(long_docs):
    """The mixed launch gives the same bits in any document range, batched and
    served; and agrees with the register solver alone within the tolerance."""
    E, C = long_docs
    rp, col, val = C.csr()
    qi, qw = synth.query(np.random.default_rng(77), C.V, 24)
    whole = swmd.swmd_query(swmd.swmd_create_corpus(C.V, C.N, rp, col, val, E, path="resident",
                                                    solver=SOLVER_COLS), qi, qw, 1.0, 15)
    cut = [0, 61, 170, C.N]
    parts = [swmd.swmd_query(swmd.swmd_create_corpus(C.V, C.N, rp, col, val, E, path="resident",
                                                     solver=SOLVER_COLS, doc_begin=a, doc_end=b),
                             qi, qw, 1.0, 15) for a, b in zip(cut[:-1], cut[1:])]
    np.testing.assert_array_equal(np.concatenate(parts), whole)
    regs = swmd.swmd_query(swmd.corpus_from_synth(E, C, path="resident", solver=1), qi, qw, 1.0, 15)
    assert rel_err(whole, regs) <= RTOL
    corpus = swmd.corpus_from_synth(E, C, path="resident", solver=SOLVER_COLS)
    qs = synth.batch_queries(C.V, 9, 1, 32, seed=81)
    alone = [swmd.swmd_query(corpus, q, w, 1.0, 15) for q, w in qs]
    batch = swmd.swmd_query_batch(corpus, qs, 1.0, 15)
    for i in range(len(qs)):
        np.testing.assert_array_equal(batch[i], alone[i])
    srv = swmd.swmd_serve_start(corpus, max_batch=4, memory_budget=1 << 28)
    tickets = [swmd.swmd_serve_submit(srv, q, w, 1.0, 15) for q, w in qs]
    for tk, ref in zip(tickets, alone):
        np.testing.assert_array_equal(swmd.swmd_serve_wait(srv, tk, 60000), ref)
    srv.stop()


def test_batch_and_server_equal_alone_bitwise(short_docs):
    E, C = short_docs
    corpus = swmd.corpus_from_synth(E, C, path="resident")
    qs = synth.batch_queries(C.V, 20, 1, 128, seed=41)
    alone = [swmd.swmd_query(corpus, qi, qw, 1.0, 15) for qi, qw in qs]
    batch = swmd.swmd_query_batch(corpus, qs, 1.0, 15)
    for i in range(len(qs)):
        np.testing.assert_array_equal(batch[i], alone[i])
    srv = swmd.swmd_serve_start(corpus, max_batch=6, memory_budget=1 << 28)
    tickets = [swmd.swmd_serve_submit(srv, qi, qw, 1.0, 15) for qi, qw in qs]
    for tk, ref in zip(tickets, alone):
        np.testing.assert_array_equal(swmd.swmd_serve_wait(srv, tk, 60000), ref)
    srv.stop()


def test_large_workload_sampled():
    """The 1,000,000-document workload (17.5M nonzeros, v_r = 32) on the resident
    path at full size: 200 sampled documents against the oracle's pair form (the
    cost over each document's words only, pinned equal to the 1-to-N column)."""
    E, C, (qi, qw) = synth.make("large")
    corpus = swmd.corpus_from_synth(E, C, path="resident")
    got = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
    sel = np.sort(np.random.default_rng(6).choice(C.N, 200, replace=False))
    docs = [(C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]], C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]]) for j in sel]
    ref = oracle.wmd_pairs(E, [(qi, qw)] * len(sel), docs, 1.0, 15)
    assert rel_err(got[sel], ref) <= RTOL
    assert np.all(np.isfinite(got)) and np.all(got > 0)


@pytest.mark.parametrize("qpt", [1, 3, 8])
def test_multi_query_launch_equals_alone_bitwise(short_docs, qpt):
    """swmd_query_batch runs the column-split queries of a layout in groups of qpt,
    one cost and one multi-query solver launch per group, the solver over (query,
    document task) tiles; every group size gives the single queries' bits."""
    E, C = short_docs
    corpus = swmd.corpus_from_synth(E, C, path="resident", queries_per_tile=qpt)
    qs = synth.batch_queries(C.V, 17, 1, 128, seed=60 + qpt)
    lams = np.linspace(0.5, 3.0, len(qs)).astype(np.float32)
    batch = swmd.swmd_query_batch(corpus, qs, lams, 15)
    for i, (qi, qw) in enumerate(qs):
        np.testing.assert_array_equal(batch[i], swmd.swmd_query(corpus, qi, qw, float(lams[i]), 15))
    i = 5
    assert rel_err(batch[i], oracle_wmd(E, C, qs[i][0], qs[i][1], float(lams[i]), 15)) <= RTOL


def test_batch_autotuner_picks_a_tile_size(short_docs):
    E, C = short_docs
    corpus = swmd.corpus_from_synth(E, C, path="resident")
    qs = synth.batch_queries(C.V, 12, 4, 40, seed=71)
    res = swmd.swmd_autotune_batch(corpus, qs, 1.0, 15, reps=1)
    assert res["layouts"] >= 1 and res["candidates"] >= 1 + 4 * res["layouts"]
    assert all(q in (1, 2, 4, 8) for q in res["queries_per_tile"])
    assert res["best_ms"] <= res["default_ms"] * 1.0001
    batch = swmd.swmd_query_batch(corpus, qs, 1.0, 15)
    for i in (0, 6, 11):
        np.testing.assert_array_equal(batch[i], swmd.swmd_query(corpus, qs[i][0], qs[i][1], 1.0, 15))


def test_large_workload_batch_and_server_equal_alone():
    """Six queries of 4..128 words on the 1,000,000-document workload: one batch call
    (one multi-query launch per layout) and the server (grouped launches) give each
    query's single-query bits."""
    E, C, _ = synth.make("large")
    corpus = swmd.corpus_from_synth(E, C, k_precision="bf16")
    qs = synth.batch_queries(C.V, 6, 4, 128, seed=91)
    alone = [swmd.swmd_query(corpus, qi, qw, 1.0, 15) for qi, qw in qs]
    batch = swmd.swmd_query_batch(corpus, qs, 1.0, 15)
    for i in range(len(qs)):
        np.testing.assert_array_equal(batch[i], alone[i])
    srv = swmd.swmd_serve_start(corpus, max_batch=8, memory_budget=8 << 30)
    tickets = [swmd.swmd_serve_submit(srv, qi, qw, 1.0, 15) for qi, qw in qs]
    for tk, ref in zip(tickets, alone):
        np.testing.assert_array_equal(swmd.swmd_serve_wait(srv, tk, 120000), ref)
    st = swmd.swmd_serve_stats(srv)
    srv.stop()
    assert st["completed"] == len(qs)
