"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Tolerance: the FP32 path must match the oracle to a relative error of 1e-5 on
every distance (the PIUMA FP32-vs-FP64 precedent of Section IV-A is 9.5e-7).
Reduced-precision K storage has its own stated bounds (test_gpu_precision.py).
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


def oracle_wmd(E, C, qi, qw, lam, t):
    rp, col, val = C.csr()
    return oracle.wmd(E, rp, col, val, C.N, qi, qw, lam, t)


@pytest.fixture(scope="module")
def tiny():
    return synth.make("tiny")


@pytest.fixture(scope="module")
def paper():
    return synth.make("paper")


@pytest.mark.parametrize("path", ["resident", "fused", "plain"])
@pytest.mark.parametrize("t", [0, 1, 15])
@pytest.mark.parametrize("lam", [1.0, 10.0])
def test_tiny_all_paths(tiny, path, t, lam):
    E, C, (qi, qw) = tiny
    corpus = swmd.corpus_from_synth(E, C, path=path)
    got = swmd.swmd_query(corpus, qi, qw, lam, t)
    ref = oracle_wmd(E, C, qi, qw, lam, t)
    assert rel_err(got, ref) <= RTOL


@pytest.mark.parametrize("use_graph", [0, 1])
@pytest.mark.parametrize("shift", [0, 1])
def test_tiny_graph_and_shift(tiny, use_graph, shift):
    E, C, (qi, qw) = tiny
    corpus = swmd.corpus_from_synth(E, C, path="fused", use_graph=use_graph, column_shift=shift)
    ref = oracle_wmd(E, C, qi, qw, 1.0, 15)
    for _ in range(3):   # replays of a captured graph give the same answer
        got = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
        assert rel_err(got, ref) <= RTOL


@pytest.mark.parametrize("path", ["resident", "fused", "plain"])
def test_paper_shaped_query(paper, path):
    E, C, (qi, qw) = paper
    corpus = swmd.corpus_from_synth(E, C, path=path)
    got = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
    ref = oracle_wmd(E, C, qi, qw, 1.0, 15)
    assert rel_err(got, ref) <= RTOL


def test_paper_shaped_short_documents():
    E, C, (qi, qw) = synth.make("paper_short")
    corpus = swmd.corpus_from_synth(E, C)
    got = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
    assert rel_err(got, oracle_wmd(E, C, qi, qw, 1.0, 15)) <= RTOL


@pytest.mark.parametrize("tl,lq", [(4, 1), (8, 1), (8, 2), (16, 4), (32, 8)])
def test_every_lane_mapping(tiny, tl, lq):
    E, C, (qi, qw) = tiny
    ref = oracle_wmd(E, C, qi, qw, 1.0, 15)
    for path in ("resident", "fused"):
        corpus = swmd.corpus_from_synth(E, C, path=path, team_lanes=tl, lanes_per_nz=lq)
        assert rel_err(swmd.swmd_query(corpus, qi, qw, 1.0, 15), ref) <= RTOL


@pytest.mark.parametrize("vr", [1, 3, 4, 5, 17, 32, 33, 47, 64, 65, 100, 128])
def test_query_sizes_span_every_padding(vr):
    E, C, _ = synth.make("tiny", N=60)
    rng = np.random.default_rng(vr)
    qi = rng.choice(C.V, size=vr, replace=False).astype(np.int32)
    qw = rng.integers(1, 4, size=vr).astype(np.float32)
    ref = oracle_wmd(E, C, qi, qw, 1.0, 15)
    for path in ("resident", "fused"):
        corpus = swmd.corpus_from_synth(E, C, path=path)
        assert rel_err(swmd.swmd_query(corpus, qi, qw, 1.0, 15), ref) <= RTOL


def test_step_cost_matches_oracle_kernel(tiny):
    """a1 alone: K^T and (K.*M)^T against the oracle's M (column shift off)."""
    import torch
    E, C, (qi, qw) = tiny
    corpus = swmd.corpus_from_synth(E, C, column_shift=0)
    ids, r = swmd.swmd_select(C.V, qi, qw)
    d_ids = torch.from_numpy(ids).cuda()
    swmd.swmd_step_cost(corpus, d_ids, None, len(ids), 2.0)
    torch.cuda.synchronize()
    used = swmd.swmd_debug_read(corpus, "used")
    KT = swmd.swmd_debug_read(corpus, "KT", len(ids))
    KMT = swmd.swmd_debug_read(corpus, "KMT", len(ids))
    M = oracle.cdist(E, ids)[:, used]
    K, KM = oracle.kernel(M, 2.0)
    np.testing.assert_allclose(KT, K.T, rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(KMT, KM.T, rtol=1e-5, atol=1e-6)


def test_steps_compose_to_the_query(paper):
    import torch
    E, C, (qi, qw) = paper
    corpus = swmd.corpus_from_synth(E, C, path="fused")
    ids, r = swmd.swmd_select(C.V, qi, qw)
    d_ids = torch.from_numpy(ids).cuda()
    d_r = torch.from_numpy(r).cuda()
    out = torch.empty(C.N, dtype=torch.float64, device="cuda")
    swmd.swmd_step_cost(corpus, d_ids, d_r, len(ids), 1.0)
    swmd.swmd_step_iterate(corpus, len(ids), 15, 1, "fused")
    swmd.swmd_step_final(corpus, len(ids), 0, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert rel_err(got, oracle_wmd(E, C, qi, qw, 1.0, 15)) <= RTOL
    # the plain SDDMM + SpMM iteration gives the same u up to rounding
    swmd.swmd_step_cost(corpus, d_ids, d_r, len(ids), 1.0)
    swmd.swmd_step_iterate(corpus, len(ids), 15, 1, "plain")
    swmd.swmd_step_final(corpus, len(ids), 0, out)
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), got) <= 1e-6
    # and the resident step
    swmd.swmd_step_cost(corpus, d_ids, d_r, len(ids), 1.0)
    swmd.swmd_step_resident(corpus, len(ids), 15, out)
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), got) <= 1e-6


def test_device_entry_point_equals_host_entry_point(paper):
    import torch
    E, C, (qi, qw) = paper
    corpus = swmd.corpus_from_synth(E, C)
    host = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
    ids, r = swmd.swmd_select(C.V, qi, qw)
    d_ids = torch.from_numpy(ids).cuda()
    d_r = torch.from_numpy(r).cuda()
    out = torch.empty(C.N, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        swmd.swmd_query_device(corpus, d_ids, d_r, len(ids), 1.0, 15, out, st, stream=s)
    s.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), host)
    assert int(st.item()) == 0


# --------------------------------------------------------------------------- closed forms

def test_single_word_query_closed_form():
    E, C, _ = synth.make("tiny")
    q = 17
    corpus = swmd.corpus_from_synth(E, C)
    for t in (0, 3, 15):
        got = swmd.swmd_query(corpus, [q], [1.0], 1.0, t)
        for j in range(0, C.N, 7):
            ws = C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]]
            cv = C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]].astype(np.float64)
            cv /= cv.sum()
            m = np.linalg.norm(E[ws].astype(np.float64) - E[q].astype(np.float64), axis=1)
            assert got[j] == pytest.approx(float(cv @ m), rel=RTOL)


def test_single_word_documents_closed_form():
    rng = np.random.default_rng(9)
    V, N, d = 300, 50, 16
    E = rng.standard_normal((V, d)).astype(np.float32)
    E /= np.linalg.norm(E, axis=1, keepdims=True)
    words = rng.choice(V, size=N, replace=False)
    order = np.argsort(words, kind="stable")
    row_ptr = np.zeros(V + 1, np.int64)
    np.cumsum(np.bincount(words, minlength=V), out=row_ptr[1:])
    doc_idx = np.arange(N, dtype=np.int32)[order]
    val = np.ones(N, np.float32)
    corpus = swmd.swmd_create_corpus(V, N, row_ptr, doc_idx, val, E)
    qi = np.array([3, 50, 77, 200], np.int32)
    qw = np.array([1, 2, 3, 4], np.float32)
    got = swmd.swmd_query(corpus, qi, qw, 3.0, 15)
    r = qw / qw.sum()
    for j in range(N):
        m = np.linalg.norm(E[qi].astype(np.float64) - E[words[j]].astype(np.float64), axis=1)
        assert got[j] == pytest.approx(float(r @ m), rel=RTOL)


# --------------------------------------------------------------------------- edge cases

def test_empty_corpus_and_zero_documents():
    E = np.eye(8, dtype=np.float32)
    corpus = swmd.swmd_create_corpus(8, 0, np.zeros(9, np.int64), np.zeros(0, np.int32),
                                     np.zeros(0, np.float32), E)
    assert swmd.swmd_query(corpus, [1], [1.0], 1.0, 15).shape == (0,)


def test_ragged_lengths_and_document_range():
    """Documents of every length 1..300 (many warps with mixed lengths), loaded
    whole and as two halves; the halves concatenate to the whole."""
    rng = np.random.default_rng(4)
    V, d = 5000, 32
    E = rng.standard_normal((V, d)).astype(np.float32)
    E /= np.linalg.norm(E, axis=1, keepdims=True)
    lens = np.concatenate([np.arange(1, 301), rng.integers(1, 40, size=200)])
    rng.shuffle(lens)
    C = synth.corpus(rng, V, len(lens), lens, 10)
    rp, col, val = C.csr()
    qi, qw = synth.query(rng, V, 23)
    ref = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, 15)
    whole = swmd.swmd_query(swmd.swmd_create_corpus(V, C.N, rp, col, val, E), qi, qw, 1.0, 15)
    assert rel_err(whole, ref) <= RTOL
    h = C.N // 2
    a = swmd.swmd_query(swmd.swmd_create_corpus(V, C.N, rp, col, val, E, doc_begin=0, doc_end=h),
                        qi, qw, 1.0, 15)
    b = swmd.swmd_query(swmd.swmd_create_corpus(V, C.N, rp, col, val, E, doc_begin=h,
                                                doc_end=C.N), qi, qw, 1.0, 15)
    np.testing.assert_array_equal(np.concatenate([a, b]), whole)


def test_embedding_width_not_multiple_of_four():
    rng = np.random.default_rng(5)
    V, d = 700, 37
    E = rng.standard_normal((V, d)).astype(np.float32)
    C = synth.corpus(rng, V, 90, rng.integers(1, 25, size=90), 5)
    rp, col, val = C.csr()
    qi, qw = synth.query(rng, V, 9)
    ref = oracle.wmd(E, rp, col, val, C.N, qi, qw, 0.5, 15)
    got = swmd.swmd_query(swmd.swmd_create_corpus(V, C.N, rp, col, val, E), qi, qw, 0.5, 15)
    assert rel_err(got, ref) <= RTOL


def test_duplicate_query_words_merge(tiny):
    E, C, (qi, qw) = tiny
    corpus = swmd.corpus_from_synth(E, C)
    a = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
    dup_i = np.concatenate([qi, qi[:3]])
    dup_w = np.concatenate([qw * 0.5, qw[:3] * 0.5])
    dup_w[3:len(qi)] = qw[3:]
    b = swmd.swmd_query(corpus, dup_i, dup_w, 1.0, 15)
    assert rel_err(b, a) <= 1e-6


def test_invalid_queries_rejected(tiny):
    E, C, (qi, qw) = tiny
    corpus = swmd.corpus_from_synth(E, C)
    for ids, w, lam, t in [([C.V], [1.0], 1.0, 15), ([1], [-1.0], 1.0, 15),
                           ([1], [1.0], 0.0, 15), ([1], [1.0], float("nan"), 15),
                           ([1], [1.0], 1.0, -1), (list(range(129)), [1.0] * 129, 1.0, 15)]:
        with pytest.raises(swmd.SwmdError) as e:
            swmd.swmd_query(corpus, ids, w, lam, t)
        assert e.value.code == swmd.SWMD_EINVAL
    # the corpus still works afterwards
    assert rel_err(swmd.swmd_query(corpus, qi, qw, 1.0, 15),
                   oracle_wmd(E, C, qi, qw, 1.0, 15)) <= RTOL


def test_device_path_flags_bad_ids_without_faulting(tiny):
    import torch
    E, C, (qi, qw) = tiny
    corpus = swmd.corpus_from_synth(E, C)
    d_ids = torch.tensor([1, C.V + 5, 3], dtype=torch.int32, device="cuda")
    d_r = torch.tensor([0.2, 0.3, 0.5], dtype=torch.float32, device="cuda")
    out = torch.empty(C.N, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    swmd.swmd_query_device(corpus, d_ids, d_r, 3, 1.0, 15, out, st)
    torch.cuda.synchronize()
    assert int(st.item()) & 1          # bad id bit
    assert rel_err(swmd.swmd_query(corpus, qi, qw, 1.0, 15),
                   oracle_wmd(E, C, qi, qw, 1.0, 15)) <= RTOL


# --------------------------------------------------------------------------- batch / serve

def test_batch_equals_alone_bitwise(paper):
    E, C, _ = paper
    corpus = swmd.corpus_from_synth(E, C)
    qs = synth.batch_queries(C.V, 6, 4, 64)
    lams = np.array([1.0, 2.0, 1.0, 0.5, 1.0, 3.0], np.float32)
    batch = swmd.swmd_query_batch(corpus, qs, lams, 15)
    for i, (qi, qw) in enumerate(qs):
        alone = swmd.swmd_query(corpus, qi, qw, float(lams[i]), 15)
        np.testing.assert_array_equal(batch[i], alone)
    i = 2
    assert rel_err(batch[i], oracle_wmd(E, C, qs[i][0], qs[i][1], float(lams[i]), 15)) <= RTOL


def test_served_results_equal_alone_bitwise(paper):
    E, C, _ = paper
    corpus = swmd.corpus_from_synth(E, C)
    qs = synth.batch_queries(C.V, 24, 4, 128)
    alone = [swmd.swmd_query(corpus, qi, qw, 1.0, 15) for qi, qw in qs]
    srv = swmd.swmd_serve_start(corpus, max_batch=8, memory_budget=1 << 30)
    tickets = [swmd.swmd_serve_submit(srv, qi, qw, 1.0, 15) for qi, qw in qs]
    for tk, ref in zip(tickets, alone):
        np.testing.assert_array_equal(swmd.swmd_serve_wait(srv, tk, 60000), ref)
    st = swmd.swmd_serve_stats(srv)
    assert st["completed"] == len(qs) and st["p99_ms"] >= st["p50_ms"] > 0
    srv.stop()


def test_batch_spanning_every_layout_equals_alone_bitwise(paper):
    """40 queries of 1..128 words (every resident layout, register and shared-memory
    solvers) in one call: each equals its own single query bit for bit."""
    E, C, _ = paper
    corpus = swmd.corpus_from_synth(E, C)
    qs = synth.batch_queries(C.V, 40, 1, 128, seed=77)
    batch = swmd.swmd_query_batch(corpus, qs, 1.0, 15)
    for i, (qi, qw) in enumerate(qs):
        np.testing.assert_array_equal(batch[i], swmd.swmd_query(corpus, qi, qw, 1.0, 15))


def test_one_kernel_with_different_shared_memory_in_turn(paper):
    """Two corpora whose shared-memory resident launches take different dynamic
    shared memory (64-nonzero tiles, then tiles of about 110 KB), queried in turn in
    one process: each launch sets the attribute it needs on its device, and every
    query agrees with the oracle (a launcher that kept the first size would fail the
    larger launch)."""
    E, C, _ = paper
    qi, qw = synth.query(np.random.default_rng(40), C.V, 40)
    ref = oracle_wmd(E, C, qi, qw, 1.0, 15)
    small = swmd.corpus_from_synth(E, C, path="resident", solver=2, tile_nnz=64)
    large = swmd.corpus_from_synth(E, C, path="resident", solver=2)
    for corpus in (small, large, small, large):
        assert rel_err(swmd.swmd_query(corpus, qi, qw, 1.0, 15), ref) <= RTOL


@pytest.mark.parametrize("vr", [5, 19, 32, 64])
def test_autotune_then_query_matches_oracle(paper, vr):
    E, C, _ = paper
    corpus = swmd.corpus_from_synth(E, C)
    res = swmd.swmd_autotune(corpus, vr, 3)
    assert res["candidates"] >= 2 and res["best_ms"] > 0
    assert res["best_ms"] <= res["default_ms"] * 1.0001
    assert res["solver"] in (0, 1, 2, 4) and res["vrp"] >= vr
    qi, qw = synth.query(np.random.default_rng(vr), C.V, vr)
    got = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
    assert rel_err(got, oracle_wmd(E, C, qi, qw, 1.0, 15)) <= RTOL
    # the tuned settings serve batches too, bit for bit
    qs = [(qi, qw), synth.query(np.random.default_rng(vr + 1), C.V, vr)]
    batch = swmd.swmd_query_batch(corpus, qs, 1.0, 15)
    np.testing.assert_array_equal(batch[0], got)


def test_autotune_rejects_per_iteration_paths(paper):
    E, C, _ = paper
    corpus = swmd.corpus_from_synth(E, C, path="fused")
    with pytest.raises(swmd.SwmdError):
        swmd.swmd_autotune(corpus, 8, 1)


@pytest.fixture(scope="module")
def wide():
    """24,000 short documents (5-30 Zipf words): above the automatic path's
    resident-only size, so wide queries take the per-iteration fused path."""
    rng = np.random.default_rng(2024)
    V, N, d = 20000, 24000, 64
    E = synth.embeddings(rng, V, d)
    lens = rng.integers(5, 31, size=N)
    C = synth.corpus(rng, V, N, lens, 10)
    return E, C


def test_automatic_path_by_query_width(wide):
    E, C = wide
    # the row-per-lane register solver: the automatic path then depends on the width
    corpus = swmd.corpus_from_synth(E, C, solver=1)
    assert swmd.swmd_resolve_path(corpus, 8) == "resident"
    assert swmd.swmd_resolve_path(corpus, 64) == "fused"
    qs = [synth.query(np.random.default_rng(k), C.V, vr) for k, vr in enumerate((8, 64, 20, 40))]
    for qi, qw in qs[:2]:
        got = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
        assert rel_err(got, oracle_wmd(E, C, qi, qw, 1.0, 15)) <= RTOL
    # one batch mixing both paths: every query equals itself alone, bit for bit
    batch = swmd.swmd_query_batch(corpus, qs, 1.0, 15)
    for i, (qi, qw) in enumerate(qs):
        np.testing.assert_array_equal(batch[i], swmd.swmd_query(corpus, qi, qw, 1.0, 15))
    # and served alongside each other
    srv = swmd.swmd_serve_start(corpus, max_batch=4, memory_budget=1 << 30)
    tickets = [swmd.swmd_serve_submit(srv, qi, qw, 1.0, 15) for qi, qw in qs]
    for tk, ref in zip(tickets, batch):
        np.testing.assert_array_equal(swmd.swmd_serve_wait(srv, tk, 60000), ref)
    srv.stop()


def test_autotune_records_the_path(wide):
    E, C = wide
    corpus = swmd.corpus_from_synth(E, C, solver=1)
    res = swmd.swmd_autotune(corpus, 48, 2)
    assert res["path"] in (swmd.PATH_RESIDENT, swmd.PATH_FUSED)
    assert swmd.swmd_resolve_path(corpus, 48) == {swmd.PATH_RESIDENT: "resident",
                                                  swmd.PATH_FUSED: "fused"}[res["path"]]
    qi, qw = synth.query(np.random.default_rng(48), C.V, 48)
    got = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
    assert rel_err(got, oracle_wmd(E, C, qi, qw, 1.0, 15)) <= RTOL


def test_batch_graph_replays_new_inputs(paper, wide):
    """A batch shape runs eagerly the first time and as a captured CUDA graph the
    second; the third batch of that shape, with other weights and lambdas than the
    captured one, replays the graph on its own inputs."""
    for E, C in ((paper[0], paper[1]), wide):
        corpus = swmd.corpus_from_synth(E, C)
        qs1 = [synth.query(np.random.default_rng(10 + k), C.V, vr) for k, vr in enumerate((6, 19, 40))]
        qs2 = [(qi, np.random.default_rng(99).uniform(0.5, 2.0, len(qi)).astype(np.float32)) for qi, _ in qs1]
        for qs, lams in ((qs1, [1.0, 2.0, 0.5]), (qs2, [3.0, 1.0, 2.0]), (qs1, [1.0, 2.0, 0.5])):
            batch = swmd.swmd_query_batch(corpus, qs, np.array(lams, np.float32), 15)
            for i, (qi, qw) in enumerate(qs):
                np.testing.assert_array_equal(batch[i], swmd.swmd_query(corpus, qi, qw, lams[i], 15))
        nog = swmd.corpus_from_synth(E, C, use_graph=0)
        batch = swmd.swmd_query_batch(nog, qs2, np.array([3.0, 1.0, 2.0], np.float32), 15)
        for i, (qi, qw) in enumerate(qs2):
            np.testing.assert_array_equal(batch[i], swmd.swmd_query(corpus, qi, qw, [3.0, 1.0, 2.0][i], 15))


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_convergence_mode_stops_where_the_oracle_does(tiny, tol):
    """tol > 0: the fused path stops after the x-update in which the row marginal of P
    came below tol (the oracle checks before that update, so it counts one fewer);
    the distances are those of exactly that many x-updates."""
    E, C, (qi, qw) = tiny
    rp, col, val = C.csr()
    ids, r = oracle.select(C.V, qi, qw)
    K, KM = oracle.kernel(oracle.cdist(E, ids), 1.0)
    c = oracle.normalize_columns(C.V, C.N, rp, col, val)
    _, it, _, _ = oracle.sinkhorn_converge(K, KM, r, C.N, rp, col, c, tol=tol, max_iter=4000)
    corpus = swmd.corpus_from_synth(E, C, tol=tol)
    assert swmd.swmd_resolve_path(corpus, len(ids)) == "fused"
    got = swmd.swmd_query(corpus, qi, qw, 1.0, 4000)
    n = swmd.swmd_last_iterations(corpus)
    assert abs(n - (it + 1)) <= 1, (n, it)
    assert rel_err(got, oracle_wmd(E, C, qi, qw, 1.0, n)) <= RTOL
    # a cap below the convergence point stops at the cap
    swmd.swmd_query(corpus, qi, qw, 1.0, 2)
    assert swmd.swmd_last_iterations(corpus) == 2


def test_convergence_mode_needs_the_fused_path(tiny):
    E, C, (qi, qw) = tiny
    with pytest.raises(swmd.SwmdError):
        swmd.swmd_query(swmd.corpus_from_synth(E, C, path="resident", tol=1e-6), qi, qw, 1.0, 50)
    for path in ("fused", "resident", "plain"):
        corpus = swmd.corpus_from_synth(E, C, path=path)
        swmd.swmd_query(corpus, qi, qw, 1.0, 15)
        assert swmd.swmd_last_iterations(corpus) == 15
