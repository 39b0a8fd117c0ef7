"""Reduced-precision K storage and the FP64 guard, against the FP64 oracle.

K^T and KM^T stored in BF16 or FP16 (FP32 accumulation, FP64 final sum).  Stated
bounds on the relative error of every distance: FP32 1e-5, BF16 1e-2, FP16 2e-3,
for lambda in {1, 10} (the CUDA path's column shift keeps every column's largest
K at 1, so FP16's narrow range does not underflow the useful entries).
"""
import numpy as np
import pytest

import oracle
import paper_2107_06433_gb300 as swmd
from paper_2107_06433_gb300 import synth

pytestmark = pytest.mark.gpu
BOUND = {"fp32": 1e-5, "bf16": 1e-2, "fp16": 2e-3}


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
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


@pytest.fixture(scope="module")
def paper():
    E, C, (qi, qw) = synth.make("paper")
    rp, col, val = C.csr()
    refs = {lam: oracle.wmd(E, rp, col, val, C.N, qi, qw, lam, 15) for lam in (1.0, 10.0)}
    return E, C, qi, qw, refs


@pytest.mark.parametrize("kprec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("path", ["resident", "fused", "plain"])
@pytest.mark.parametrize("lam", [1.0, 10.0])
def test_stated_bounds_paper_shaped(paper, kprec, path, lam):
    E, C, qi, qw, refs = paper
    corpus = swmd.corpus_from_synth(E, C, path=path, k_precision=kprec)
    got = swmd.swmd_query(corpus, qi, qw, lam, 15)
    err = rel_err(got, refs[lam])
    print(f"{kprec} {path} lambda={lam}: max relative error {err:.3e}")
    assert err <= BOUND[kprec]


@pytest.fixture(scope="module")
def tiny():
    E, C, (qi, qw) = synth.make("tiny")
    rp, col, val = C.csr()
    refs = {lam: oracle.wmd(E, rp, col, val, C.N, qi, qw, lam, 15) for lam in (1.0, 10.0)}
    return E, C, qi, qw, refs


@pytest.mark.parametrize("kprec", ["bf16", "fp16"])
@pytest.mark.parametrize("path", ["resident", "fused", "plain"])
@pytest.mark.parametrize("lam", [1.0, 10.0])
def test_stated_bounds_tiny(tiny, kprec, path, lam):
    """The 200-document workload (V = 2,000, d = 64, v_r = 8): the BF16 and FP16
    bounds hold there too, on every path."""
    E, C, qi, qw, refs = tiny
    corpus = swmd.corpus_from_synth(E, C, path=path, k_precision=kprec)
    err = rel_err(swmd.swmd_query(corpus, qi, qw, lam, 15), refs[lam])
    print(f"tiny {kprec} {path} lambda={lam}: max relative error {err:.3e}")
    assert err <= BOUND[kprec]


def test_error_table_large_corpus_sampled():
    """1M documents (17.5M nonzeros), v_r = 32: every precision and lambda against
    the oracle on 200 sampled documents (each document is an independent problem, so
    the oracle runs on the sample alone)."""
    E, C, (qi, qw) = synth.make("large")
    rng = np.random.default_rng(3)
    sel = np.sort(rng.choice(C.N, 200, replace=False))
    lens = np.diff(C.doc_ptr)[sel]
    dp = np.zeros(len(sel) + 1, np.int64)
    np.cumsum(lens, out=dp[1:])
    wids = np.concatenate([C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]] for j in sel])
    vals = np.concatenate([C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]] for j in sel])
    sub = synth.Corpus(C.V, len(sel), dp, wids, np.ones_like(wids), vals)
    rp, col, val = sub.csr()
    table = {}
    for lam in (1.0, 10.0):
        ref = oracle.wmd(E, rp, col, val, sub.N, qi, qw, lam, 15)
        for kprec in ("fp32", "bf16", "fp16"):
            corpus = swmd.corpus_from_synth(E, C, k_precision=kprec)
            got = swmd.swmd_query(corpus, qi, qw, lam, 15)[sel]
            corpus.close()
            table[(kprec, lam)] = rel_err(got, ref)
    for (kprec, lam), err in sorted(table.items()):
        print(f"large corpus {kprec} lambda={lam}: max relative error {err:.3e}")
        assert err <= BOUND[kprec]


@pytest.mark.parametrize("path", ["resident", "fused", "plain"])
def test_fp64_guard_when_kt_u_underflows(path):
    """One query word, column shift off, K = exp(-lambda M) around e^-80: the FP32
    K^T u of the first iteration is below 2^-100, so the guard recomputes it in FP64.
    The distance still equals the closed form sum_w c_wj M[q, w] (one query word),
    and the status word reports the guard."""
    import torch
    rng = np.random.default_rng(21)
    V, N, d = 400, 60, 16
    E = rng.standard_normal((V, d)).astype(np.float32) * 0.02
    E[:, 0] -= 1.0        # every word near -e1 ...
    E[0] = 0.0
    E[0, 0] = 1.0         # ... the query word at +e1: distances near 2
    lens = rng.integers(1, 12, size=N)
    C = synth.corpus(rng, V, N, lens, 5)
    rp, col, val = C.csr()
    corpus = swmd.swmd_create_corpus(V, N, rp, col, val, E, path=path, column_shift=0)
    lam = 40.0
    ids = torch.tensor([0], dtype=torch.int32, device="cuda")
    r = torch.tensor([1.0], dtype=torch.float32, device="cuda")
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    swmd.swmd_query_device(corpus, ids, r, 1, lam, 15, out, st)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    status = int(st.item())
    assert status & 4, f"guard not reported (status {status})"
    assert not status & 2, f"numeric failure reported (status {status})"
    for j in range(N):
        ws = C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]]
        cv = C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]].astype(np.float64)
        cv /= cv.sum()
        m = np.linalg.norm(E[ws].astype(np.float64) - E[0].astype(np.float64), axis=1)
        assert got[j] == pytest.approx(float(cv @ m), rel=1e-5)
