"""Parity at the full sizes of the batched and served workloads, on sampled outputs.

The oracle's reference for a sampled document is its 1-to-1 pair distance (cost over
that document's words only), which equals the document's entry of the 1-to-N result
(pinned in test_oracle_pins.py), so the oracle's cost stays small at full size.
Bounds: FP32 1e-5, BF16 K 1e-2 (the stated per-distance bounds).
"""
import numpy as np
import pytest

import oracle
import paper_2107_06433_gb300 as swmd
from paper_2107_06433_gb300 import synth

pytestmark = pytest.mark.gpu
BOUND = {"fp32": 1e-5, "bf16": 1e-2}


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


def sampled_refs(E, C, queries, sel, lam, t):
    docs = [(C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]], C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]])
            for j in sel]
    return [oracle.wmd_pairs(E, [q] * len(docs), docs, lam, t) for q in queries]


def test_batched_workload_sampled():
    """100,000 documents of 10-200 words: 16 queries with v_r spanning 4..64 in one
    swmd_query_batch call, FP32 and BF16 K, against the oracle on 60 sampled documents;
    the batch equals the single queries bit for bit."""
    E, C, _ = synth.make("batch")
    qs = synth.batch_queries(C.V, 16, 4, 64, seed=synth.SEED + 11)
    sel = np.sort(np.random.default_rng(4).choice(C.N, 60, replace=False))
    refs = sampled_refs(E, C, qs, sel, 1.0, 15)
    for kp in ("fp32", "bf16"):
        corpus = swmd.corpus_from_synth(E, C, k_precision=kp)
        batch = swmd.swmd_query_batch(corpus, qs, 1.0, 15)
        errs = [rel_err(batch[i][sel], refs[i]) for i in range(len(qs))]
        print(f"batch workload {kp}: max relative error {max(errs):.3e}")
        assert max(errs) <= BOUND[kp]
        for i in (0, 7, 15):
            np.testing.assert_array_equal(batch[i], swmd.swmd_query(corpus, qs[i][0], qs[i][1], 1.0, 15))
        corpus.close()


def test_served_workload_sampled():
    """1,000,000 documents: 8 queries with v_r spanning 4..128 served with BF16 K
    (continuous batching), against the oracle on 40 sampled documents; each served
    result equals the same query alone, bit for bit."""
    E, C, _ = synth.make("large")
    qs = synth.batch_queries(C.V, 8, 4, 128, seed=synth.SEED + 12)
    sel = np.sort(np.random.default_rng(5).choice(C.N, 40, replace=False))
    refs = sampled_refs(E, C, qs, sel, 1.0, 15)
    corpus = swmd.corpus_from_synth(E, C, k_precision="bf16")
    srv = swmd.swmd_serve_start(corpus, max_batch=4, memory_budget=8 << 30)
    tickets = [swmd.swmd_serve_submit(srv, qi, qw, 1.0, 15) for qi, qw in qs]
    served = [swmd.swmd_serve_wait(srv, tk, 120000) for tk in tickets]
    srv.stop()
    errs = [rel_err(served[i][sel], refs[i]) for i in range(len(qs))]
    print(f"served large workload bf16: max relative error {max(errs):.3e}")
    assert max(errs) <= BOUND["bf16"]
    for i in (0, 5):
        np.testing.assert_array_equal(served[i], swmd.swmd_query(corpus, qs[i][0], qs[i][1], 1.0, 15))
    corpus.close()
