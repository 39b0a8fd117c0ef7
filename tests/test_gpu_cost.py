"""The cost step (a1: M = cdist(E[q], E), K = exp(-lambda M), K.*M; Algorithm 1 and
Table I) against the FP64 oracle's distances, through the C ABI, where the two
ways the library evaluates M differ most.

Layouts of 16 and 32 columns (and the 32-column chunks of 64 and 128) compute M^2
as |q|^2 + |e|^2 - 2 q.e, which cancels when a corpus word lies close to a query
word; those entries are evaluated again in the direct difference form.  The
corpus here puts words at every distance from the query words, from exact copies
(M = 0) through the switch-over (M^2 = (|q|^2 + |e|^2) / 4) to unrelated words,
with embedding norms from 0.5 to 2.  cost_split = 1 asks for the difference-form
row kernel instead; both must agree with the oracle.

The distances are read back as KM^T / K^T (both stored in FP32, each rounded once,
so the ratio is M to a few ulps).  Tolerance on M: 5e-6 relative.  FP32 rounding of
a 300-term dot of near-parallel rows, and of the two norms, is a few 1e-7 of
|q|^2 near the switch-over, where M^2 is half of |q|^2; a product form without the
fallback is wrong by 1e-2 and more on the close pairs.  Exact copies must give
M = 0 exactly.  The whole query must match the oracle to the FP32 path's 1e-5.
"""
import numpy as np
import pytest

import oracle
import paper_2107_06433_gb300 as swmd

pytestmark = pytest.mark.gpu
RTOL_M = 5e-6
RTOL = 1e-5
V, D, VR, DOC_LEN = 4096, 300, 32, 10
# distances of the planted words from their query word, as a fraction of its norm
OFFSETS = (0.0, 1e-5, 1e-3, 0.05, 0.3, 0.6, 0.72, 1.0)


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
def planted():
    """Embeddings of mixed norms, a 32-word query, and for each query word eight
    corpus words at the distances OFFSETS x its norm; documents of 10 consecutive
    word ids, so that every word is used."""
    rng = np.random.default_rng(2107064)
    E = rng.standard_normal((V, D))
    E /= np.linalg.norm(E, axis=1, keepdims=True)
    E *= rng.uniform(0.5, 2.0, size=(V, 1))
    qi = rng.choice(np.arange(0, 2048), size=VR, replace=False).astype(np.int32)
    for k, q in enumerate(qi):
        for j, off in enumerate(OFFSETS):
            w = 2048 + len(OFFSETS) * k + j
            u = rng.standard_normal(D)
            u -= (u @ E[q]) / (E[q] @ E[q]) * E[q]      # orthogonal to the query row
            E[w] = E[q] + off * np.linalg.norm(E[q]) * u / np.linalg.norm(u)
    E = E.astype(np.float32)
    for k, q in enumerate(qi):                           # exact copies after the FP32 rounding
        E[2048 + len(OFFSETS) * k] = E[q]
    N = (V + DOC_LEN - 1) // DOC_LEN
    doc_of_word = np.arange(V) // DOC_LEN
    counts = rng.integers(1, 6, size=V).astype(np.float64)
    tot = np.bincount(doc_of_word, weights=counts, minlength=N)
    row_ptr = np.arange(V + 1, dtype=np.int64)           # word w: one nonzero, in its document
    doc_idx = doc_of_word.astype(np.int32)
    val = (counts / tot[doc_of_word]).astype(np.float32)
    qw = rng.integers(1, 4, size=VR).astype(np.float32)
    return E, N, row_ptr, doc_idx, val, qi, qw


def _distances(corpus, E, qi):
    import torch
    ids, _ = swmd.swmd_select(V, qi, np.ones(len(qi), np.float32))
    swmd.swmd_step_cost(corpus, torch.from_numpy(ids).cuda(), None, len(ids), 1.0)
    torch.cuda.synchronize()
    used = swmd.swmd_debug_read(corpus, "used")
    KT = swmd.swmd_debug_read(corpus, "KT", len(ids)).astype(np.float64)
    KMT = swmd.swmd_debug_read(corpus, "KMT", len(ids)).astype(np.float64)
    assert np.all(KT > 0)
    return (KMT / KT).T, oracle.cdist(E, ids)[:, used]


@pytest.mark.parametrize("split", [0, 1])
def test_distances_at_every_range(planted, split):
    E, N, row_ptr, doc_idx, val, qi, _ = planted
    corpus = swmd.swmd_create_corpus(V, N, row_ptr, doc_idx, val, E, cost_split=split)
    got, ref = _distances(corpus, E, qi)
    zero = ref == 0.0
    assert zero.sum() >= VR                               # the planted copies at least
    assert np.all(got[zero] == 0.0)
    assert rel_err(got[~zero], ref[~zero]) <= RTOL_M


def test_product_and_difference_forms_agree(planted):
    E, N, row_ptr, doc_idx, val, qi, _ = planted
    a, _ = _distances(swmd.swmd_create_corpus(V, N, row_ptr, doc_idx, val, E, cost_split=0), E, qi)
    b, ref = _distances(swmd.swmd_create_corpus(V, N, row_ptr, doc_idx, val, E, cost_split=1), E, qi)
    nz = ref > 0.0
    assert rel_err(a[nz], b[nz]) <= 2 * RTOL_M


@pytest.mark.parametrize("vr", [16, 32, 64, 128])
@pytest.mark.parametrize("path", ["resident", "fused"])
def test_query_over_planted_words(planted, vr, path):
    """Whole queries whose words have close neighbours in the corpus, every
    product-form layout (64 and 128 in 32-column chunks)."""
    E, N, row_ptr, doc_idx, val, qi, qw = planted
    rng = np.random.default_rng(vr)
    ids = np.concatenate([qi, rng.choice(np.arange(3000, V), size=max(0, vr - VR), replace=False)])[:vr]
    w = np.concatenate([qw, rng.integers(1, 4, size=max(0, vr - VR))])[:vr].astype(np.float32)
    corpus = swmd.swmd_create_corpus(V, N, row_ptr, doc_idx, val, E, path=path)
    got = swmd.swmd_query(corpus, ids.astype(np.int32), w, 1.0, 15)
    ref = oracle.wmd(E, row_ptr, doc_idx, val, N, ids.astype(np.int32), w, 1.0, 15)
    assert rel_err(got, ref) <= RTOL
