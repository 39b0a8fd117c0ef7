"""The device-allocator hook: with swmd_set_allocator wired to PyTorch's caching
allocator, a corpus, its batch and pair workspaces and a server take their device
memory from it and give all of it back, and the distances are those of a corpus that
used cudaMalloc (bit for bit)."""
import numpy as np
import pytest

import paper_2107_06433_gb300 as swmd
from paper_2107_06433_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2107_06433_gb300 import build
    build.build()
    return torch


def test_corpus_memory_comes_from_the_hook(torch):
    E, C, (qi, qw) = synth.make("tiny")
    plain = swmd.corpus_from_synth(E, C)
    ref = swmd.swmd_query(plain, qi, qw, 1.0, 15)
    qs = synth.batch_queries(C.V, 5, 3, 40, seed=8)
    ref_batch = swmd.swmd_query_batch(plain, qs, 1.0, 15)
    plain.close()

    live, calls = {}, {"alloc": 0, "free": 0}

    def alloc(nbytes, device, stream):
        ptr = torch.cuda.caching_allocator_alloc(nbytes, device, stream)
        live[ptr] = nbytes
        calls["alloc"] += 1
        return ptr

    def release(ptr, nbytes, device, stream):
        assert live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)
        calls["free"] += 1

    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    swmd.swmd_set_allocator(alloc, release)
    try:
        corpus = swmd.corpus_from_synth(E, C)
        assert calls["alloc"] > 0 and torch.cuda.memory_allocated() > before
        np.testing.assert_array_equal(swmd.swmd_query(corpus, qi, qw, 1.0, 15), ref)
        n0 = calls["alloc"]
        np.testing.assert_array_equal(swmd.swmd_query_batch(corpus, qs, 1.0, 15), ref_batch)
        docs = [(C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]], C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]])
                for j in range(4)]
        swmd.swmd_wmd_pairs(corpus, [(qi, qw)] * 4, docs, 1.0, 15)
        assert calls["alloc"] > n0          # the batch and pair workspaces
        srv = swmd.swmd_serve_start(corpus, max_batch=2, memory_budget=1 << 26)
        tk = swmd.swmd_serve_submit(srv, qi, qw, 1.0, 15)
        np.testing.assert_array_equal(swmd.swmd_serve_wait(srv, tk, 60000), ref)
        srv.stop()
        corpus.close()
        torch.cuda.synchronize()
        assert calls["free"] == calls["alloc"] and not live
        assert torch.cuda.memory_allocated() == before
    finally:
        swmd.swmd_set_allocator(None, None)


def test_torch_allocator_helper(torch):
    E, C, (qi, qw) = synth.make("tiny")
    ref = swmd.swmd_query(swmd.corpus_from_synth(E, C), qi, qw, 1.0, 15)
    before = torch.cuda.memory_allocated()
    swmd.use_torch_allocator()
    try:
        corpus = swmd.corpus_from_synth(E, C)
        assert torch.cuda.memory_allocated() > before
        np.testing.assert_array_equal(swmd.swmd_query(corpus, qi, qw, 1.0, 15), ref)
        corpus.close()
        assert torch.cuda.memory_allocated() == before
    finally:
        swmd.swmd_set_allocator(None, None)


def test_failing_allocator_refuses_the_corpus(torch):
    E, C, _ = synth.make("tiny")
    swmd.swmd_set_allocator(lambda n, d, s: 0, lambda p, n, d, s: None)
    try:
        with pytest.raises(swmd.SwmdError) as e:
            swmd.corpus_from_synth(E, C)
        assert e.value.code == swmd.SWMD_ENOMEM
    finally:
        swmd.swmd_set_allocator(None, None)
