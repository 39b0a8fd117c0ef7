"""swmd_query_noalloc: the query for callers that cannot allocate device memory
when they query (a server whose pool owns the free memory, a latency-critical
path that must not synchronise on cudaMalloc / cudaFree).  Its scratch lives in a
fixed device array inside the library.  Checked through the C ABI against
swmd_query_device on two calls in a row, within the suite's 1e-5 tolerance, and
for the refusal of a query whose scratch exceeds the array.

This file is collected last so that a run stopping at the first failure has run
every other test before it; it also passes alone in a fresh process."""
import numpy as np
import pytest

import paper_2107_06433_gb300 as swmd
from paper_2107_06433_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2107_06433_gb300 import build
    build.build()
    E, C, (qi, qw) = synth.make("paper")
    corpus = swmd.corpus_from_synth(E, C)
    return torch, E, C, corpus


def _device_query(torch, C, qi, qw):
    ids, r = swmd.swmd_select(C.V, qi, qw)
    return torch.from_numpy(ids).cuda(), torch.from_numpy(r).cuda(), len(ids)


def test_noalloc_matches_device_entry_point_twice(setup):
    torch, E, C, corpus = setup
    queries = [synth.make("paper")[2], synth.query(np.random.default_rng(77), C.V, 31)]
    lams = [1.0, 3.0]
    for (qi, qw), lam in zip(queries, lams):          # two calls in a row
        d_ids, d_r, vr = _device_query(torch, C, qi, qw)
        ref = torch.empty(C.N, dtype=torch.float64, device="cuda")
        got = torch.full((C.N,), float("nan"), dtype=torch.float64, device="cuda")
        st_ref = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        swmd.swmd_query_device(corpus, d_ids, d_r, vr, lam, 15, ref, st_ref)
        swmd.swmd_query_noalloc(corpus, d_ids, d_r, vr, lam, 15, got, st)
        torch.cuda.synchronize()
        a, b = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(b))
        assert float(np.max(np.abs(b - a) / np.abs(a))) <= RTOL
        assert int(st.item()) == 0 and int(st_ref.item()) == 0


def test_noalloc_refuses_a_query_larger_than_its_array(setup):
    torch, E, C, corpus = setup
    qi, qw = synth.query(np.random.default_rng(5), C.V, 128)   # 2 x V_used x 128 x 4 B > 16 MiB
    d_ids, d_r, vr = _device_query(torch, C, qi, qw)
    out = torch.empty(C.N, dtype=torch.float64, device="cuda")
    with pytest.raises(swmd.SwmdError) as e:
        swmd.swmd_query_noalloc(corpus, d_ids, d_r, vr, 1.0, 15, out)
    assert e.value.code == swmd.SWMD_EINVAL and "scratch" in str(e.value)


def test_noalloc_allocates_nothing(setup):
    """The property the entry point exists for: after a first call on the device,
    further calls leave the device's free memory and PyTorch's allocator counters
    exactly where they were."""
    torch, E, C, corpus = setup
    qi, qw = synth.query(np.random.default_rng(3), C.V, 19)
    d_ids, d_r, vr = _device_query(torch, C, qi, qw)
    out = torch.empty(C.N, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    swmd.swmd_query_noalloc(corpus, d_ids, d_r, vr, 1.0, 15, out, st)   # first call on the device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for lam in (0.5, 1.0, 2.0, 4.0, 8.0):
        swmd.swmd_query_noalloc(corpus, d_ids, d_r, vr, lam, 15, out, st)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
    assert int(st.item()) == 0 and np.all(np.isfinite(out.cpu().numpy()))
