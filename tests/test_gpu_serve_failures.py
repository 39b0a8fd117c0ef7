"""The server's failure paths, made on the host (no GPU fault involved): admission
refused for a memory budget below one query, submissions refused at the queue's
capacity, a wait that runs out of time, pending requests failed by a stop (and
their blocked waiters released), a result handed out once to two concurrent
waiters, and tuning / option changes refused while a server is attached.

A long query (20,000 or 200,000 x-updates on the 5,000-document workload, tens of
ms to about a second on the device) keeps the server's only slot busy while the
test acts."""
import threading
import time

import numpy as np
import pytest

import paper_2107_06433_gb300 as swmd
from paper_2107_06433_gb300 import synth

pytestmark = pytest.mark.gpu
LONG = 20000
VERY_LONG = 200000   # about a second on the device: still running when the test stops the server


@pytest.fixture(scope="module")
def served():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2107_06433_gb300 import build
    build.build()
    E, C, (qi, qw) = synth.make("paper")
    corpus = swmd.corpus_from_synth(E, C, path="resident")
    return E, C, qi, qw, corpus


def test_budget_below_one_query_is_refused(served):
    E, C, qi, qw, corpus = served
    with pytest.raises(swmd.SwmdError) as e:
        swmd.swmd_serve_start(corpus, max_batch=2, memory_budget=4096)
    assert e.value.code == swmd.SWMD_ENOMEM


def test_queue_capacity_refuses_and_counts(served):
    E, C, qi, qw, corpus = served
    srv = swmd.swmd_serve_start(corpus, max_batch=1, queue_capacity=2, memory_budget=1 << 30)
    try:
        first = swmd.swmd_serve_submit(srv, qi, qw, 1.0, LONG)
        time.sleep(0.05)                        # admitted: the only slot is busy
        accepted, refused = [first], 0
        for _ in range(6):
            try:
                accepted.append(swmd.swmd_serve_submit(srv, qi, qw, 1.0, 15))
            except swmd.SwmdError as err:
                assert err.code == swmd.SWMD_ENOMEM and "queue full" in str(err)
                refused += 1
        assert refused >= 1 and len(accepted) <= 4
        ref = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
        for tk in accepted[1:]:
            np.testing.assert_array_equal(swmd.swmd_serve_wait(srv, tk, 120000), ref)
        swmd.swmd_serve_wait(srv, first, 120000)
        st = swmd.swmd_serve_stats(srv)
        assert st["rejected"] == refused and st["completed"] == len(accepted)
    finally:
        srv.stop()


def test_wait_times_out_then_completes(served):
    E, C, qi, qw, corpus = served
    srv = swmd.swmd_serve_start(corpus, max_batch=1, memory_budget=1 << 30)
    try:
        tk = swmd.swmd_serve_submit(srv, qi, qw, 1.0, LONG)
        with pytest.raises(swmd.SwmdError) as e:
            swmd.swmd_serve_wait(srv, tk, 0)
        assert e.value.code == swmd.SWMD_ETIMEDOUT
        got = swmd.swmd_serve_wait(srv, tk, -1)       # still queued: waited for again
        assert np.all(np.isfinite(got)) and np.all(got > 0)
        with pytest.raises(swmd.SwmdError) as e:      # collected once
            swmd.swmd_serve_wait(srv, tk, 0)
        assert e.value.code == swmd.SWMD_EINVAL
    finally:
        srv.stop()


def test_stop_fails_pending_requests_and_releases_their_waiters(served):
    E, C, qi, qw, corpus = served
    srv = swmd.swmd_serve_start(corpus, max_batch=1, memory_budget=1 << 30)
    swmd.swmd_serve_submit(srv, qi, qw, 1.0, VERY_LONG)     # in flight: finished by the stop
    time.sleep(0.05)
    pending = [swmd.swmd_serve_submit(srv, qi, qw, 1.0, 15) for _ in range(3)]
    codes = {}

    def waiter(tk):
        try:
            swmd.swmd_serve_wait(srv, tk, -1)
            codes[tk] = swmd.SWMD_OK
        except swmd.SwmdError as err:
            codes[tk] = err.code

    threads = [threading.Thread(target=waiter, args=(tk,)) for tk in pending[1:]]
    for th in threads:
        th.start()
    time.sleep(0.2)                               # the waiters are blocked inside the library
    srv.stop()
    for th in threads:
        th.join(timeout=60)
        assert not th.is_alive()
    assert all(codes[tk] == swmd.SWMD_ESTOPPED for tk in pending[1:]), codes


def test_tuning_and_options_wait_for_the_server(served):
    E, C, qi, qw, corpus = served
    srv = swmd.swmd_serve_start(corpus, max_batch=2, memory_budget=1 << 30)
    try:
        with pytest.raises(swmd.SwmdError) as e:
            swmd.swmd_autotune(corpus, 19, 1)
        assert e.value.code == swmd.SWMD_EINVAL and "server" in str(e.value)
        with pytest.raises(swmd.SwmdError) as e:
            swmd.swmd_corpus_set_options(corpus, k_precision="bf16")
        assert e.value.code == swmd.SWMD_EINVAL
        tk = swmd.swmd_serve_submit(srv, qi, qw, 1.0, 15)
        np.testing.assert_array_equal(swmd.swmd_serve_wait(srv, tk, 60000),
                                      swmd.swmd_query(corpus, qi, qw, 1.0, 15))
    finally:
        srv.stop()
    swmd.swmd_corpus_set_options(corpus, k_precision="fp32")   # allowed again


def test_two_waiters_of_one_ticket_get_it_once(served):
    """Both block until the query is done; one receives the distances, the other
    SWMD_EINVAL (the result is handed out once)."""
    E, C, qi, qw, corpus = served
    srv = swmd.swmd_serve_start(corpus, max_batch=1, memory_budget=1 << 30)
    try:
        tk = swmd.swmd_serve_submit(srv, qi, qw, 1.0, LONG)
        got = {}

        def waiter(name):
            try:
                got[name] = swmd.swmd_serve_wait(srv, tk, -1)
            except swmd.SwmdError as err:
                got[name] = err.code

        threads = [threading.Thread(target=waiter, args=(n,)) for n in ("a", "b")]
        for th in threads:
            th.start()
        for th in threads:
            th.join(timeout=120)
            assert not th.is_alive()
        arrays = [v for v in got.values() if isinstance(v, np.ndarray)]
        codes = [v for v in got.values() if not isinstance(v, np.ndarray)]
        assert len(arrays) == 1 and codes == [swmd.SWMD_EINVAL], got
        assert np.all(np.isfinite(arrays[0])) and np.all(arrays[0] > 0)
    finally:
        srv.stop()
