"""Multi-GPU host logic on CPU ranks (gloo, world size 2 and 3).

The corpus shards by document ranges with no exchange during a query (every
column of c is an independent problem in Algorithm 1).  Each rank takes its
nnz-balanced range from swmd_partition_documents, computes its documents' distances
(the FP64 oracle stands in for the GPU here), and the ranks all-gather; the
concatenation must equal the unsharded result bit for bit."""
import os
import socket

import numpy as np
import pytest

import paper_2107_06433_gb300 as swmd


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sub_corpus(C, b, e):
    from paper_2107_06433_gb300 import synth
    lens = np.diff(C.doc_ptr)[b:e]
    dp = np.zeros(e - b + 1, np.int64)
    np.cumsum(lens, out=dp[1:])
    lo, hi = C.doc_ptr[b], C.doc_ptr[e]
    return synth.Corpus(C.V, e - b, dp, C.word_ids[lo:hi], C.counts[lo:hi], C.vals[lo:hi])


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle
    from paper_2107_06433_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    E, C, (qi, qw) = synth.make("tiny")
    bounds = swmd.swmd_partition_documents(C.N, np.diff(C.doc_ptr), world)
    b, e = int(bounds[rank]), int(bounds[rank + 1])
    part = _sub_corpus(C, b, e)
    rp, col, val = part.csr()
    local = oracle.wmd(E, rp, col, val, part.N, qi, qw, 1.0, 15) if part.N else np.zeros(0)
    gathered = [None] * world
    dist.all_gather_object(gathered, (b, e, local))
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.concatenate([g[2] for g in gathered]))
        np.save(os.path.join(out_dir, "bounds.npy"), bounds)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_query_equals_unsharded(tmp_path, world):
    import torch.multiprocessing as mp
    import oracle
    from paper_2107_06433_gb300 import build, synth
    build.build()
    oracle.build()
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    E, C, (qi, qw) = synth.make("tiny")
    rp, col, val = C.csr()
    full = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, 15)
    np.testing.assert_array_equal(np.load(tmp_path / "gathered.npy"), full)
    bounds = np.load(tmp_path / "bounds.npy")
    nnz = np.diff(C.doc_ptr)
    loads = [nnz[bounds[g]:bounds[g + 1]].sum() for g in range(world)]
    assert max(loads) - min(loads) <= nnz.max()      # balanced to within one document


def test_partition_properties():
    from paper_2107_06433_gb300 import build
    build.build()
    rng = np.random.default_rng(0)
    nnz = rng.integers(1, 300, size=1000)
    for parts in (1, 2, 7, 64):
        b = swmd.swmd_partition_documents(len(nnz), nnz, parts)
        assert b[0] == 0 and b[-1] == len(nnz) and np.all(np.diff(b) >= 0)
        loads = np.array([nnz[b[g]:b[g + 1]].sum() for g in range(parts)])
        assert loads.max() - nnz.sum() / parts <= nnz.max()
    assert list(swmd.swmd_partition_documents(0, np.zeros(0), 3)) == [0, 0, 0, 0]
    with pytest.raises(swmd.SwmdError):
        swmd.swmd_partition_documents(3, [1, -1, 2], 2)
