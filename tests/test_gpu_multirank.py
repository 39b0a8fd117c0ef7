"""The sharded CUDA path across ranks: gloo ranks in separate processes, each
loading its own nnz-balanced document range (swmd_partition_documents,
doc_begin / doc_end) into the library on the one GPU this test has, each running
the query through swmd_query, then an all-gather.  The concatenation must equal the
unsharded query bit for bit: every column of c is an independent problem in
Algorithm 1, and a document's arithmetic does not depend on the other documents
of its range.  (The ranks' kernels never wait on one another, so sharing one GPU
between the processes only serialises them.)"""
import os
import socket

import numpy as np
import pytest

import paper_2107_06433_gb300 as swmd

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir, workload):
    import torch
    import torch.distributed as dist
    from paper_2107_06433_gb300 import synth
    torch.cuda.set_device(0)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    E, C, (qi, qw) = synth.make(workload)
    bounds = swmd.swmd_partition_documents(C.N, np.diff(C.doc_ptr), world)
    b, e = int(bounds[rank]), int(bounds[rank + 1])
    rp, col, val = C.csr()
    local = np.zeros(0)
    if e > b:
        corpus = swmd.swmd_create_corpus(C.V, C.N, rp, col, val, E, doc_begin=b, doc_end=e)
        local = swmd.swmd_query(corpus, qi, qw, 1.0, 15)
        corpus.close()
    gathered = [None] * world
    dist.all_gather_object(gathered, (b, e, local))
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.concatenate([g[2] for g in gathered]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("workload,world", [("paper", 2), ("tiny", 3)])
def test_ranks_on_document_ranges_equal_the_whole_corpus(tmp_path, workload, world):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    from paper_2107_06433_gb300 import build, synth
    build.build()
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), workload), nprocs=world, join=True)
    E, C, (qi, qw) = synth.make(workload)
    rp, col, val = C.csr()
    whole = swmd.swmd_query(swmd.swmd_create_corpus(C.V, C.N, rp, col, val, E), qi, qw, 1.0, 15)
    np.testing.assert_array_equal(np.load(tmp_path / "gathered.npy"), whole)
