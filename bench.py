"""Benchmark: Sinkhorn WMD of one query against a corpus on GB300.

One step = one whole query through the hot path (query staging, cost/kernel
matrix, all Sinkhorn iterations and the final distances) over the resident corpus
of the 1,000,000-document workload (V=500,000, d=300, documents of 5-30 Zipf words,
17.5M nonzeros, v_r=32, lambda=1, 15 iterations, FP32).  Inputs are synthetic
(synth.py).

  value      WMD/s (documents x queries / device time), inputs resident in HBM,
             L2 flushed (1 GiB write) before every timed step, outside the events.
  e2e        WMD/s through swmd_query with host buffers: the query's ids and
             weights go host->device and the N distances device->host every step.
  roofline   the dominant kernel of a step: algorithmic bytes or flops per launch
             over its CUDA-event duration, against MEASURED_PEAKS.json; `traffic`
             from the committed ncu capture when it matches the current sources.
  fused_iteration  the per-iteration fused SDDMM-SpMM and the plain SDDMM + SpMM
             kernels on the same workload (FP32 and BF16 K): effective GB/s against
             the HBM peak, and whole queries on each path (`hbm_regime`).
  paper_shaped the 5,000-document paper-shaped workload (V=100,000, 10-300 words,
             v_r=19): the whole query, its paths and the 1-to-1 pairs of Table II.
  batched    256 queries (v_r uniform in [4,64]) over 100,000 documents of 10-200
             words in one swmd_query_batch call after autotuning, FP32 and BF16 K,
             against the same queries one at a time.
  serving    a query server over the resident 1,000,000-document corpus with BF16 K
             fed by Poisson arrivals at 50, 200 and 1000 queries/s (v_r uniform in
             [4,128]): queries/s and p50/p99 latency, against the same queries run
             one at a time through swmd_query (FP32 and BF16 K) and through
             swmd_query_batch (BF16 K, 16 per call), and the BF16 error.
  cpu_baseline  the FP64 oracle timed on the host cores on whole queries of the
             workload, and on one host thread on a document sample (`single_core`);
             the dense oracle on the 200-document workload and on 64 documents of the
             paper-shaped one (`dense`).

`--impl reference` times the oracle alone (the reference arm).  Under torchrun
(N > 1) every rank holds its own partition of the workload's size (weak scaling,
no collective on the data path) and rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "large"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP32 CUDA-core peak: the device's SMs x 128 FP32 lanes x 2 flop (FMA), times the SM clock.
FP32_LANES = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--path", default="auto", choices=["resident", "fused", "plain", "auto"])
    ap.add_argument("--kprec", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paths", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the per-iteration kernel section")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper-shaped section")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-pairs", action="store_true")
    ap.add_argument("--max-iter", type=int, default=None,
                    help="x-updates per query in the timed step (default: the workload's, 15); "
                         "0 times the gathers and the final step alone")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


# the kernel sources each measured traffic figure depends on
KERNEL_SOURCES = {
    "resident": ["common.cuh", "resident_cols.cu", "resident_cols.cuh", "resident_cols_long.cu",
                 "resident_regs.cuh", "resident_tiled.cu", "walk.cuh", "walk3.cuh", "walk_resident.cu"],
    "cost": ["common.cuh", "cost.cu"],
    "fused": ["common.cuh", "walk.cuh", "walk3.cuh", "walk_fused.cu"],
    "plain": ["common.cuh", "walk.cuh", "walk3.cuh", "walk_plain.cu"],
}


def source_hash(kind):
    """Hash of the CUDA sources of one kernel family: its ncu traffic is valid only
    for these sources."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2107_06433_gb300", "csrc")
    for name in KERNEL_SOURCES[kind]:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if it matches the
    current sources of that kernel."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    e = t.get(kernel_key)
    if not e or e.get("source_hash") != source_hash(kernel_key.split(":")[0]):
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ algorithmic counts
def cost_counts(Vu, d, vrp, vr, kb):
    """a1: reads the used embedding rows, writes K^T and KM^T; 3 flops per
    (query word, word, dimension): subtract, multiply, add."""
    return Vu * d * 4 + 2 * Vu * vrp * kb, 3.0 * Vu * vr * d


def fused_iter_bytes(nnz, N, Vu, vrp, kb):
    """a3 per launch: c's nonzeros (id + value), doc_ptr, K^T once, u read and written."""
    return nnz * 8 + (N + 1) * 4 + Vu * vrp * kb + 2 * N * vrp * 4


def plain_iter_bytes(nnz, N, Vu, vrp, kb):
    """SDDMM (c, K^T, u; writes v) + SpMM (c, v, K^T; writes u)."""
    return (nnz * 8 + (N + 1) * 4 + Vu * vrp * kb + N * vrp * 4 + nnz * 4) + \
        (nnz * 8 + (N + 1) * 4 + nnz * 4 + Vu * vrp * kb + N * vrp * 4)


def resident_counts(nnz, N, Vu, vrp, vr, kb, t):
    """a3 x t + a4 in one launch: compulsory bytes (c, doc_ptr, K^T, KM^T, the
    output) and flops: per nonzero and iteration 2 v_r FMAs + 1 divide (4 v_r + 1
    flop), in the final step 2 dots, a divide and an add (4 v_r + 3)."""
    byts = nnz * 8 + (N + 1) * 4 + 2 * Vu * vrp * kb + N * (8 + 4)
    flops = float(t) * nnz * (4 * vr + 1) + nnz * (4 * vr + 3) + t * N * vr
    return byts, flops


# ------------------------------------------------------------------ oracle timing
def time_oracle(E, C, qi, qw, lam, t, budget_s=12.0, max_runs=50):
    import oracle
    rp, col, val = C.csr()
    runs, t0 = 0, time.perf_counter()
    while True:
        oracle.wmd(E, rp, col, val, C.N, qi, qw, lam, t, "sparse")
        runs += 1
        el = time.perf_counter() - t0
        if el >= budget_s or runs >= max_runs:
            break
    return runs, el, oracle.get_threads()


def time_oracle_one_core(E, C, qi, qw, lam, t, n=20000, budget_s=6.0, max_runs=10):
    """The same oracle on one host thread, on the first n documents (document_sample)."""
    n, runs, el, cores = time_oracle_sample(E, C, qi, qw, lam, t, n, budget_s, max_runs, threads=1)
    return {"value": n * runs / el, "unit": "WMD/s", "cores": cores,
            "sample": f"{runs} queries against the first {n} documents, one thread, sparse FP64 mode"}


def first_documents_csr(C, n):
    """The V x n CSR of the corpus's first n documents (columns 0..n-1)."""
    end = int(C.doc_ptr[n])
    words = np.asarray(C.word_ids[:end], np.int64)
    docs = np.repeat(np.arange(n, dtype=np.int32), np.diff(np.asarray(C.doc_ptr[:n + 1])))
    order = np.lexsort((docs, words))
    rp = np.zeros(C.V + 1, np.int64)
    np.cumsum(np.bincount(words, minlength=C.V), out=rp[1:])
    return rp, docs[order], np.asarray(C.vals[:end], np.float32)[order]


def document_sample(E, C, qi, n):
    """The first n documents as an oracle input over the words they and the query use:
    (E rows of those words, V' x n CSR, query ids remapped).  Every document is an
    independent problem in Algorithm 1 and a word no document holds adds nothing, so
    the oracle gives these documents the same distances on the smaller vocabulary."""
    n = min(n, C.N)
    end = int(C.doc_ptr[n])
    words = np.asarray(C.word_ids[:end], np.int64)
    used = np.unique(np.concatenate([words, np.asarray(qi, np.int64)]))
    remap = np.full(C.V, -1, np.int64)
    remap[used] = np.arange(len(used))
    w2 = remap[words]
    docs = np.repeat(np.arange(n, dtype=np.int32), np.diff(np.asarray(C.doc_ptr[:n + 1])))
    order = np.lexsort((docs, w2))
    rp = np.zeros(len(used) + 1, np.int64)
    np.cumsum(np.bincount(w2, minlength=len(used)), out=rp[1:])
    return (np.ascontiguousarray(E[used]), rp, docs[order], np.asarray(C.vals[:end], np.float32)[order],
            remap[np.asarray(qi, np.int64)].astype(np.int32), n)


def time_oracle_sample(E, C, qi, qw, lam, t, n, budget_s, max_runs, threads=None):
    """The sparse oracle on the first n documents (document_sample), repeated until
    budget_s has passed; threads: host threads (None = all)."""
    import oracle
    Es, rp, col, val, qs, n = document_sample(E, C, qi, n)
    n0 = oracle.get_threads()
    try:
        if threads:
            oracle.set_threads(threads)
        runs, t0 = 0, time.perf_counter()
        while True:
            oracle.wmd(Es, rp, col, val, n, qs, qw, lam, t, "sparse")
            runs += 1
            el = time.perf_counter() - t0
            if el >= budget_s or runs >= max_runs:
                break
        cores = oracle.get_threads()
    finally:
        oracle.set_threads(n0)
    return n, runs, el, cores


def time_oracle_dense(synth, budget_s=4.0):
    """The dense oracle (Algorithm 1 with dense matrices, as Table I runs it) on the
    200-document workload and on the first 64 documents of the paper-shaped one."""
    import oracle
    out = {}
    for name, ndocs in (("tiny", None), ("paper", 64)):
        E, C, (qi, qw) = synth.make(name)
        w = synth.WORKLOADS[name]
        if ndocs is None:
            rp, col, val = C.csr()
            ndocs = C.N
        else:
            rp, col, val = first_documents_csr(C, ndocs)
        runs, t0 = 0, time.perf_counter()
        while True:
            oracle.wmd(E, rp, col, val, ndocs, qi, qw, w.lam, w.max_iter, "dense")
            runs += 1
            el = time.perf_counter() - t0
            if el >= budget_s or runs >= 20:
                break
        out[name] = {"value": ndocs * runs / el, "unit": "WMD/s", "cores": oracle.get_threads(),
                     "sample": f"{runs} queries against {ndocs} documents, dense FP64 mode"}
    return out


def config_dict(w, C):
    return {"workload": w.name, "V": w.V, "d": w.d, "documents": C.N, "nnz": C.nnz,
            "v_r": w.v_r, "lambda": w.lam, "max_iter": w.max_iter,
            "doc_lengths": f"{w.len_kind} {w.len_lo}-{w.len_hi}",
            "word_ids": "Zipf(1.1)", "l2": "flushed (1 GiB write) before every timed step"}


def reference_arm(args, budget_s=240.0):
    """The oracle as the reference arm: exactly --steps steps, each one query against a
    sample of the workload's documents: all of them when the steps fit the time budget,
    else the first n (document_sample: their words only), n sized from a warm-up query
    on a sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2107_06433_gb300 import synth
    import oracle
    w = synth.WORKLOADS[args.workload]
    E, C, (qi, qw) = synth.make(w)
    oracle.build()
    steps = max(int(args.steps), 1)
    n0 = min(C.N, 20000)
    n0, runs, el, _ = time_oracle_sample(E, C, qi, qw, w.lam, w.max_iter, n0, 0.0, 1)
    per_doc = el / n0
    n_docs = max(16, min(C.N, int(budget_s / (steps * per_doc))))
    if n_docs >= C.N:
        n_docs = C.N
        rp, col, val = C.csr()
        Es, qs = E, qi
    else:
        Es, rp, col, val, qs, n_docs = document_sample(E, C, qi, n_docs)
    for _ in range(max(args.warmup - 1, 0)):
        oracle.wmd(Es, rp, col, val, n_docs, qs, qw, w.lam, w.max_iter)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.wmd(Es, rp, col, val, n_docs, qs, qw, w.lam, w.max_iter)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n_docs * steps / total
    cores = oracle.get_threads()
    sample = (f"{steps} queries of the {w.name} workload against "
              f"{'all ' if n_docs == C.N else 'its first '}{n_docs} documents"
              f"{'' if n_docs == C.N else ' (cost matrix over their words)'}, sparse FP64 mode")
    line = {
        "impl": "reference", "metric": "WMDs/s", "value": value, "unit": "WMD/s",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(w, C),
        "cpu_baseline": {"value": value, "unit": "WMD/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "WMD/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def event_pair():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def compare_paths(swmd, corpus, d_ids, d_r, d_out, d_status, flush, stream, vr, lam, t, info, C,
                  peaks, kb):
    """Whole-query time of each path, and one fused vs one plain iteration."""
    import torch
    res = {}
    reps = 50

    def timed(path):
        times = []
        with torch.cuda.stream(stream):
            for k in range(reps + 3):
                flush.zero_()
                a, b = event_pair()
                a.record(stream)
                swmd.swmd_query_device(corpus, d_ids, d_r, vr, lam, t, d_out, d_status,
                                       stream=stream)
                b.record(stream)
                if k >= 3:
                    times.append((a, b))
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in times)
        res[path] = {"ms_per_query": ms, "wmds_per_s": C.N / (ms * 1e-3)}

    for path in ("resident", "fused", "plain"):
        swmd.swmd_corpus_set_options(corpus, path=path)
        timed(path)
    # the column-split solver with its buckets of up to 96 rows and the longest
    # documents on the register solver (solver 4; not the automatic choice here): a
    # supplementary figure, which cannot cost the line
    try:
        swmd.swmd_corpus_set_options(corpus, path="resident", solver=4)
        timed("resident_long_buckets")
    except Exception as e:
        res["resident_long_buckets"] = {"error": str(e)[:200]}
    swmd.swmd_corpus_set_options(corpus, path="auto", solver=0)
    res["iteration_kernel"] = iteration_kernels(swmd, corpus, d_ids, d_r, d_status, flush, stream,
                                                vr, lam, info, C, peaks, kb)
    swmd.swmd_corpus_set_options(corpus, path="auto")
    return res


def iteration_kernels(swmd, corpus, d_ids, d_r, d_status, flush, stream, vr, lam, info, C, peaks,
                      kb, reps=30, traffic_key=None):
    """One fused SDDMM-SpMM launch vs one SDDMM + one SpMM launch, on the
    per-iteration layout (swmd_get_mapping of the fused path)."""
    import torch
    swmd.swmd_corpus_set_options(corpus, path="fused")
    vrp = swmd.swmd_get_mapping(corpus, vr, "fused")[0]
    per = {}
    for path in ("fused", "plain"):
        with torch.cuda.stream(stream):
            swmd.swmd_step_cost(corpus, d_ids, d_r, vr, lam, d_status, stream=stream)
            swmd.swmd_step_iterate(corpus, vr, 1, 1, path, stream=stream)
            evs = []
            for k in range(reps):
                flush.zero_()
                a, b = event_pair()
                a.record(stream)
                swmd.swmd_step_iterate(corpus, vr, 1, 0, path, stream=stream)
                b.record(stream)
                evs.append((a, b))
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        byts = (fused_iter_bytes if path == "fused" else plain_iter_bytes)(
            info.nnz, C.N, info.V_used, vrp, kb)
        gbs = byts / (ms * 1e-3) / 1e9
        per[path] = {"ms_per_iteration": ms, "algorithmic_bytes": byts, "vrp": vrp, "gbs": gbs,
                     "frac_of_hbm": gbs / peaks["hbm_gbs"]}
        if traffic_key:
            per[path]["traffic"] = measured_traffic(f"{path}:{traffic_key}")
    per["fusion_speedup"] = per["plain"]["ms_per_iteration"] / per["fused"]["ms_per_iteration"]
    return per


def time_query_device(swmd, torch, corpus, stream, flush, ids, r, lam, t, out, status, reps=3):
    d_ids = torch.from_numpy(ids).cuda()
    d_r = torch.from_numpy(r).cuda()
    evs = []
    with torch.cuda.stream(stream):
        swmd.swmd_query_device(corpus, d_ids, d_r, len(ids), lam, t, out, status, stream=stream)
        for _ in range(reps):
            flush.zero_()
            a, b = event_pair()
            a.record(stream)
            swmd.swmd_query_device(corpus, d_ids, d_r, len(ids), lam, t, out, status, stream=stream)
            b.record(stream)
            evs.append((a, b))
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in evs)


def one_to_one(swmd, torch, corpus, C, qi, qw, lam, t, flush, stream, d, alu_peak, one_to_n_ms,
               one_to_n_out):
    """1-to-1 WMD (Section III-E, Table II): the query against documents as independent
    pairs whose cost is built over each document's words only.  All documents of the
    corpus, and a 100-candidate re-ranking set beside the whole 1-to-N query.
    Algorithmic flops per pair: v_r v_x (3 d + 4 t + 4) -- the cost block (a
    subtraction and an FMA per dimension), t SDDMM + SpMM passes (2 FMAs per entry)
    and the final pass (2 FMAs per entry)."""
    ids, r = swmd.swmd_select(C.V, qi, qw)
    vr = len(ids)
    docs = [swmd.swmd_select(C.V, C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]],
                             C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]]) for j in range(C.N)]
    dev = lambda x: torch.from_numpy(x).cuda()
    res = {}
    for label, sel, reps in (("all_documents", list(range(C.N)), 50),
                             ("rerank_100", list(range(0, C.N, max(1, C.N // 100)))[:100], 200)):
        qp, qi_, qr = swmd._ragged([(ids, r)] * len(sel))
        xp, xi_, xc = swmd._ragged([docs[j] for j in sel])
        args = [dev(x) for x in (qp, qi_, qr, xp, xi_, xc)]
        max_x = max(len(docs[j][0]) for j in sel)
        out = torch.empty(len(sel), dtype=torch.float64, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        evs = []
        with torch.cuda.stream(stream):
            for k in range(reps + 3):
                flush.zero_()
                a_, b_ = event_pair()
                a_.record(stream)
                swmd.swmd_wmd_pairs_device(corpus, len(sel), *args, vr, max_x, lam, t, out, status,
                                           stream=stream)
                b_.record(stream)
                if k >= 3:
                    evs.append((a_, b_))
        torch.cuda.synchronize()
        ms = statistics.mean(x.elapsed_time(y) for x, y in evs)
        flops = float(sum(vr * len(docs[j][0]) * (3 * d + 4 * t + 4) for j in sel))
        ach = flops / (ms * 1e-3) / 1e12
        got = out.cpu().numpy()
        res[label] = {"pairs": len(sel), "ms": ms, "wmds_per_s": len(sel) / (ms * 1e-3),
                      "algorithmic_flops": flops, "tflops": ach, "frac_of_alu": ach / alu_peak,
                      "status": int(status.item()),
                      "max_rel_vs_one_to_n": float(np.max(np.abs(got - one_to_n_out[sel]) /
                                                          np.abs(one_to_n_out[sel])))}
    res["rerank_100"]["one_to_n_whole_query_ms"] = one_to_n_ms
    # end to end through the host entry point (selection on the host, copies both ways)
    reps = 10
    targets = [(C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]], C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]])
               for j in range(C.N)]
    swmd.swmd_wmd_pairs(corpus, [(qi, qw)] * C.N, targets, lam, t)
    t0 = time.perf_counter()
    for _ in range(reps):
        swmd.swmd_wmd_pairs(corpus, [(qi, qw)] * C.N, targets, lam, t)
    res["all_documents"]["e2e_wmds_per_s"] = C.N * reps / (time.perf_counter() - t0)
    res["alu_peak_tflops"] = alu_peak
    return res


def hbm_regime(swmd, torch, corpus, C, ids, r, w, flush, stream, peaks):
    """The per-iteration fused and plain kernels where c and u exceed L2 (the
    headline corpus), in FP32 and BF16 K, and whole queries on each path."""
    info = corpus.info()
    d_ids = torch.from_numpy(ids).cuda()
    d_r = torch.from_numpy(r).cuda()
    d_status = torch.zeros(1, dtype=torch.int32, device="cuda")
    per = {}
    for kp, kb in (("fp32", 4), ("bf16", 2)):
        swmd.swmd_corpus_set_options(corpus, k_precision=kp)
        per[kp] = iteration_kernels(swmd, corpus, d_ids, d_r, d_status, flush, stream, len(ids),
                                    w.lam, info, C, peaks, kb, reps=10, traffic_key=f"{w.name}:{kp}")
    d_out = torch.empty(C.N, dtype=torch.float64, device="cuda")
    q = {}
    for path, kp in (("resident", "fp32"), ("fused", "fp32"), ("plain", "fp32"), ("resident", "bf16"),
                     ("fused", "bf16")):
        swmd.swmd_corpus_set_options(corpus, path=path, k_precision=kp)
        ms = time_query_device(swmd, torch, corpus, stream, flush, ids, r, w.lam, w.max_iter,
                               d_out, d_status)
        q[f"{path}/{kp}"] = {"ms_per_query": ms, "wmds_per_s": C.N / (ms * 1e-3)}
    swmd.swmd_corpus_set_options(corpus, path="auto", k_precision="fp32")
    q["resident_over_fused_fp32"] = q["fused/fp32"]["ms_per_query"] / q["resident/fp32"]["ms_per_query"]
    return {"workload": w.name, "documents": C.N, "nnz": info.nnz, "v_r": len(ids),
            "l2": "flushed before every timed launch", "iteration_kernel": per, "query": q}


def paper_shaped(swmd, synth, torch, flush, stream, peaks, alu_peak, rank):
    """The paper-shaped workload (Section III-B2 statistics: V = 100,000, d = 300, 5,000
    documents, v_r = 19): the whole query (automatic path), each path, the fused vs plain
    iteration kernels and the 1-to-1 pairs of Table II."""
    w = synth.WORKLOADS["paper"]
    E, C, (qi, qw) = synth.make(w)
    corpus = swmd.corpus_from_synth(E, C)
    info = corpus.info()
    ids, r = swmd.swmd_select(C.V, qi, qw)
    vr = len(ids)
    d_ids = torch.from_numpy(ids).cuda()
    d_r = torch.from_numpy(r).cuda()
    d_out = torch.empty(C.N, dtype=torch.float64, device="cuda")
    d_status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ms = time_query_device(swmd, torch, corpus, stream, flush, ids, r, w.lam, w.max_iter, d_out,
                           d_status, reps=50)
    out_dev = d_out.cpu().numpy()
    host = np.empty(C.N, np.float64)
    for _ in range(3):
        swmd.swmd_query(corpus, qi, qw, w.lam, w.max_iter, out=host)
    reps, t0 = 200, time.perf_counter()
    for _ in range(reps):
        swmd.swmd_query(corpus, qi, qw, w.lam, w.max_iter, out=host)
    e2e = C.N * reps / (time.perf_counter() - t0)
    res = {"workload": w.name, "documents": C.N, "nnz": info.nnz, "v_r": vr,
           "path": swmd.swmd_resolve_path(corpus, vr), "ms_per_query": ms,
           "wmds_per_s": C.N / (ms * 1e-3), "e2e_wmds_per_s": e2e}
    res["paths"] = compare_paths(swmd, corpus, d_ids, d_r, d_out, d_status, flush, stream, vr, w.lam,
                                 w.max_iter, info, C, peaks, 4)
    res["one_to_one"] = one_to_one(swmd, torch, corpus, C, qi, qw, w.lam, w.max_iter, flush, stream,
                                   w.d, alu_peak, ms, out_dev)
    corpus.close()
    return res


def batched(swmd, synth, torch):
    """256 queries (v_r uniform in [4, 64]) over 100,000 documents in one
    swmd_query_batch call, autotuned, FP32 and BF16 K, against the same queries
    one at a time through swmd_query."""
    w = synth.WORKLOADS["batch"]
    E, C, _ = synth.make(w)
    qs = synth.batch_queries(C.V, 256, 4, 64, seed=synth.SEED + 2)
    res = {"workload": "batch", "documents": C.N, "nnz": C.nnz, "queries": len(qs),
           "v_r": "uniform 4-64", "lambda": 1.0, "max_iter": 15}
    ref = None
    for kp in ("fp32", "bf16"):
        corpus = swmd.corpus_from_synth(E, C, k_precision=kp)
        t0 = time.perf_counter()
        paths = {}
        for vr in sorted({len(q[0]) for q in qs}):
            tr = swmd.swmd_autotune(corpus, vr, 2)
            paths[tr["path"]] = paths.get(tr["path"], 0) + 1
        tune_s = time.perf_counter() - t0
        # the first call of a batch shape runs eagerly, the second captures its
        # graph; later calls replay it
        t0 = time.perf_counter()
        swmd.swmd_query_batch(corpus, qs, 1.0, 15)
        first = time.perf_counter() - t0
        t0 = time.perf_counter()
        swmd.swmd_query_batch(corpus, qs, 1.0, 15)
        second = time.perf_counter() - t0
        t0 = time.perf_counter()
        out = swmd.swmd_query_batch(corpus, qs, 1.0, 15)
        tb = time.perf_counter() - t0
        row = {"batch_qps": len(qs) / tb, "batch_wmds_per_s": len(qs) * C.N / tb,
               "batch_s": tb, "first_call_s": first, "capture_call_s": second, "autotune_s": tune_s,
               "paths_chosen": {("fused" if k == 0 else "resident"): v for k, v in paths.items()}}
        if kp == "fp32":
            t0 = time.perf_counter()
            alone = [swmd.swmd_query(corpus, qi, qw, 1.0, 15) for qi, qw in qs]
            ts = time.perf_counter() - t0
            row["one_at_a_time_qps"] = len(qs) / ts
            row["batch_speedup"] = ts / tb
            row["batch_equals_alone_bitwise"] = bool(all(np.array_equal(out[i], alone[i])
                                                         for i in range(len(qs))))
            ref = out
        else:
            row["max_rel_err_vs_fp32"] = float(np.max(np.abs(out - ref) / np.abs(ref)))
        res[kp] = row
        corpus.close()
    return res


def serving(swmd, synth, torch, rates=(50.0, 200.0, 1000.0), n=200, E=None, C=None):
    """Poisson arrivals (v_r uniform in [4, 128]) into a server over the resident
    1,000,000-document corpus with BF16 K, against the same queries one at a time
    through swmd_query with FP32 K.  E, C: that workload's arrays if already made."""
    w = synth.WORKLOADS["large"]
    if E is None or C is None or C.N != w.N:
        E, C, _ = synth.make(w)
    qs = synth.batch_queries(C.V, n, 4, 128, seed=synth.SEED + 1)
    res = {"workload": "large", "documents": C.N, "queries_per_rate": n, "v_r": "uniform 4-128",
           "lambda": 1.0, "max_iter": 15}
    c32 = swmd.corpus_from_synth(E, C, k_precision="fp32")
    lat, alone = [], []
    t0 = time.perf_counter()
    for qi, qw in qs:
        a = time.perf_counter()
        alone.append(swmd.swmd_query(c32, qi, qw, 1.0, 15))
        lat.append((time.perf_counter() - a) * 1e3)
    one_qps = n / (time.perf_counter() - t0)
    c32.close()
    res["one_at_a_time_fp32"] = {"qps": one_qps, "p50_ms": float(np.percentile(lat, 50)),
                                 "p99_ms": float(np.percentile(lat, 99))}
    c16 = swmd.corpus_from_synth(E, C, k_precision="bf16")
    lat16 = []
    t0 = time.perf_counter()
    for qi, qw in qs:
        a = time.perf_counter()
        swmd.swmd_query(c16, qi, qw, 1.0, 15)
        lat16.append((time.perf_counter() - a) * 1e3)
    res["one_at_a_time_bf16"] = {"qps": n / (time.perf_counter() - t0), "p50_ms": float(np.percentile(lat16, 50)),
                                 "p99_ms": float(np.percentile(lat16, 99))}
    # the same queries through swmd_query_batch, 16 per call (one cost and one
    # multi-query solver launch per layout group of each call)
    nb = 16
    swmd.swmd_query_batch(c16, qs[:nb], 1.0, 15)
    t0 = time.perf_counter()
    for i in range(0, n, nb):
        swmd.swmd_query_batch(c16, qs[i:i + nb], 1.0, 15)
    res["batched_bf16"] = {"qps": n / (time.perf_counter() - t0), "queries_per_call": nb}
    served = {}
    err = 0.0
    for rate in rates:
        arrivals = synth.poisson_arrivals(rate, n, seed=synth.SEED + int(rate))
        srv = swmd.swmd_serve_start(c16, max_batch=32, memory_budget=4 << 30)
        tickets = []
        t0 = time.perf_counter()
        for (qi, qw), at in zip(qs, arrivals):
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            tickets.append(swmd.swmd_serve_submit(srv, qi, qw, 1.0, 15))
        outs = [swmd.swmd_serve_wait(srv, tk, 120000) for tk in tickets]
        st = swmd.swmd_serve_stats(srv)
        srv.stop()
        if rate == rates[0]:
            err = max(float(np.max(np.abs(o - r) / np.abs(r))) for o, r in zip(outs, alone))
        served[f"{rate:.0f}"] = {"offered_qps": rate, "qps": st["qps"], "p50_ms": st["p50_ms"],
                                 "p99_ms": st["p99_ms"], "mean_batch": st["mean_batch"]}
    c16.close()
    res["served_bf16"] = served
    res["bf16_max_rel_err_vs_fp32"] = err
    return res


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import paper_2107_06433_gb300 as swmd
    from paper_2107_06433_gb300 import build as nbuild, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist
    nbuild.build()

    w = synth.WORKLOADS[args.workload]
    if args.max_iter is not None:
        w = dataclasses.replace(w, max_iter=args.max_iter)
    # weak scaling: rank r holds its own partition of w.N documents (its own seed)
    E, C, (qi, qw) = synth.make(w, seed=synth.SEED + 7919 * rank)
    if rank > 0:   # every rank answers the same query
        _, _, (qi, qw) = synth.make(w)
    kprec = {"fp32": 0, "bf16": 1, "fp16": 2}[args.kprec]
    kb = 4 if kprec == 0 else 2
    corpus = swmd.corpus_from_synth(E, C, path=args.path, k_precision=kprec, device=local)
    info = corpus.info()
    ids, r = swmd.swmd_select(C.V, qi, qw)
    vr = len(ids)
    run_path = args.path if args.path != "auto" else swmd.swmd_resolve_path(corpus, vr)
    d_ids = torch.from_numpy(ids).cuda()
    d_r = torch.from_numpy(r).cuda()
    d_out = torch.empty(C.N, dtype=torch.float64, device="cuda")
    d_status = torch.zeros(1, dtype=torch.int32, device="cuda")
    flush = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    lam, t = w.lam, w.max_iter

    def one_step(ev=None):
        # the query's launches, with events around the cost kernel and the solver
        if ev is not None:
            ev[0].record(stream)
        swmd.swmd_step_cost(corpus, d_ids, d_r, vr, lam, d_status, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        if run_path == "resident":
            swmd.swmd_step_resident(corpus, vr, t, d_out, stream=stream)
        else:
            swmd.swmd_step_iterate(corpus, vr, t, 1, run_path, stream=stream)
            swmd.swmd_step_final(corpus, vr, int(t == 0), d_out, stream=stream)
        if ev is not None:
            ev[2].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            flush.zero_()
            one_step()
    torch.cuda.synchronize()

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.zero_()
            one_step(evs[k])
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    cost_ms = [evs[k][0].elapsed_time(evs[k][1]) for k in range(K)]
    solve_ms = [evs[k][1].elapsed_time(evs[k][2]) for k in range(K)]
    total_ms = sum(a + b for a, b in zip(cost_ms, solve_ms))
    if pg:
        tt = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        total_ms = float(tt.item())
    st = int(d_status.item())
    out_dev = d_out.cpu().numpy()

    # ---- e2e through the host API (host ids/weights in, host distances out)
    e2e_steps = min(K, 200)
    host_out = np.empty(C.N, np.float64)
    for _ in range(3):
        swmd.swmd_query(corpus, qi, qw, lam, t, out=host_out)
    e2e_s = 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        swmd.swmd_query(corpus, qi, qw, lam, t, out=host_out)
        e2e_s += time.perf_counter() - t0
    if pg:
        tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        e2e_s = float(tt.item())
    if not np.allclose(host_out, out_dev, rtol=1e-12, atol=0):
        raise SystemExit("host and device entry points disagree")

    # ---- roofline of the dominant kernel
    peaks, peak_kind = load_peaks()
    vrp = swmd.swmd_get_mapping(corpus, vr, run_path)[0]
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    cost_avg = statistics.mean(cost_ms) * 1e-3
    solve_avg = statistics.mean(solve_ms) * 1e-3
    cb, cf = cost_counts(info.V_used, w.d, vrp, vr, kb)
    if run_path == "resident":
        sb, sf = resident_counts(info.nnz, C.N, info.V_used, vrp, vr, kb, t)
        skey = f"resident:{w.name}:{args.kprec}"
    else:
        sb = t * fused_iter_bytes(info.nnz, C.N, info.V_used, vrp, kb)
        sf = float(t + 1) * info.nnz * (4 * vr + 1)
        skey = f"{run_path}:{w.name}:{args.kprec}"
    alu_peak = sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12   # TFLOP/s at the sampled clock
    if solve_avg >= cost_avg:
        name, key, dur, byts, flops = f"{run_path} solver (a3 x t + a4)", skey, solve_avg, sb, sf
    else:
        name, key, dur, byts, flops = "cost/kernel matrix (a1)", f"cost:{w.name}:{args.kprec}", cost_avg, cb, cf
    ridge = alu_peak * 1e12 / (peaks["hbm_gbs"] * 1e9)
    traffic = measured_traffic(key)
    if flops / byts >= ridge:
        ach = flops / dur / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": ach / alu_peak, "traffic": traffic, "kernel": name,
                "peak_source": f"derived: {sms} SMs x {FP32_LANES} FP32 lanes x 2 flop x "
                               f"{sm_mhz:.0f} MHz (median sampled SM clock)",
                "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": byts}
    else:
        ach = byts / dur / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": traffic, "kernel": name,
                "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": byts, "algorithmic_flops_per_launch": flops}

    # ---- the per-iteration fused vs plain kernels on this workload (metric's HBM GB/s)
    hbm = None
    if rank == 0 and not args.no_large:
        hbm = hbm_regime(swmd, torch, corpus, C, ids, r, w, flush, stream, peaks)

    line = {
        "metric": "WMDs/s", "value": C.N * world * K / (total_ms * 1e-3), "unit": "WMD/s",
        "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if kprec == 0 else args.kprec + "-K/f32",
        "data": "synthetic", "config": config_dict(w, C) | {"path": run_path,
                                                           "k_precision": args.kprec},
        "e2e": {"value": C.N * world * e2e_steps / e2e_s, "unit": "WMD/s",
                "h2d_bytes_per_step": int(len(qi) * 8), "d2h_bytes_per_step": int(C.N * 8 + 4)},
        "roofline": roof,
    }
    if hbm:
        it = hbm["iteration_kernel"]
        line["fused_iteration"] = {
            kp: {"fused_us": 1e3 * it[kp]["fused"]["ms_per_iteration"], "fused_gbs": it[kp]["fused"]["gbs"],
                 "fused_frac_of_hbm": it[kp]["fused"]["frac_of_hbm"],
                 "plain_us": 1e3 * it[kp]["plain"]["ms_per_iteration"],
                 "fusion_speedup": it[kp]["fusion_speedup"]} for kp in ("fp32", "bf16")}
        line["fused_iteration"]["whole_query_ms"] = {k: v["ms_per_query"] for k, v in hbm["query"].items()
                                                     if isinstance(v, dict)}
    line |= {
        "kernels_ms": {"cost": statistics.mean(cost_ms), "solver": statistics.mean(solve_ms)},
        "gpu_launches": K * (3 if run_path == "resident" else
                             (2 + t * (2 if run_path == "plain" else 1) + 1)),
        "sms": sms, "clocks": clocks, "status": st,
    }
    if hbm:
        line["hbm_regime"] = hbm
    if rank == 0:
        corpus.close()
    if rank == 0 and not args.no_paper:
        line["paper_shaped"] = paper_shaped(swmd, synth, torch, flush, stream, peaks, alu_peak, rank)
    if rank == 0 and not args.no_batch:
        line["batched"] = batched(swmd, synth, torch)
    if rank == 0 and not args.no_serve:
        line["serving"] = serving(swmd, synth, torch, E=E, C=C)
    if rank == 0 and not args.no_cpu_baseline:
        runs, el, cores = time_oracle(E, C, qi, qw, lam, t, budget_s=12.0, max_runs=3)
        line["cpu_baseline"] = {"value": C.N * runs / el, "unit": "WMD/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"{runs} whole queries of the {w.name} workload "
                                          f"({C.N} documents each), sparse FP64 mode"}
        # supplementary oracle timings: a failure here is recorded, not fatal to the line
        for key, fn in (("single_core", lambda: time_oracle_one_core(E, C, qi, qw, lam, t)),
                        ("dense", lambda: time_oracle_dense(synth))):
            try:
                line["cpu_baseline"][key] = fn()
            except Exception as exc:   # noqa: BLE001
                line["cpu_baseline"][key] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
