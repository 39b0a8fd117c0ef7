"""Python binding of libswmd, the GB300 Sinkhorn WMD library (arXiv 2107.06433).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libswmd.so``.  The functions carry the C ABI's names
(``swmd_create_corpus``, ``swmd_query``, ...; see include/swmd.h).  Device
buffers may be passed as torch CUDA tensors or raw integer addresses; streams
as ``torch.cuda.Stream`` objects or raw ``cudaStream_t`` integers.

There is no CPU fallback: if the library has not been built, importing the
native layer raises ``ImportError``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SWMD_DEBUG=1 loads the debug library (build(debug=True): kernels with bounds checks)
LIB_PATH = os.path.join(_HERE, "_build_debug" if os.environ.get("SWMD_DEBUG") == "1" else "_build", "libswmd.so")

SWMD_OK, SWMD_EINVAL, SWMD_ENOMEM, SWMD_ECUDA, SWMD_ETIMEDOUT, SWMD_ENUMERIC, SWMD_ESTOPPED = range(7)
K_FP32, K_BF16, K_FP16 = 0, 1, 2
PATH_FUSED, PATH_PLAIN, PATH_RESIDENT, PATH_AUTO = 0, 1, 2, 3
_KPREC = {"fp32": K_FP32, "bf16": K_BF16, "fp16": K_FP16}
_PATHS = {"fused": PATH_FUSED, "plain": PATH_PLAIN, "resident": PATH_RESIDENT, "auto": PATH_AUTO}
_PATH_NAMES = {v: k for k, v in _PATHS.items()}


class SwmdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"swmd error {code}: {msg}")
        self.code = code


class swmd_options(ctypes.Structure):
    _fields_ = [("k_precision", ctypes.c_int32), ("path", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("column_shift", ctypes.c_int32),
                ("max_vr", ctypes.c_int32), ("device", ctypes.c_int32),
                ("doc_begin", ctypes.c_int32), ("doc_end", ctypes.c_int32),
                ("team_lanes", ctypes.c_int32), ("lanes_per_nz", ctypes.c_int32),
                ("tile_threads", ctypes.c_int32), ("nnz_per_lane", ctypes.c_int32),
                ("tile_nnz", ctypes.c_int32), ("cost_split", ctypes.c_int32),
                ("solver", ctypes.c_int32), ("tol", ctypes.c_float),
                ("queries_per_tile", ctypes.c_int32)]


class swmd_corpus_info(ctypes.Structure):
    _fields_ = [("V", ctypes.c_int32), ("N", ctypes.c_int32), ("d", ctypes.c_int32),
                ("V_used", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("doc_begin", ctypes.c_int32), ("doc_end", ctypes.c_int32),
                ("device", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]


class swmd_serve_config(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("memory_budget", ctypes.c_int64),
                ("max_wait_us", ctypes.c_int32), ("queue_capacity", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class swmd_serve_stats_t(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("qps", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_batch", ctypes.c_double),
                ("batches", ctypes.c_int64)]


class swmd_tune_result(ctypes.Structure):
    _fields_ = [("vrp", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("nnz_per_lane", ctypes.c_int32), ("cost_split", ctypes.c_int32),
                ("default_ms", ctypes.c_float), ("best_ms", ctypes.c_float),
                ("candidates", ctypes.c_int32), ("path", ctypes.c_int32)]


class swmd_batch_tune_result(ctypes.Structure):
    _fields_ = [("layouts", ctypes.c_int32), ("vrp", ctypes.c_int32 * 4),
                ("queries_per_tile", ctypes.c_int32 * 4), ("default_ms", ctypes.c_float),
                ("best_ms", ctypes.c_float), ("candidates", ctypes.c_int32)]


_lib = None

P = ctypes.c_void_p
_SIGS = {
    "swmd_default_options": (None, [P]),
    "swmd_set_allocator": (ctypes.c_int, [P, P, P]),
    "swmd_last_error": (ctypes.c_char_p, []),
    "swmd_select": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, P, P, P, P, P]),
    "swmd_create_corpus": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, P, P, P,
                                          P, ctypes.c_int32, P, P]),
    "swmd_destroy_corpus": (None, [P]),
    "swmd_corpus_get_info": (ctypes.c_int, [P, P]),
    "swmd_corpus_set_options": (ctypes.c_int, [P, P]),
    "swmd_corpus_get_options": (ctypes.c_int, [P, P]),
    "swmd_query": (ctypes.c_int, [P, P, P, ctypes.c_int32, ctypes.c_float, ctypes.c_int32, P]),
    "swmd_query_device": (ctypes.c_int, [P, P, P, ctypes.c_int32, ctypes.c_float, ctypes.c_int32,
                                         P, P, P]),
    "swmd_step_cost": (ctypes.c_int, [P, P, P, ctypes.c_int32, ctypes.c_float, P, P]),
    "swmd_step_iterate": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, P]),
    "swmd_step_final": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, P, P]),
    "swmd_step_resident": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, P, P]),
    "swmd_get_mapping": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, P]),
    "swmd_partition_documents": (ctypes.c_int, [ctypes.c_int32, P, ctypes.c_int32, P]),
    "swmd_query_noalloc": (ctypes.c_int, [P, P, P, ctypes.c_int32, ctypes.c_float, ctypes.c_int32,
                                          P, P, P]),
    "swmd_debug_plant": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32]),
    "swmd_debug_read": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, P]),
    "swmd_query_batch": (ctypes.c_int, [P, ctypes.c_int32, P, P, P, P, ctypes.c_int32, P]),
    "swmd_autotune": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, P]),
    "swmd_autotune_batch": (ctypes.c_int, [P, ctypes.c_int32, P, P, P, P, ctypes.c_int32,
                                           ctypes.c_int32, P]),
    "swmd_resolve_path": (ctypes.c_int, [P, ctypes.c_int32, P]),
    "swmd_last_iterations": (ctypes.c_int, [P, P]),
    "swmd_wmd_pairs": (ctypes.c_int, [P, ctypes.c_int32, P, P, P, P, P, P, ctypes.c_float,
                                      ctypes.c_int32, ctypes.c_float, P, P]),
    "swmd_wmd_pairs_device": (ctypes.c_int, [P, ctypes.c_int32, P, P, P, P, P, P, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_float, ctypes.c_int32,
                                             ctypes.c_float, P, P, P, P]),
    "swmd_default_serve_config": (None, [P]),
    "swmd_serve_start": (ctypes.c_int, [P, P, P]),
    "swmd_serve_submit": (ctypes.c_int, [P, P, P, ctypes.c_int32, ctypes.c_float, ctypes.c_int32,
                                         P]),
    "swmd_serve_wait": (ctypes.c_int, [P, ctypes.c_uint64, P, ctypes.c_int32]),
    "swmd_serve_stats": (ctypes.c_int, [P, P]),
    "swmd_serve_stop": (ctypes.c_int, [P]),
}


def lib() -> ctypes.CDLL:
    """The loaded libswmd.so (ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _err(code: int, what: str):
    if code != SWMD_OK:
        msg = lib().swmd_last_error()
        raise SwmdError(code, f"{what}: {msg.decode() if msg else ''}")


def _np(a, dt):
    a = np.ascontiguousarray(a, dtype=dt)
    return a, a.ctypes.data_as(P)


def _dptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return P(x)
    return P(x.data_ptr())


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return P(s)
    return P(s.cuda_stream)


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_void_p,
                             ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_void_p,
                            ctypes.c_void_p)
_allocator_refs = None   # keeps the C callbacks alive while the library may call them


def swmd_set_allocator(alloc=None, release=None):
    """Device memory of corpora created from now on: alloc(bytes, device, stream) -> int
    pointer (0 on failure) and release(ptr, bytes, device, stream), Python callables;
    both None restores cudaMalloc / cudaFree."""
    global _allocator_refs
    if alloc is None and release is None:
        _err(lib().swmd_set_allocator(None, None, None), "swmd_set_allocator")
        _allocator_refs = None
        return

    def c_alloc(nbytes, device, stream, user):
        return int(alloc(int(nbytes), int(device), stream or 0)) or None

    def c_free(ptr, nbytes, device, stream, user):
        release(int(ptr), int(nbytes), int(device), stream or 0)

    refs = (_ALLOC_FN(c_alloc), _FREE_FN(c_free)) if alloc is not None and release is not None else \
        (_ALLOC_FN(c_alloc) if alloc is not None else None, _FREE_FN(c_free) if release is not None else None)
    _err(lib().swmd_set_allocator(ctypes.cast(refs[0], P) if refs[0] else None,
                                  ctypes.cast(refs[1], P) if refs[1] else None, None), "swmd_set_allocator")
    _allocator_refs = refs


def use_torch_allocator():
    """Routes the library's device memory (corpora created from now on) through
    PyTorch's caching allocator."""
    import torch

    def alloc(nbytes, device, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, device, stream)

    def release(ptr, nbytes, device, stream):
        torch.cuda.caching_allocator_delete(ptr)

    swmd_set_allocator(alloc, release)


def swmd_default_options(**kw) -> swmd_options:
    o = swmd_options()
    lib().swmd_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "k_precision" and isinstance(v, str):
            v = _KPREC[v]
        if k == "path" and isinstance(v, str):
            v = _PATHS[v]
        setattr(o, k, float(v) if k == "tol" else int(v))
    return o


def swmd_select(V, ids, weights):
    ids, pi = _np(ids, np.int32)
    w, pw = _np(weights, np.float32)
    n = len(ids)
    out_ids = np.empty(max(n, 1), np.int32)
    out_r = np.empty(max(n, 1), np.float32)
    vr = ctypes.c_int32(0)
    _err(lib().swmd_select(V, n, pi, pw, out_ids.ctypes.data_as(P), out_r.ctypes.data_as(P),
                           ctypes.byref(vr)), "swmd_select")
    return out_ids[:vr.value].copy(), out_r[:vr.value].copy()


def swmd_partition_documents(N, doc_nnz, parts):
    """Contiguous document ranges for `parts` GPUs, balanced by nonzeros: int32[parts+1]."""
    cnt, pc = _np(doc_nnz, np.int64)
    out = np.empty(int(parts) + 1, np.int32)
    _err(lib().swmd_partition_documents(int(N), pc, int(parts), out.ctypes.data_as(P)),
         "swmd_partition_documents")
    return out


class Corpus:
    """Owns a swmd_corpus*; destroyed with the object."""

    def __init__(self, handle, N):
        self._h = handle
        self.N = N

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().swmd_destroy_corpus(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> swmd_corpus_info:
        return swmd_corpus_get_info(self)


def swmd_create_corpus(V, N, row_ptr, doc_idx, val, emb, opt: swmd_options | None = None,
                       **kw) -> Corpus:
    """c as V x N CSR (row_ptr int64[V+1], doc_idx int32[nnz], val float32[nnz]); emb [V, d]."""
    rp, prp = _np(row_ptr, np.int64)
    di, pdi = _np(doc_idx, np.int32)
    vv, pvv = _np(val, np.float32)
    E, pE = _np(emb, np.float32)
    assert E.ndim == 2 and E.shape[0] == V
    if opt is None:
        opt = swmd_default_options(**kw)
    h = P()
    _err(lib().swmd_create_corpus(V, N, int(rp[-1]), prp, pdi, pvv, pE, E.shape[1],
                                  ctypes.byref(opt), ctypes.byref(h)), "swmd_create_corpus")
    b = opt.doc_begin if opt.doc_begin >= 0 else 0
    e = opt.doc_end if opt.doc_end >= 0 else N
    return Corpus(h, e - b)


def swmd_destroy_corpus(corpus: Corpus):
    corpus.close()


def swmd_corpus_get_info(corpus: Corpus) -> swmd_corpus_info:
    info = swmd_corpus_info()
    _err(lib().swmd_corpus_get_info(corpus.handle, ctypes.byref(info)), "swmd_corpus_get_info")
    return info


def swmd_corpus_get_options(corpus: Corpus) -> swmd_options:
    o = swmd_options()
    _err(lib().swmd_corpus_get_options(corpus.handle, ctypes.byref(o)), "swmd_corpus_get_options")
    return o


def swmd_corpus_set_options(corpus: Corpus, opt: swmd_options | None = None, **kw):
    """Sets the corpus's options: `opt` whole, or the fields named in `kw` on top of
    the current ones."""
    if opt is None:
        opt = swmd_corpus_get_options(corpus)
        for k, v in kw.items():
            if k == "k_precision" and isinstance(v, str):
                v = _KPREC[v]
            if k == "path" and isinstance(v, str):
                v = _PATHS[v]
            setattr(opt, k, float(v) if k == "tol" else int(v))
    _err(lib().swmd_corpus_set_options(corpus.handle, ctypes.byref(opt)), "swmd_corpus_set_options")


def swmd_query(corpus: Corpus, ids, weights, lam: float, max_iter: int, out=None) -> np.ndarray:
    """Distances (float64[N]) of the query to every document; host in, host out."""
    ids, pi = _np(ids, np.int32)
    w, pw = _np(weights, np.float32)
    if out is None:
        out = np.empty(corpus.N, np.float64)
    _err(lib().swmd_query(corpus.handle, pi, pw, len(ids), float(lam), int(max_iter),
                          out.ctypes.data_as(P)), "swmd_query")
    return out


def swmd_query_device(corpus: Corpus, d_ids, d_r, v_r: int, lam: float, max_iter: int, d_out,
                      d_status=None, stream=None):
    _err(lib().swmd_query_device(corpus.handle, _dptr(d_ids), _dptr(d_r), int(v_r), float(lam),
                                 int(max_iter), _dptr(d_out), _dptr(d_status), _stream(stream)),
         "swmd_query_device")


def swmd_query_noalloc(corpus: Corpus, d_ids, d_r, v_r: int, lam: float, max_iter: int, d_out,
                       d_status=None, stream=None):
    """swmd_query_device without any allocation in the call: the scratch lives in a
    fixed 16 MiB device array inside the library (see include/swmd.h)."""
    _err(lib().swmd_query_noalloc(corpus.handle, _dptr(d_ids), _dptr(d_r), int(v_r), float(lam),
                                  int(max_iter), _dptr(d_out), _dptr(d_status), _stream(stream)),
         "swmd_query_noalloc")


def swmd_step_cost(corpus: Corpus, d_ids, d_r, v_r, lam, d_status=None, stream=None):
    _err(lib().swmd_step_cost(corpus.handle, _dptr(d_ids), _dptr(d_r), int(v_r), float(lam),
                              _dptr(d_status), _stream(stream)), "swmd_step_cost")


def swmd_step_iterate(corpus: Corpus, v_r, n_iter, first, path="fused", stream=None):
    path = _PATHS[path] if isinstance(path, str) else int(path)
    _err(lib().swmd_step_iterate(corpus.handle, int(v_r), int(n_iter), int(first), path,
                                 _stream(stream)), "swmd_step_iterate")


def swmd_step_final(corpus: Corpus, v_r, t0, d_out, stream=None):
    _err(lib().swmd_step_final(corpus.handle, int(v_r), int(t0), _dptr(d_out), _stream(stream)),
         "swmd_step_final")


def swmd_step_resident(corpus: Corpus, v_r, max_iter, d_out, stream=None):
    _err(lib().swmd_step_resident(corpus.handle, int(v_r), int(max_iter), _dptr(d_out),
                                  _stream(stream)), "swmd_step_resident")


def swmd_get_mapping(corpus: Corpus, v_r: int, path="resident"):
    """(VRP, lanes per nonzero Q, nonzeros in flight per document P)."""
    path = _PATHS[path] if isinstance(path, str) else int(path)
    out = (ctypes.c_int32 * 3)()
    _err(lib().swmd_get_mapping(corpus.handle, int(v_r), path, out), "swmd_get_mapping")
    return int(out[0]), int(out[1]), int(out[2])


def swmd_last_iterations(corpus: Corpus) -> int:
    """x-updates the corpus's last single query applied (max_iter, or fewer under tol)."""
    out = ctypes.c_int32()
    _err(lib().swmd_last_iterations(corpus.handle, ctypes.byref(out)), "swmd_last_iterations")
    return out.value


def swmd_resolve_path(corpus: Corpus, v_r: int) -> str:
    """The path ("resident", "fused" or "plain") a query of v_r words takes."""
    out = ctypes.c_int32()
    _err(lib().swmd_resolve_path(corpus.handle, int(v_r), ctypes.byref(out)), "swmd_resolve_path")
    return _PATH_NAMES[out.value]


def swmd_debug_plant(corpus: Corpus, what: str, index: int, value: int):
    """Debug builds: overwrite the word id of one nonzero ("nz": document-major copy,
    "slices": the sliced copy) to test the kernels' bounds checks."""
    _err(lib().swmd_debug_plant(corpus.handle, {"nz": 0, "slices": 1}[what], int(index), int(value)),
         "swmd_debug_plant")


def swmd_debug_read(corpus: Corpus, what: str, v_r: int = 0) -> np.ndarray:
    info = corpus.info()
    code = {"KT": 0, "KMT": 1, "u": 2, "used": 3}[what]
    if code == 3:
        out = np.empty(info.V_used, np.int32)
    elif code == 2:
        out = np.empty((corpus.N, v_r), np.float32)
    else:
        out = np.empty((info.V_used, v_r), np.float32)
    _err(lib().swmd_debug_read(corpus.handle, code, int(v_r), out.ctypes.data_as(P)),
         "swmd_debug_read")
    return out


def _batch_arrays(queries, lambdas):
    n = len(queries)
    q_ptr = np.zeros(n + 1, np.int64)
    for i, (qi, _) in enumerate(queries):
        q_ptr[i + 1] = q_ptr[i] + len(qi)
    ids = np.concatenate([np.asarray(q[0], np.int32) for q in queries]) if n else np.zeros(0, np.int32)
    ws = np.concatenate([np.asarray(q[1], np.float32) for q in queries]) if n else np.zeros(0, np.float32)
    lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lambdas, np.float32), (n,)), np.float32)
    return n, q_ptr, np.ascontiguousarray(ids, np.int32), np.ascontiguousarray(ws, np.float32), lam


def swmd_query_batch(corpus: Corpus, queries, lambdas, max_iter: int) -> np.ndarray:
    """queries: list of (ids, weights).  Returns float64[n_queries, N]."""
    n, q_ptr, ids, ws, lam = _batch_arrays(queries, lambdas)
    out = np.empty((n, corpus.N), np.float64)
    _err(lib().swmd_query_batch(corpus.handle, n, q_ptr.ctypes.data_as(P), ids.ctypes.data_as(P),
                                ws.ctypes.data_as(P), lam.ctypes.data_as(P), int(max_iter),
                                out.ctypes.data_as(P)), "swmd_query_batch")
    return out


def swmd_autotune_batch(corpus: Corpus, queries, lambdas, max_iter: int, reps: int = 2) -> dict:
    """Times swmd_query_batch on this batch for every queries-per-tile candidate of its
    column-split layouts and keeps the fastest.  Returns the chosen tile sizes."""
    n, q_ptr, ids, ws, lam = _batch_arrays(queries, lambdas)
    res = swmd_batch_tune_result()
    _err(lib().swmd_autotune_batch(corpus.handle, n, q_ptr.ctypes.data_as(P), ids.ctypes.data_as(P),
                                   ws.ctypes.data_as(P), lam.ctypes.data_as(P), int(max_iter),
                                   int(reps), ctypes.byref(res)), "swmd_autotune_batch")
    k = res.layouts
    return {"layouts": k, "vrp": list(res.vrp)[:k], "queries_per_tile": list(res.queries_per_tile)[:k],
            "default_ms": res.default_ms, "best_ms": res.best_ms, "candidates": res.candidates}


def swmd_autotune(corpus: Corpus, v_r: int, reps: int = 5) -> dict:
    """Times the resident path's candidate mappings for queries of v_r words on this
    corpus and keeps the fastest for that layout.  Returns the chosen settings."""
    res = swmd_tune_result()
    _err(lib().swmd_autotune(corpus.handle, int(v_r), int(reps), ctypes.byref(res)),
         "swmd_autotune")
    return {f: getattr(res, f) for f, _ in swmd_tune_result._fields_}


def _ragged(sides):
    """[(ids, weights), ...] -> (ptr int64[n+1], ids int32, weights float32)."""
    ptr = np.zeros(len(sides) + 1, np.int64)
    for i, (ids, _) in enumerate(sides):
        ptr[i + 1] = ptr[i] + len(ids)
    if sides:
        ids = np.concatenate([np.asarray(s[0], np.int32).ravel() for s in sides])
        w = np.concatenate([np.asarray(s[1], np.float32).ravel() for s in sides])
    else:
        ids, w = np.zeros(0, np.int32), np.zeros(0, np.float32)
    return ptr, np.ascontiguousarray(ids), np.ascontiguousarray(w)


def swmd_wmd_pairs(corpus: Corpus, queries, targets, lam: float, max_iter: int, tol: float = 0.0,
                   want_iters: bool = False):
    """1-to-1 WMD (Table II): distance of queries[p] to targets[p], each an (ids, weights)
    histogram over the corpus's vocabulary.  Returns float64[n] (and int32[n] x-updates)."""
    if len(queries) != len(targets):
        raise ValueError("swmd_wmd_pairs: as many queries as targets")
    n = len(queries)
    qp, qi, qw = _ragged(queries)
    xp, xi, xw = _ragged(targets)
    out = np.empty(n, np.float64)
    its = np.empty(n, np.int32)
    _err(lib().swmd_wmd_pairs(corpus.handle, n, qp.ctypes.data_as(P), qi.ctypes.data_as(P),
                              qw.ctypes.data_as(P), xp.ctypes.data_as(P), xi.ctypes.data_as(P),
                              xw.ctypes.data_as(P), float(lam), int(max_iter), float(tol),
                              out.ctypes.data_as(P), its.ctypes.data_as(P)), "swmd_wmd_pairs")
    return (out, its) if want_iters else out


def swmd_wmd_pairs_device(corpus: Corpus, n_pairs: int, d_q_ptr, d_q_ids, d_r, d_x_ptr, d_x_ids,
                          d_c, max_q_words: int, max_x_words: int, lam: float, max_iter: int,
                          d_out, d_status, tol: float = 0.0, d_iters=None, stream=None):
    """swmd_wmd_pairs on selected, normalised sides already in device memory."""
    _err(lib().swmd_wmd_pairs_device(corpus.handle, int(n_pairs), _dptr(d_q_ptr), _dptr(d_q_ids),
                                     _dptr(d_r), _dptr(d_x_ptr), _dptr(d_x_ids), _dptr(d_c),
                                     int(max_q_words), int(max_x_words), float(lam),
                                     int(max_iter), float(tol), _dptr(d_out), _dptr(d_iters),
                                     _dptr(d_status), _stream(stream)), "swmd_wmd_pairs_device")


class Server:
    def __init__(self, handle, corpus: Corpus):
        self._h = handle
        self.corpus = corpus     # keeps the corpus alive while serving

    @property
    def handle(self):
        return self._h

    def stop(self):
        if self._h:
            _err(lib().swmd_serve_stop(self._h), "swmd_serve_stop")
            self._h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def swmd_default_serve_config(**kw) -> swmd_serve_config:
    cfg = swmd_serve_config()
    lib().swmd_default_serve_config(ctypes.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, k, int(v))
    return cfg


def swmd_serve_start(corpus: Corpus, cfg: swmd_serve_config | None = None, **kw) -> Server:
    if cfg is None:
        cfg = swmd_default_serve_config(**kw)
    h = P()
    _err(lib().swmd_serve_start(corpus.handle, ctypes.byref(cfg), ctypes.byref(h)),
         "swmd_serve_start")
    return Server(h, corpus)


def swmd_serve_submit(srv: Server, ids, weights, lam: float, max_iter: int) -> int:
    ids, pi = _np(ids, np.int32)
    w, pw = _np(weights, np.float32)
    t = ctypes.c_uint64(0)
    _err(lib().swmd_serve_submit(srv.handle, pi, pw, len(ids), float(lam), int(max_iter),
                                 ctypes.byref(t)), "swmd_serve_submit")
    return t.value


def swmd_serve_wait(srv: Server, ticket: int, timeout_ms: int = -1) -> np.ndarray:
    out = np.empty(srv.corpus.N, np.float64)
    _err(lib().swmd_serve_wait(srv.handle, ctypes.c_uint64(ticket), out.ctypes.data_as(P),
                               int(timeout_ms)), "swmd_serve_wait")
    return out


def swmd_serve_stats(srv: Server) -> dict:
    s = swmd_serve_stats_t()
    _err(lib().swmd_serve_stats(srv.handle, ctypes.byref(s)), "swmd_serve_stats")
    return {k: getattr(s, k) for k, _ in s._fields_}


def swmd_serve_stop(srv: Server):
    srv.stop()


def corpus_from_synth(E, C, **kw) -> Corpus:
    """Convenience: a corpus from paper_2107_06433_gb300.synth outputs."""
    rp, col, val = C.csr()
    return swmd_create_corpus(C.V, C.N, rp, col, val, E, **kw)
