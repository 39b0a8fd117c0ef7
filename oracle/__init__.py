"""FP64 CPU oracle of Sinkhorn WMD (arXiv 2107.06433, Algorithm 1; Algorithms 2-3;
the 1-to-1 variant of Section III-E, Table II).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA product path never
imports, links or calls it, and the two share no code.

The arithmetic lives in ``swmd_oracle.c`` (plain C, FP64, OpenMP over independent
outputs); this module compiles it with gcc on first use and marshals numpy
arrays through ctypes.  ``build()`` compiles it eagerly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swmd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

EINVAL = -1
ENOMEM = -2


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, -O2, OpenMP, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.oracle_select.argtypes = [i64, i64, P, P, P, P]
        lib.oracle_select.restype = i64
        lib.oracle_cdist.argtypes = [i64, i32, P, i32, P, P]
        lib.oracle_cdist.restype = None
        lib.oracle_kernel.argtypes = [i64, P, f64, P, P]
        lib.oracle_kernel.restype = None
        lib.oracle_normalize_columns.argtypes = [i64, i64, P, P, P, P]
        lib.oracle_normalize_columns.restype = ctypes.c_int
        lib.oracle_sinkhorn_dense.argtypes = [i32, i64, i64, P, P, P, P, P, P, i32, i64, P, P]
        lib.oracle_sinkhorn_dense.restype = ctypes.c_int
        lib.oracle_sinkhorn_sparse.argtypes = [i32, i64, i64, P, P, P, P, P, P, i32, P, P, P, P]
        lib.oracle_sinkhorn_sparse.restype = ctypes.c_int
        lib.oracle_sinkhorn_converge.argtypes = [i32, i64, i64, P, P, P, P, P, P, i32, f64, P, P,
                                                 P, P]
        lib.oracle_sinkhorn_converge.restype = ctypes.c_int
        lib.oracle_wmd.argtypes = [i64, i32, P, i64, P, P, P, i64, P, P, f64, i32, i32, P]
        lib.oracle_wmd.restype = ctypes.c_int
        lib.oracle_wmd_pairs.argtypes = [i64, i32, P, i64, P, P, P, P, P, P, f64, i32, f64, P, P]
        lib.oracle_wmd_pairs.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        lib.oracle_get_threads.argtypes = []
        lib.oracle_get_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what}: oracle returned {rc}")


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def select(V, ids, weights):
    """(ids int32[v_r] ascending, r float64[v_r] summing to 1)."""
    ids = _c(ids, np.int32)
    w = _c(weights, np.float64)
    out_ids = np.empty(max(len(ids), 1), np.int32)
    out_r = np.empty(max(len(ids), 1), np.float64)
    vr = _load().oracle_select(V, len(ids), _p(ids), _p(w), _p(out_ids), _p(out_r))
    if vr <= 0:
        raise OracleError(f"select: oracle returned {vr}")
    return out_ids[:vr].copy(), out_r[:vr].copy()


def cdist(E, q):
    """M [v_r, V] float64: Euclidean distances from rows E[q] to every row of E."""
    E = _c(E, np.float32)
    q = _c(q, np.int32)
    V, d = E.shape
    M = np.empty((len(q), V), np.float64)
    _load().oracle_cdist(V, d, _p(E), len(q), _p(q), _p(M))
    return M


def kernel(M, lam):
    """(K, KM) = (exp(-lam M), K * M)."""
    M = _c(M, np.float64)
    K = np.empty_like(M)
    KM = np.empty_like(M)
    _load().oracle_kernel(M.size, _p(M), float(lam), _p(K), _p(KM))
    return K, KM


def normalize_columns(V, N, row_ptr, col, val):
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    val = _c(val, np.float64)
    out = np.empty_like(val)
    _check(_load().oracle_normalize_columns(V, N, _p(row_ptr), _p(col), _p(val), _p(out)),
           "normalize_columns")
    return out


def sinkhorn_dense(K, KM, r, N, row_ptr, col, cval, t, nb=64, want_x=False):
    K = _c(K, np.float64)
    KM = _c(KM, np.float64)
    r = _c(r, np.float64)
    vr, V = K.shape
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    cval = _c(cval, np.float64)
    wmd = np.empty(N, np.float64)
    x = np.empty((N, vr), np.float64) if want_x else None
    _check(_load().oracle_sinkhorn_dense(vr, V, N, _p(K), _p(KM), _p(r), _p(row_ptr), _p(col),
                                         _p(cval), int(t), int(nb), _p(wmd), _p(x)),
           "sinkhorn_dense")
    return (wmd, x) if want_x else wmd


def sinkhorn_sparse(K, KM, r, N, row_ptr, col, cval, t, want_state=False):
    """WMD [N]; with want_state also (x [N,v_r], u [N,v_r], v [nnz] in CSR order)."""
    K = _c(K, np.float64)
    KM = _c(KM, np.float64)
    r = _c(r, np.float64)
    vr, V = K.shape
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    cval = _c(cval, np.float64)
    wmd = np.empty(N, np.float64)
    x = u = v = None
    if want_state:
        x = np.empty((N, vr), np.float64)
        u = np.empty((N, vr), np.float64)
        v = np.empty(len(cval), np.float64)
    _check(_load().oracle_sinkhorn_sparse(vr, V, N, _p(K), _p(KM), _p(r), _p(row_ptr), _p(col),
                                          _p(cval), int(t), _p(wmd), _p(x), _p(u), _p(v)),
           "sinkhorn_sparse")
    return (wmd, x, u, v) if want_state else wmd


def sinkhorn_converge(K, KM, r, N, row_ptr, col, cval, tol, max_iter=100000):
    """(WMD [N], iterations, u [N,v_r], v [nnz]) iterating until row sums are within tol of r."""
    K = _c(K, np.float64)
    KM = _c(KM, np.float64)
    r = _c(r, np.float64)
    vr, V = K.shape
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    cval = _c(cval, np.float64)
    wmd = np.empty(N, np.float64)
    u = np.empty((N, vr), np.float64)
    v = np.empty(len(cval), np.float64)
    it = ctypes.c_int32(0)
    _check(_load().oracle_sinkhorn_converge(vr, V, N, _p(K), _p(KM), _p(r), _p(row_ptr), _p(col),
                                            _p(cval), int(max_iter), float(tol),
                                            ctypes.byref(it), _p(wmd), _p(u), _p(v)),
           "sinkhorn_converge")
    return wmd, int(it.value), u, v


def wmd(E, row_ptr, col, cval, N, q_ids, q_w, lam, t, mode="sparse"):
    """The whole problem statement: WMD [N] of the query against every column of c."""
    E = _c(E, np.float32)
    V, d = E.shape
    row_ptr = _c(row_ptr, np.int64)
    col = _c(col, np.int32)
    cval = _c(cval, np.float32)
    q_ids = _c(q_ids, np.int32)
    q_w = _c(q_w, np.float32)
    out = np.empty(N, np.float64)
    m = {"sparse": 0, "dense": 1}[mode]
    _check(_load().oracle_wmd(V, d, _p(E), N, _p(row_ptr), _p(col), _p(cval), len(q_ids),
                              _p(q_ids), _p(q_w), float(lam), int(t), m, _p(out)), "wmd")
    return out


def _ragged(sides):
    """[(ids, weights), ...] -> (ptr int64, ids int32, weights float32)."""
    ptr = np.zeros(len(sides) + 1, np.int64)
    for i, (ids, _) in enumerate(sides):
        ptr[i + 1] = ptr[i] + len(ids)
    ids = np.concatenate([np.asarray(s[0], np.int32) for s in sides]) if sides else np.zeros(0, np.int32)
    w = np.concatenate([np.asarray(s[1], np.float32) for s in sides]) if sides else np.zeros(0, np.float32)
    return ptr, _c(ids, np.int32), _c(w, np.float32)


def wmd_pairs(E, queries, targets, lam, t, tol=0.0, want_iters=False):
    """1-to-1 WMD (Section III-E, Table II): the distance of queries[p] to targets[p],
    each an (ids, weights) histogram, with the cost built over the target's words only.
    tol > 0 runs the convergence mode with t as the cap."""
    if len(queries) != len(targets):
        raise ValueError("wmd_pairs: as many queries as targets")
    E = _c(E, np.float32)
    V, d = E.shape
    qp, qi, qw = _ragged(queries)
    xp, xi, xw = _ragged(targets)
    n = len(queries)
    out = np.empty(n, np.float64)
    its = np.empty(n, np.int32)
    _check(_load().oracle_wmd_pairs(V, d, _p(E), n, _p(qp), _p(qi), _p(qw), _p(xp), _p(xi),
                                    _p(xw), float(lam), int(t), float(tol), _p(out), _p(its)),
           "wmd_pairs")
    return (out, its) if want_iters else out
