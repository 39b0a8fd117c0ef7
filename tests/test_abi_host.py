"""CPU-only checks of the C ABI library: it loads, exports every declared symbol,
and its host-side logic (query selection, argument validation, defaults)
behaves as documented.  No call here reaches a GPU."""
import os
import re
import subprocess

import ctypes

import numpy as np
import pytest

import paper_2107_06433_gb300 as swmd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swmd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2107_06433_gb300 import build
    build.build()
    return swmd.lib()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SWMD_API\s+[\w\s\*]*?\b(swmd_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("swmd_create_corpus", "swmd_destroy_corpus", "swmd_query",
                     "swmd_query_batch", "swmd_serve_start", "swmd_serve_submit",
                     "swmd_serve_wait", "swmd_serve_stats", "swmd_serve_stop", "swmd_last_error",
                     "swmd_autotune", "swmd_query_noalloc", "swmd_wmd_pairs",
                     "swmd_wmd_pairs_device"):
        assert required in names


def test_binding_covers_every_declared_function():
    missing = [n for n in declared_functions() if n not in swmd._SIGS]
    assert not missing, missing


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", swmd.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # nothing but the ABI is exported
    extra = sorted(n for n in exported if not n.startswith("swmd_") and not n.startswith("_"))
    assert not extra, extra
    for n in declared_functions():
        assert hasattr(lib, n)


def test_default_options(lib):
    o = swmd.swmd_default_options()
    assert (o.k_precision, o.path, o.use_graph, o.column_shift, o.max_vr, o.device) == \
        (swmd.K_FP32, swmd.PATH_AUTO, 1, 1, 128, -1)
    cfg = swmd.swmd_default_serve_config()
    assert cfg.max_batch == 32 and cfg.memory_budget == 4 << 30


def test_select_merges_duplicates_and_normalises(lib):
    ids, r = swmd.swmd_select(10, [7, 3, 7, 5, 1], [1.0, 2.0, 3.0, 0.0, 2.0])
    assert ids.tolist() == [1, 3, 7]
    np.testing.assert_allclose(r, [0.25, 0.25, 0.5], rtol=1e-7)


def test_select_matches_oracle_selection(lib):
    import oracle
    rng = np.random.default_rng(3)
    ids = rng.integers(0, 50, size=40)
    w = rng.integers(0, 4, size=40).astype(np.float32)
    a_ids, a_r = swmd.swmd_select(50, ids, w)
    b_ids, b_r = oracle.select(50, ids, w)
    np.testing.assert_array_equal(a_ids, b_ids)
    np.testing.assert_allclose(a_r, b_r, rtol=1e-7)


@pytest.mark.parametrize("ids,w", [([10], [1.0]), ([-1], [1.0]), ([2], [-1.0]),
                                   ([2], [float("nan")]), ([2], [float("inf")]), ([2], [0.0]),
                                   ([], [])])
def test_select_rejects(lib, ids, w):
    with pytest.raises(swmd.SwmdError) as e:
        swmd.swmd_select(10, ids, w)
    assert e.value.code == swmd.SWMD_EINVAL


def _tiny_csr():
    # 4 words, 2 documents
    row_ptr = np.array([0, 1, 2, 3, 4], np.int64)
    doc_idx = np.array([0, 1, 0, 1], np.int32)
    val = np.array([1, 2, 3, 4], np.float32)
    E = np.eye(4, dtype=np.float32)
    return row_ptr, doc_idx, val, E


@pytest.mark.parametrize("mutate,expect", [
    (lambda rp, di, v: (rp, np.array([0, 1, 0, 2], np.int32), v), "outside"),     # doc 2 >= N
    (lambda rp, di, v: (rp, di, np.array([1, 0, 3, 4], np.float32)), "finite and > 0"),
    (lambda rp, di, v: (rp, di, np.array([1, np.nan, 3, 4], np.float32)), "finite and > 0"),
    (lambda rp, di, v: (np.array([0, 2, 1, 3, 4], np.int64), di, v), "decreases"),
    (lambda rp, di, v: (rp, np.array([0, 0, 0, 0], np.int32), v), "no words"),   # doc 1 empty
])
def test_create_corpus_validates_before_touching_the_gpu(lib, mutate, expect):
    rp, di, v, E = _tiny_csr()
    rp, di, v = mutate(rp, di, v)
    with pytest.raises(swmd.SwmdError) as e:
        swmd.swmd_create_corpus(4, 2, rp, di, v, E)
    assert e.value.code == swmd.SWMD_EINVAL
    assert expect in str(e.value)


def test_create_corpus_argument_checks(lib):
    rp, di, v, E = _tiny_csr()
    with pytest.raises(swmd.SwmdError):
        swmd.swmd_create_corpus(4, 2, rp, di, v, E, max_vr=500)
    with pytest.raises(swmd.SwmdError):
        swmd.swmd_create_corpus(4, 2, rp, di, v, E, doc_begin=2, doc_end=1)


def test_options_marshalling(lib):
    o = swmd.swmd_default_options(path="fused", k_precision="bf16", tol=1e-6, cost_split=1)
    assert (o.path, o.k_precision, o.cost_split) == (swmd.PATH_FUSED, swmd.K_BF16, 1)
    assert abs(o.tol - 1e-6) < 1e-12
    assert swmd.swmd_default_options().tol == 0.0


def test_pair_calls_check_arguments_before_the_gpu(lib):
    """The 1-to-1 entry points refuse a NULL corpus and a negative pair count
    without a CUDA call."""
    z = ctypes.c_void_p()
    assert lib.swmd_wmd_pairs(None, 1, z, z, z, z, z, z, 1.0, 15, 0.0, z, z) == swmd.SWMD_EINVAL
    assert b"NULL corpus" in lib.swmd_last_error()
    assert lib.swmd_wmd_pairs_device(None, 1, z, z, z, z, z, z, 8, 8, 1.0, 15, 0.0, z, z, z,
                                     None) == swmd.SWMD_EINVAL


def test_pair_binding_marshals_ragged_sides(lib):
    """The binding's ragged packing of pair sides (pointer arrays and concatenated
    ids / weights), and its length check, need no GPU."""
    ptr, ids, w = swmd._ragged([([3, 1], [1.0, 2.0]), ([7], [5.0]), ([], [])])
    np.testing.assert_array_equal(ptr, [0, 2, 3, 3])
    np.testing.assert_array_equal(ids, [3, 1, 7])
    np.testing.assert_array_equal(w, np.array([1.0, 2.0, 5.0], np.float32))
    assert ids.dtype == np.int32 and w.dtype == np.float32 and ptr.dtype == np.int64
    with pytest.raises(ValueError):
        swmd.swmd_wmd_pairs(None, [([1], [1.0])], [], 1.0, 15)


def test_allocator_needs_both_functions(lib):
    fn = swmd._ALLOC_FN(lambda n, d, s, u: None)
    rc = lib.swmd_set_allocator(ctypes.cast(fn, ctypes.c_void_p), None, None)
    assert rc == swmd.SWMD_EINVAL and b"both" in lib.swmd_last_error()
    assert lib.swmd_set_allocator(None, None, None) == swmd.SWMD_OK
