"""Builds libswmd.so in-tree for sm_103a (GB300) with nvcc.

Each .cu translation unit is compiled in parallel to an object file, then the
objects are linked into one shared library (CUDA runtime linked statically, only
the swmd_* C ABI exported).  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libswmd.so")
# The debug library: the translation units whose kernels follow corpus indices (and
# the C ABI layer, for its debug-only hook) compiled with SWMD_DEBUG_CHECKS=1, linked
# with the release objects of the rest.
DEBUG_BUILD = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_BUILD, "libswmd.so")
DEBUG_SOURCES = ("api.cu", "resident_cols.cu", "resident_cols_long.cu", "walk_fused.cu", "walk_final.cu", "walk_plain.cu")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libswmd")
    return cand


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, debug: bool = False) -> str:
    """Builds libswmd.so (debug=True: the debug library, DEBUG_LIB) and returns its path."""
    if debug:
        build(force, jobs, verbose)   # the release objects it links with
    out_dir = DEBUG_BUILD if debug else BUILD
    os.makedirs(os.path.join(out_dir, "obj"), exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = _headers()
    objs = []
    todo = []
    for src in sources:
        name = os.path.basename(src)
        own = not debug or name in DEBUG_SOURCES
        obj = os.path.join(out_dir if own else BUILD, "obj", name + ".o")
        objs.append(obj)
        if own and (force or _stale(obj, [src] + headers + [__file__])):
            todo.append((src, obj))
    cc = nvcc()
    extra = ["-DSWMD_DEBUG_CHECKS=1"] if debug else []

    def compile_one(item):
        src, obj = item
        tmp = obj + ".%d.tmp" % os.getpid()
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", tmp]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (os.path.basename(src), p.stderr[-6000:]))
        os.replace(tmp, obj)
        return p.stderr

    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 4)
        with cf.ThreadPoolExecutor(n) as ex:
            for log in ex.map(compile_one, todo):
                if verbose and log:
                    print(log)
    lib = DEBUG_LIB if debug else LIB
    if force or todo or _stale(lib, objs):
        tmp = lib + ".%d.tmp" % os.getpid()
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fvisibility=hidden",
               "-lpthread", "-Xlinker", "--no-undefined"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n" + p.stderr[-6000:])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
