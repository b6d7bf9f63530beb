"""Compiles the mslice CUDA library in-tree for sm_103a.

Each .cu file is compiled to an object in parallel (one -gencode, -lineinfo)
and linked into ``libmslice.so`` beside this file.  Used by the package's
``build()`` and by the repository's build entry point.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmslice.so")
CHECKED_LIB = os.path.join(HERE, "libmslice_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-fmad=false", "--expt-relaxed-constexpr"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, extra, obj_dir=OBJ_DIR):
    obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
    if _stale(obj, [src] + _headers()):
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Builds libmslice.so, or with checked=True libmslice_checked.so: the
    same sources with -DMSLICE_CHECKED=1 (index and table bounds tested on the
    hot paths, violations reported as an error instead of accessed)."""
    obj_dir = OBJ_DIR + ("_checked" if checked else "")
    lib = CHECKED_LIB if checked else LIB
    extra = list(extra) + (["-DMSLICE_CHECKED=1"] if checked else [])
    os.makedirs(obj_dir, exist_ok=True)
    srcs = _sources()
    if force:
        for f in glob.glob(os.path.join(obj_dir, "*.o")):
            os.remove(f)
    jobs = int(os.environ.get("MSLICE_BUILD_JOBS", "0")) or min(8, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, obj_dir), srcs))
    if _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    if verbose:
        print(lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv)
