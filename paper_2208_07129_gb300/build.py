"""Build libfe.so (the CUDA library behind include/fe.h) in-tree for sm_103a.

Every ``csrc/*.cu`` file is compiled in parallel by nvcc into ``_objs/`` and
linked into ``paper_2208_07129_gb300/libfe.so``.  Only changed sources are
recompiled.  No cmake; one ``-gencode`` (compute_103a / sm_103a).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
OBJS = os.path.join(PKG, "_objs")
LIB = os.path.join(PKG, "libfe.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    n = shutil.which("nvcc")
    if n is None and os.path.exists("/usr/local/cuda/bin/nvcc"):
        n = "/usr/local/cuda/bin/nvcc"
    if n is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfe")
    return n


_INC = re.compile(r'^\s*#\s*include\s*"([^"]+)"', re.M)


def _local_deps(path: str, seen: set) -> set:
    """Every quoted #include reachable from `path` that resolves to a file in
    csrc/ or include/ (the only headers this library owns)."""
    try:
        text = open(path, encoding="utf-8", errors="replace").read()
    except OSError:
        return seen
    for name in _INC.findall(text):
        for base in (os.path.dirname(path), CSRC, INCLUDE):
            cand = os.path.normpath(os.path.join(base, name))
            if os.path.exists(cand):
                if cand not in seen:
                    seen.add(cand)
                    _local_deps(cand, seen)
                break
    return seen


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(OBJS, os.path.basename(src)[:-3] + ".o")
    newest = max([os.path.getmtime(src)] + [os.path.getmtime(d) for d in _local_deps(src, set())])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj
    cmd = [_nvcc(), *ARCH, *FLAGS, "-c", src, "-o", obj + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OBJS, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs = jobs or max(1, min(len(srcs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), srcs))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lcublas", "-lcusolver"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
