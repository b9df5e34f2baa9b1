"""Build libpcc.so (the CUDA library behind include/pcc.h) in-tree.

Every .cu under csrc/ is compiled for sm_103a only, in parallel, then linked
into paper_1605_01584_gb300/libpcc.so with the static CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpcc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"),
              "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required")


def _flags(verbose_ptxas: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                "-I" + INCLUDE, "-I" + CSRC, "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(obj, src, hdr_mtime):
    return (not os.path.exists(obj) or
            os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_mtime))


def build(force: bool = False, verbose_ptxas: bool = False,
          jobs: int | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    hdr = max([os.path.getmtime(h) for h in _headers()] + [0.0])
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    todo = [(s, o) for s, o in zip(srcs, objs)
            if force or verbose_ptxas or _stale(o, s, hdr)]
    cc = nvcc()

    def compile_one(so):
        s, o = so
        cmd = [cc] + _flags(verbose_ptxas) + ["-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {s}:\n{r.stdout}\n{r.stderr}")
        return s, r.stderr

    if todo:
        with cf.ThreadPoolExecutor(jobs or min(8, len(todo))) as ex:
            for s, err in ex.map(compile_one, todo):
                if verbose_ptxas and err:
                    sys.stderr.write(f"== {os.path.basename(s)}\n{err}")
    if todo or not os.path.exists(LIB) or force:
        tmp = LIB + ".tmp"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv,
                verbose_ptxas="-v" in sys.argv))
