"""Builds the C-ABI library libdg2.so (hand-written CUDA for sm_103a) in-tree.

nvcc cross-compiles without a GPU; the result is placed next to this file and
loaded by :mod:`paper_2010_02003_gb300.binding`.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", f)
       for f in ("dg2_api.cu", "dg2_ens.cu", "dg2_adj.cu", "dg2_adj32.cu", "dg2_adj_api.cu",
                 "dg2_noalloc.cu", "dg2_peak.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", f)
              for f in ("dg2_device.cuh", "dg2_fs32.cuh", "dg2_fs32_staged.cuh", "dg2_fv.cuh", "dg2_internal.h")] + [
    os.path.join(ROOT, "include", "dg2.h")]
LIB = os.path.join(HERE, "libdg2.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libdg2.so)")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libdg2.so if it is missing or older than its sources; returns its path."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= t for p in DEPS):
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    # single-precision division / square root use the hardware approximations and
    # FP32 denormals flush to zero (the FP32 path's error is stated against the FP64
    # oracle); these flags do not touch FP64 arithmetic, whose parity is 1e-12
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-prec-div=false", "-prec-sqrt=false",
             "-ftz=true", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    # one object per translation unit, compiled in parallel, then linked
    objs = [f"{tmp}.{i}.o" for i in range(len(SRC))]
    procs = [subprocess.Popen([nvcc(), *flags, "-c", src, "-o", obj])
             for src, obj in zip(SRC, objs)]
    codes = [p.wait() for p in procs]
    try:
        if any(codes):
            raise subprocess.CalledProcessError(max(codes, key=abs), "nvcc -c")
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
