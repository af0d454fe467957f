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
SRC = [os.path.join(HERE, "csrc", "dg2_api.cu"), os.path.join(HERE, "csrc", "dg2_noalloc.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", f) for f in ("dg2_device.cuh", "dg2_fs32.cuh")] + [
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
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-prec-div=false", "-prec-sqrt=false",
           "-ftz=true", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-o", tmp, *SRC]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
