"""The adjoint's reverse-mode local adjoints against its forward-mode dual numbers, on
the host: the device functions of dg2_adj.cu up to its kernels, compiled for the host
by nvcc, and tests/adjoint_local_check.cu comparing the two derivatives on 2e5 random
states (no GPU needed)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2010_02003_gb300", "csrc", "dg2_adj.cu")
MARK = "// Forward kernels (one thread per cell, dense planes)"


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


def test_reverse_mode_local_adjoints_match_dual_numbers(tmp_path):
    text = open(SRC).read()
    head = text[:text.index(MARK)]
    head = head[:head.rstrip().rfind("\n// ----")]  # drop the section rule above the marker
    head = re.sub(r"__device__ (__forceinline__|__noinline__)", r"__host__ __device__ \1", head)
    head = re.sub(r"^__device__ (void|bool) ", r"__host__ __device__ \1 ", head, flags=re.M)
    (tmp_path / "adj_head.inc").write_text(head)
    shutil.copy(os.path.join(ROOT, "tests", "adjoint_local_check.cu"), tmp_path / "check.cu")
    exe = tmp_path / "check"
    subprocess.check_call([_nvcc(), "-O2", "-std=c++17", "-I", str(tmp_path),
                           "-I", os.path.join(ROOT, "paper_2010_02003_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                           str(tmp_path / "check.cu")])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    print(out.stdout)
    assert out.returncode == 0, out.stdout
    assert "worst relative" in out.stdout
