"""The C-ABI library builds, loads and exports every symbol include/dg2.h declares
(no compute calls: runs without a GPU)."""
import ctypes

import numpy as np
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dg2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg2_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("dg2_init_grid", "dg2_set_dem", "dg2_set_bc_inflow", "dg2_step", "dg2_run_to",
                     "dg2_read_gauges", "dg2_mass"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2010_02003_gb300 import build, binding
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTS) == declared_functions()


def test_host_only_calls_without_gpu():
    """Calls that touch no device: defaults, workspace sizing, argument errors."""
    from paper_2010_02003_gb300 import binding as B
    B.load()
    p = B.dg2_default_params()
    assert p.cfl == pytest.approx(0.3) and p.tol_dry == 1e-5 and p.ds_thresh == 10.0
    assert p.flux == B.DG2_HLL and p.scheme == B.DG2_SCHEME_DG2
    n1 = B.dg2_workspace_bytes(128, 128, p)
    p.variant = B.DG2_LL
    n2 = B.dg2_workspace_bytes(128, 128, p)
    assert n2 > n1 > 128 * 128 * 8 * 22
    assert B.dg2_workspace_bytes(0, 5, p) == 0
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_init_grid(8, 8, 1.0, 1.0, p, 0, 10 ** 6, 0)
    assert e.value.code == B.DG2_E_ARG
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_tile_shape(None)
    assert e.value.code == B.DG2_E_ARG


def test_product_path_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_2010_02003_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "dg2_oracle" not in text, f


def test_ensemble_host_only_calls_without_gpu():
    from paper_2010_02003_gb300 import binding as B
    B.load()
    assert B.dg2_ens_workspace_bytes([]) == 0
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_ens_create([], 0, 0, 0)
    assert e.value.code == B.DG2_E_ARG


def test_ensemble_recipe_sizes_and_seeds():
    """The 256-member recipe: sizes log-uniform in [64, 1024] x [64, 512], ~19M cells in
    all, one Manning n and one inflow peak per member, reproducible from the seed."""
    from paper_2010_02003_gb300 import inputs
    a = inputs.ensemble(n=256)
    nx = [c.nx for c in a]
    ny = [c.ny for c in a]
    assert 64 <= min(nx) and max(nx) <= 1024 and 64 <= min(ny) and max(ny) <= 512
    assert 1.5e7 < sum(x * y for x, y in zip(nx, ny)) < 2.5e7
    for c in a[:8]:
        assert np.unique(c.manning).size == 1 and 0.02 <= c.manning[0, 0] <= 0.08
        q = c.inflows[0].q_knots.max()
        assert 5.0 <= q <= 40.0 and c.inflows[0].t_knots[1] == 1800.0
    b = inputs.ensemble(n=3)
    for x, y in zip(a[:3], b):
        assert x.nx == y.nx and np.array_equal(x.z_corner, y.z_corner)
