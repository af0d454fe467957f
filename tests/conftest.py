import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libdg2.so")
    config.addinivalue_line("markers", "slow: longer CPU-only oracle runs")


def make_oracle(case, limiter=False, **kw):
    """Oracle problem built from an inputs.Case (test helper)."""
    import oracle
    kw.setdefault("dt_max", case.dt_max)
    o = oracle.Oracle(case.nx, case.ny, case.dx, case.dy, cfl=case.cfl, limiter=limiter, bc=case.bc,
                      **kw)
    o.set_dem(case.z_corner, case.manning, case.n_uniform, case.eta_corner)
    for f in case.inflows:
        o.add_inflow(f.edge, f.s0, f.length, f.t_knots, f.q_knots)
    rx, ry, rq = case.point
    r, r0, r1 = case.rain
    if r != 0.0 or rq != 0.0:
        o.set_sources(r, r0, r1, rx, ry, rq)
    return o


def riemann_planes(nx, ny, dx, x0, left, right):
    """Piecewise-constant (zero-slope) state: `left`=(h, qx, qy) for cell centres < x0."""
    xc = (np.arange(nx) + 0.5) * dx
    P = np.zeros((9, ny, nx))
    for v in range(3):
        P[3 * v] = np.where(xc < x0, left[v], right[v])[None, :]
    return P
