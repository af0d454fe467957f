"""Oracle pins: symmetry and order of accuracy.

- The circular dam break over the centred hump is invariant under x <-> y
  transposition.  The oracle's x and y paths perform the same arithmetic
  (the y flux is the x flux in a rotated frame); only Eq. 3a's average
  (taken from the E/W face values) sums the four corners in a different order
  for the transposed cell, so the state stays symmetric to round-off.  A
  transposed operand or an x/y mix-up in Eq. 4 gives O(1) differences.
- It is also mirror-symmetric; mirroring changes the order of floating-point
  operations, so that holds to round-off.
- DG2-LL's detector (Eq. 6) switches on round-off-level discharges (its
  denominator vanishes with q), which turns round-off asymmetries into ~1e-9
  ones; LL is held to 1e-7.
- On a smooth wet flow DG2 is second order (Sec. 2): self-convergence of the
  cell averages under refinement.
"""
import numpy as np
import pytest

from conftest import make_oracle
from paper_2010_02003_gb300 import inputs


def transpose_state(s):
    # planes h0 h1x h1y qx0 qx1x qx1y qy0 qy1x qy1y under x <-> y
    perm = [0, 2, 1, 6, 8, 7, 3, 5, 4]
    return s[perm].transpose(0, 2, 1)


def mirror_x_state(s):
    sign = np.array([1, -1, 1, -1, 1, -1, 1, -1, 1], dtype=float)[:, None, None]
    return sign * s[:, :, ::-1]


@pytest.mark.parametrize("limiter", [False, True])
def test_dam_break_transposition(limiter):
    case = inputs.hump(nx=64, ny=64, eta=0.5, dam_eta=1.0, dam_radius=10.0, width2=50.0)
    assert np.array_equal(case.z_corner, case.z_corner.T)
    o = make_oracle(case, limiter=limiter)
    for _ in range(60):
        o.step()
    s = o.state()
    scale = np.abs(s).reshape(9, -1).max(axis=1)[:, None, None] + 1e-300
    assert (np.abs(s - transpose_state(s)) / scale).max() <= (1e-7 if limiter else 1e-12)


@pytest.mark.parametrize("limiter", [False, True])
def test_dam_break_mirror_symmetry(limiter):
    case = inputs.hump(nx=64, ny=64, eta=0.5, dam_eta=1.0, dam_radius=10.0, width2=50.0)
    o = make_oracle(case, limiter=limiter)
    for _ in range(60):
        o.step()
    s = o.state()
    scale = np.abs(s).reshape(9, -1).max(axis=1)[:, None, None] + 1e-300
    assert (np.abs(s - mirror_x_state(s)) / scale).max() <= (1e-7 if limiter else 1e-12)


def _smooth_run(nx):
    case = inputs.smooth_wave_1d(nx=nx, ny=2)
    o = make_oracle(case)
    o.run_to(case.t_end)
    return o.state()[0].mean(axis=0)


def test_second_order_on_smooth_flow():
    h = {n: _smooth_run(n) for n in (50, 100, 200, 400)}

    def coarsen(a):
        return 0.5 * (a[0::2] + a[1::2])

    e = [np.abs(h[n] - coarsen(h[2 * n])).mean() for n in (50, 100, 200)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders.min() >= 1.8, (e, orders)
