"""Closed-form pins of the oracle's boundary inflow (R5), friction (R4), bed-slope
term (Eq. 4a) and rain source (no GPU).

- Rain on a flat closed basin: nothing moves, so the depth rises at exactly the rain
  rate, h(t) = h(0) + r t, and every other mode stays zero.
- Uniform flow down a plane slope fed by the inflow boundary and leaving through a
  transmissive edge: Manning's normal flow, q = h^(5/3) S0^(1/2) / n per unit width, is
  a steady state of the continuous equations; started from it, the oracle must hold
  the normal depth and carry the inflow's discharge (a wrong ghost discharge,
  friction law or slope term moves the depth away from it).
"""
import numpy as np
import pytest

import oracle
from oracle import OPEN, WALL


@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_rain_on_a_flat_closed_basin(limiter):
    nx, ny, h0, r = 12, 9, 0.5, 1e-4
    o = oracle.Oracle(nx, ny, 1.0, 1.0, limiter=limiter)
    o.set_dem(np.zeros((ny + 1, nx + 1)), None, 0.03, np.full((ny + 1, nx + 1), h0))
    o.set_sources(rain=r, rain_t0=0.0, rain_t1=100.0)
    for _ in range(20):
        o.step(0.5)
    st = o.state()
    assert np.abs(st[0] - (h0 + r * o.t)).max() <= 1e-14
    assert np.abs(st[1:]).max() == 0.0
    assert abs(o.mass() - o.ledger()) <= 1e-13 * o.mass()


@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_normal_flow_on_a_slope_with_inflow(limiter):
    """Subcritical uniform flow (Froude 0.56) down a 400 m plane slope: the upstream
    half, 200 m and more from the transmissive outlet, holds Manning's normal depth.
    The stored discharge is the splitting's fixed point (R4: friction once per step
    before the two stages): the step's mean face discharge, q* - dt g h S0 / 2, equals
    the inflow q; q* itself sits dt g h S0 / 2 above it."""
    nx, ny, dx = 200, 3, 2.0
    S0, n, q, g = 1e-2, 0.05, 0.5, 9.80665            # slope, Manning n, m^2/s
    hn = (q * n / np.sqrt(S0)) ** 0.6                  # Manning normal depth, 0.435 m
    xc = np.arange(nx + 1) * dx
    z = np.tile(3.0 - S0 * xc, (ny + 1, 1))
    o = oracle.Oracle(nx, ny, dx, dx, limiter=limiter, bc=(WALL, OPEN, WALL, WALL),
                      dt_max=1.0)
    o.set_dem(z, None, n, z + hn)
    st = o.state()
    st[3] = q                                          # qx0 = q in every cell
    o.set_state(st, 0.0)
    width = ny * dx
    o.add_inflow(0, 0.0, width, [0.0, 1e6], [q * width, q * width])
    while o.t < 600.0:
        dt = o.step()
    st = o.state()
    up = slice(5, nx // 2)
    h = st[0][:, up]
    assert np.abs(h / hn - 1.0).max() < 2e-4
    mean_flux = st[3][:, up] - dt * g * h * S0 / 2
    assert np.abs(mean_flux / q - 1.0).max() < 1e-4
    assert np.abs(st[6]).max() < 1e-9                  # no transverse flow
    assert abs(o.mass() - o.ledger()) <= 1e-12 * o.mass()


def test_point_source_fills_its_cell():
    """A point inflow Q into a closed single cell raises its depth at exactly
    Q / (dx dy); on a 5 x 5 basin with the source at the centre cell, one step
    leaves the depth symmetric about that cell and the volume up by Q dt."""
    dx, dy, q, h0 = 2.0, 1.5, 0.03, 0.2
    o = oracle.Oracle(1, 1, dx, dy)
    o.set_dem(np.zeros((2, 2)), None, 0.0, np.full((2, 2), h0))
    o.set_sources(px=0.7, py=0.4, qp=q)
    for _ in range(10):
        o.step(0.5)
    assert abs(o.state()[0, 0, 0] - (h0 + q * 5.0 / (dx * dy))) <= 1e-15
    o = oracle.Oracle(5, 5, dx, dy)
    o.set_dem(np.zeros((6, 6)), None, 0.0, np.full((6, 6), h0))
    o.set_sources(px=2.5 * dx, py=2.5 * dy, qp=q)
    m0 = o.mass()
    o.step(0.1)
    h = o.state()[0]
    assert np.abs(h - h[::-1, :]).max() <= 1e-15 and np.abs(h - h[:, ::-1]).max() <= 1e-15
    assert h[2, 2] == h.max() and h[2, 2] > h0
    assert abs(o.mass() - (m0 + q * 0.1)) <= 1e-15 * o.mass()
