"""Oracle pins: mass (Eq. 11).

L0 of h is a pure flux difference (Eq. 4a); friction, limiting and the dry reset
never touch h0, and a wall face carries exactly zero mass flux.  So with closed
walls M(t) = M0 to round-off, and with open / inflow edges and sources M(t)
matches the ledger M0 + sum of boundary and source volumes.
"""
import numpy as np
import pytest

from conftest import make_oracle
from paper_2010_02003_gb300 import inputs


@pytest.mark.parametrize("limiter", [False, True])
def test_closed_walls_conserve_mass(limiter):
    case = inputs.hump(eta=0.5, dam_eta=1.0)
    o = make_oracle(case, limiter=limiter)
    m0 = o.mass()
    for _ in range(100):
        o.step()
    assert abs(o.mass() - m0) / m0 <= 1e-13


@pytest.mark.parametrize("limiter", [False, True])
def test_open_and_inflow_edges_match_ledger(limiter):
    case = inputs.floodplain(nx=60, ny=40, dx=2.0, q_peak=5.0, t_peak=30.0, initial="channel",
                             channel_width=12.0)
    o = make_oracle(case, limiter=limiter)
    m0 = o.mass()
    for _ in range(150):
        o.step()
    m = o.mass()
    assert abs(m - o.ledger()) / m <= 1e-12
    assert abs(m - m0) > 1.0            # boundaries really moved water in or out


def test_rain_and_point_source_match_ledger():
    case = inputs.hump(nx=40, ny=30, eta=0.5)
    case.rain = (1e-3, 0.0, 2.0)
    case.point = (10.5, 12.5, 0.4)
    o = make_oracle(case)
    m0 = o.mass()
    while o.t < 4.0:
        o.step()
    m = o.mass()
    # rain stops at t=2 s: volume = rate * area * 2 s (+ point inflow * elapsed time)
    area = case.nx * case.ny * case.dx * case.dy
    assert abs(m - o.ledger()) / m <= 1e-12
    assert m - m0 > 0.4 * 4.0 + 1e-3 * area * 1.9


def test_wall_face_has_zero_mass_flux():
    """HLL flux between a state and its wall mirror has exactly zero mass flux."""
    import oracle
    o = oracle.Oracle(4, 4, 1.0, 1.0)
    rng = np.random.default_rng(3)
    for _ in range(200):
        h = rng.uniform(1e-3, 3.0)
        qn, qt = rng.normal(size=2)
        f = o.hll(0, [h, qn, qt], [h, -qn, qt])
        assert f[0] == 0.0
        f = o.hll(1, [h, qt, qn], [h, qt, -qn])
        assert f[0] == 0.0
