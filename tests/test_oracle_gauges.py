"""Pins of the oracle's gauge evaluation (the sampled depth series of Sec. 3).

A gauge reads the depth of the containing cell's piecewise-planar solution
(Eq. 2): h0 + xi h1x + eta h1y with xi = (x - x_c) / (dx / 2), eta likewise,
clipped at zero.  A depth field that is one plane over the whole grid is held
exactly by the modes (h0 = the plane at the centre, h1x = its x-gradient times
dx / 2), so at any point the gauge must return the plane itself: a mis-scaled or
swapped xi / eta, a wrong cell index or a missing clip fails below.  The grid is
anisotropic (dx != dy) so that x and y cannot stand in for each other.
"""
import numpy as np

from conftest import make_oracle
from paper_2010_02003_gb300 import inputs
import oracle

NX, NY, DX, DY = 13, 7, 3.0, 1.25


def _plane(a, b, c):
    """Mode planes of the depth field h(x, y) = a + b x + c y (discharges zero)."""
    xc = (np.arange(NX) + 0.5) * DX
    yc = (np.arange(NY) + 0.5) * DY
    P = np.zeros((9, NY, NX))
    P[0] = a + b * xc[None, :] + c * yc[:, None]
    P[1] = b * DX / 2
    P[2] = c * DY / 2
    return P


def _oracle_with(planes):
    o = oracle.Oracle(NX, NY, DX, DY)
    o.set_dem(np.zeros((NY + 1, NX + 1)))
    o.set_state(planes, 0.0)
    return o


def test_gauge_returns_a_global_plane_exactly_at_interior_points():
    a, b, c = 0.4, 0.013, -0.021
    o = _oracle_with(_plane(a, b, c))
    rng = np.random.default_rng(3)
    for x, y in rng.uniform([0, 0], [NX * DX, NY * DY], size=(200, 2)):
        want = a + b * x + c * y
        assert abs(o.gauge_h(x, y) - max(want, 0.0)) <= 1e-14, (x, y)


def test_gauge_at_cell_edges_and_domain_edges():
    a, b, c = 0.3, 0.02, 0.05
    o = _oracle_with(_plane(a, b, c))
    # on a face between two cells the plane is continuous: either cell gives it
    for i in range(NX + 1):
        for j in range(NY + 1):
            x, y = i * DX, j * DY
            assert abs(o.gauge_h(x, y) - (a + b * x + c * y)) <= 1e-14, (i, j)


def test_gauge_clips_negative_planar_depth_to_zero():
    # a plane crossing zero inside the grid: depth a + b x is negative west of x = 12 m
    a, b = -0.24, 0.02
    o = _oracle_with(_plane(a, b, 0.0))
    for x in np.linspace(0.0, NX * DX, 53):
        want = a + b * x
        got = o.gauge_h(x, 2.0)
        assert got >= 0.0
        assert abs(got - max(want, 0.0)) <= 1e-14, x


def test_gauge_reads_each_direction_with_its_own_half_width():
    # x-gradient only, then y-gradient only: a swapped or common half width fails one
    for b, c in ((0.05, 0.0), (0.0, 0.05)):
        o = _oracle_with(_plane(1.0, b, c))
        for x, y in ((DX * 0.9, DY * 3.1), (DX * 5.25, DY * 0.6), (DX * 12.99, DY * 6.99)):
            assert abs(o.gauge_h(x, y) - (1.0 + b * x + c * y)) <= 1e-14, (b, c, x, y)


def test_run_to_samples_a_lake_at_rest_over_a_tilted_bed():
    """Still water over a planar bed is a fixed point of the scheme (well-balanced,
    Sec. 2.1.2), so the depth stays the plane eta - z: run_to must land on every
    multiple of the sample interval and record that plane at each gauge."""
    case = inputs.hump(nx=NX, ny=NY, dx=DX, eta=2.0, amp=0.0)
    case.dy = DY
    xs = np.arange(NX + 1) * DX
    ys = np.arange(NY + 1) * DY
    case.z_corner = 0.01 * xs[None, :] + 0.03 * ys[:, None]
    case.eta_corner = np.full_like(case.z_corner, 2.0)
    o = make_oracle(case)
    gauges = np.array([[1.0, 1.0], [DX * 6, DY * 3.5], [20.3, 6.1], [NX * DX, NY * DY]])
    steps, t, h = o.run_to(3.0, 0.5, gauges)
    assert steps > 0
    assert np.array_equal(t, 0.5 * np.arange(1, 7))
    want = 2.0 - (0.01 * gauges[:, 0] + 0.03 * gauges[:, 1])
    assert np.abs(h - want[None, :]).max() <= 1e-12
