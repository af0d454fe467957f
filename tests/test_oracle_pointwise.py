"""Oracle pins for the pointwise pieces: Eq. 3 initialisation, friction (Sec. 2.1.3),
the CFL time step and the local limiter (Eqs. 6-7).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2010_02003_gb300 import inputs

G = 9.80665
S3 = np.sqrt(3.0)


def test_eq3_modes_of_a_linear_field_are_exact():
    """Eq. 3 applied to face values averaged from corners reproduces a linear field:
    z0 = value at the centre, z1x = b dx/2, z1y = c dy/2."""
    nx, ny, dx, dy = 7, 5, 0.8, 1.3
    o = oracle.Oracle(nx, ny, dx, dy)
    X, Y = inputs.corner_xy(nx, ny, dx, dy)
    a, b, c = 0.25, 0.5, -0.125          # dyadic values keep every sum exact
    o.set_dem(a + b * X + c * Y)
    top = o.topo()
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dy
    XC, YC = np.meshgrid(xc, yc)
    assert np.allclose(top[0], a + b * XC + c * YC, rtol=0, atol=1e-15)
    assert np.allclose(top[1], b * dx / 2, rtol=0, atol=1e-15)
    assert np.allclose(top[2], c * dy / 2, rtol=0, atol=1e-15)


def test_initial_depth_keeps_flat_surface_and_dries_negative_cells():
    nx, ny = 6, 4
    o = oracle.Oracle(nx, ny, 1.0, 1.0)
    X, Y = inputs.corner_xy(nx, ny, 1.0, 1.0)
    z = 0.2 * X
    o.set_dem(z, eta_corner=np.full_like(z, 0.5))
    s, top = o.state(), o.topo()
    wet = s[0] > 0
    # wet cells: h + z planar is flat (h1 = -z1), including cells with a negative face limit
    assert np.allclose(s[1][wet], -top[1][wet], atol=1e-15)
    assert np.allclose((s[0] + top[0])[wet], 0.5, atol=1e-15)
    # cells whose average depth is not positive start dry (all h modes zero)
    assert np.all(s[:3, ~wet] == 0.0)
    assert (~wet).sum() == 16           # centres x = 2.5 .. 5.5 (4 columns x 4 rows): 0.5 - 0.2 x <= 0


def test_friction_matches_exact_ode_solution_over_many_steps():
    """Friction alone on uniform flow, applied 40 times: the implicit update with |q| frozen
    equals the exact solution of dq/dt = -g n^2 q|q| / h^(7/3), i.e.
    1/|q|(t) = 1/|q0| + t g n^2 / h^(7/3), at every step (not just in the limit)."""
    nx, ny, h, qx, qy, n = 6, 5, 0.7, 0.8, -0.6, 0.05
    o = oracle.Oracle(nx, ny, 2.0, 2.0)
    o.set_dem(np.zeros((ny + 1, nx + 1)), n_uniform=n)
    P = np.zeros((9, ny, nx))
    P[0], P[3], P[6] = h, qx, qy
    t = 0.0
    for _ in range(40):
        P = o.friction(P, 0.05)
        t += 0.05
    q0 = np.hypot(qx, qy)
    q_exact = 1.0 / (1.0 / q0 + t * G * n * n / h ** (7.0 / 3.0))
    assert np.allclose(np.hypot(P[3], P[6]), q_exact, rtol=1e-12)
    assert np.allclose(P[3] / P[6], qx / qy, rtol=1e-12)          # direction unchanged
    assert np.array_equal(P[0], np.full((ny, nx), h))
    assert np.abs(P[[1, 2, 4, 5, 7, 8]]).max() == 0.0               # slopes stay zero


def test_friction_at_gauss_points_differentiates_to_slopes():
    """Friction acts at the centre (average) and at the two Gauss points +-1/sqrt(3) of each
    centreline; the new slope is sqrt(3)/2 times the difference of the Gauss-point values
    (Sec. 2.1.3).  Each point follows the exact ODE solution above."""
    o = oracle.Oracle(1, 1, 1.0, 1.0)
    o.set_dem(np.zeros((2, 2)), n_uniform=0.04)
    U = np.array([0.9, 0.2, -0.15, 0.5, 0.12, -0.07, -0.3, 0.05, 0.09]).reshape(9, 1, 1)
    dt = 0.3
    out = o.friction(U, dt)
    a = G * 0.04 ** 2

    def fr(h, qx, qy):
        qm = np.hypot(qx, qy)
        f = (1.0 / (1.0 / qm + dt * a / h ** (7.0 / 3.0))) / qm
        return qx * f, qy * f

    u = U[:, 0, 0]
    cx, cy = fr(u[0], u[3], u[6])
    assert np.isclose(out[3, 0, 0], cx, rtol=1e-13) and np.isclose(out[6, 0, 0], cy, rtol=1e-13)
    for d in (1, 2):
        gp = fr(u[0] + u[d] / S3, u[3] + u[3 + d] / S3, u[6] + u[6 + d] / S3)
        gm = fr(u[0] - u[d] / S3, u[3] - u[3 + d] / S3, u[6] - u[6 + d] / S3)
        assert np.isclose(out[3 + d, 0, 0], S3 / 2 * (gp[0] - gm[0]), rtol=1e-12)
        assert np.isclose(out[6 + d, 0, 0], S3 / 2 * (gp[1] - gm[1]), rtol=1e-12)
    assert np.array_equal(out[:3], U[:3])          # depth untouched


def test_cfl_dt_uniform_state():
    nx, ny, dx, dy = 4, 3, 2.0, 1.5
    o = oracle.Oracle(nx, ny, dx, dy, cfl=0.33, dt_max=100.0)
    o.set_dem(np.zeros((ny + 1, nx + 1)))
    P = np.zeros((9, ny, nx))
    h, u, v = 1.2, 0.7, -2.1
    P[0], P[3], P[6] = h, h * u, h * v
    o.set_state(P)
    c = np.sqrt(G * h)
    assert np.isclose(o.cfl_dt(), 0.33 * min(dx / (abs(u) + c), dy / (abs(v) + c)), rtol=1e-14)
    # no wet cell: dt_max
    o.set_state(np.zeros((9, ny, nx)))
    assert o.cfl_dt() == 100.0


def test_minmod_table():
    vals = [-2.0, -0.5, 0.0, 0.75, 3.0]
    for a, b, c in itertools.product(vals, repeat=3):
        m = oracle.minmod(a, b, c)
        if a > 0 and b > 0 and c > 0:
            assert m == min(a, b, c)
        elif a < 0 and b < 0 and c < 0:
            assert m == max(a, b, c)
        else:
            assert m == 0.0


def _paper_limit_1d(k0, k1, dxh, thresh=10.0):
    """Eqs. 6-7 in their printed ratio form, for the middle of three cells (numpy)."""
    jE = abs((k0[2] - k1[2]) - (k0[1] + k1[1]))
    jW = abs((k0[1] - k1[1]) - (k0[0] + k1[0]))
    den = dxh * max(abs(k0[1] - k1[1] / S3), abs(k0[1] + k1[1] / S3))
    with np.errstate(divide="ignore", invalid="ignore"):
        ds = max(jE / den if den > 0 else (np.inf if jE > 0 else 0.0),
                 jW / den if den > 0 else (np.inf if jW > 0 else 0.0))
    if not ds > thresh:
        return k1[1]
    a, b, c = k1[1], k0[2] - k0[1], k0[1] - k0[0]
    if a > 0 and b > 0 and c > 0:
        return min(a, b, c)
    if a < 0 and b < 0 and c < 0:
        return max(a, b, c)
    return 0.0


@pytest.mark.parametrize("seed", range(6))
def test_limiter_matches_printed_detector_and_minmod(seed):
    """Random three-cell rows (x) and columns (y): the limited slope of the middle cell equals
    Eqs. 6-7 evaluated in ratio form, for qx, qy and (via eta = h + z) h; dry neighbours
    switch limiting off; edge cells are never limited normal to the edge."""
    rng = np.random.default_rng(seed)
    for axis in (0, 1):
        nx, ny = (3, 1) if axis == 0 else (1, 3)
        d = 1 if axis == 0 else 2
        dxh = 0.5 * (1.7 if axis == 0 else 0.9)
        o = oracle.Oracle(nx, ny, 1.7, 0.9, limiter=True)
        z = rng.uniform(0, 0.3, size=(ny + 1, nx + 1))
        o.set_dem(z)
        top = o.topo()
        for _ in range(40):
            U = np.zeros((9, ny, nx))
            U[0] = rng.uniform(0.05, 1.0, size=(ny, nx))
            for k in range(1, 9):
                U[k] = rng.normal(scale=0.3, size=(ny, nx)) * rng.integers(0, 2)
            if rng.random() < 0.2:
                U[0].flat[rng.integers(0, 3)] = 1e-6          # a dry neighbour or cell
            out = o.limit(U)
            h0 = U[0].ravel()
            dry = (h0 <= 1e-5).any()
            for v, plane0 in ((1, 3), (2, 6)):
                k0, k1 = U[plane0].ravel(), U[plane0 + d].ravel()
                want = k1[1] if dry else _paper_limit_1d(k0, k1, dxh)
                assert out[plane0 + d].ravel()[1] == pytest.approx(want, rel=0, abs=1e-15)
            e0 = U[0].ravel() + top[0].ravel()
            e1 = U[d].ravel() + top[d].ravel()
            lim = e1[1] if dry else _paper_limit_1d(e0, e1, dxh)
            assert out[d].ravel()[1] == pytest.approx(lim - top[d].ravel()[1], abs=1e-14)
            # the two edge cells keep their slopes along this axis; averages never change
            for c in (0, 2):
                for p in (d, 3 + d, 6 + d):
                    assert out[p].ravel()[c] == U[p].ravel()[c]
            assert np.array_equal(out[[0, 3, 6]], U[[0, 3, 6]])


def test_limiter_is_inactive_on_smooth_flow():
    """On a smooth wet flow whose discharges stay far from zero the detector (Eq. 6) never
    fires, so DG2-LL takes exactly the DG2-NL step (cf. the identical DG2 variants on the
    smooth bowl flow, Sec. 2.3)."""
    nx, ny, dx = 24, 20, 1.0
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dx
    XC, YC = np.meshgrid(xc, yc)
    P = np.zeros((9, ny, nx))
    P[0] = 1.0 + 0.05 * np.sin(0.2 * XC) * np.cos(0.15 * YC)
    P[1] = 0.05 * 0.2 * 0.5 * dx * np.cos(0.2 * XC) * np.cos(0.15 * YC)
    P[3] = 0.6 + 0.03 * np.cos(0.1 * YC)
    P[6] = 0.4 + 0.02 * np.sin(0.1 * XC)
    runs = []
    for limiter in (False, True):
        o = oracle.Oracle(nx, ny, dx, dx, limiter=limiter)
        o.set_dem(np.zeros((ny + 1, nx + 1)))
        o.set_state(P)
        for _ in range(3):
            o.step(0.02)
        runs.append(o.state())
    assert np.array_equal(runs[0], runs[1])


def test_limiter_is_inactive_at_rest():
    """Still water against walls: the discharges are round-off, below the detector's floor,
    so DG2-LL takes exactly the DG2-NL steps."""
    from conftest import make_oracle
    case = inputs.wall_blocks()
    a, b = make_oracle(case, limiter=False), make_oracle(case, limiter=True)
    for _ in range(30):
        a.step()
        b.step()
    assert np.array_equal(a.state(), b.state())
