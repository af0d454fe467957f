"""Oracle pins for the Roe flux option (the paper's Riemann solver, Sec. 2.1.2).

Roe's linearisation has a defining property: A(UL, UR) (UR - UL) = F(UR) - F(UL).
When every wave moves the same way the upwinded flux is then exactly the upwind
side's physical flux; a wrong Roe average, eigenvector or wave strength breaks
it.  Consistency (Roe(U, U) = F(U)), the rotation to y, the dry-dry case, the
lake at rest, mass and convergence to the Stoker closed form follow."""
import numpy as np
import pytest

from conftest import riemann_planes
import oracle
from test_oracle_riemann import l1_error, stoker_h

G = 9.80665


def _fx(h, qx, qy):
    u, v = qx / h, qy / h
    return np.array([h * u, h * u * u + 0.5 * G * h * h, h * u * v])


def test_roe_consistency_rotation_and_dry():
    o = oracle.Oracle(2, 2, 1.0, 1.0, flux="roe")
    rng = np.random.default_rng(5)
    for _ in range(200):
        h = rng.uniform(1e-3, 4.0)
        qx, qy = rng.normal(size=2)
        assert np.allclose(o.hll(0, [h, qx, qy], [h, qx, qy]), _fx(h, qx, qy), rtol=1e-13, atol=1e-13)
        hr = rng.uniform(1e-3, 4.0)
        qxr, qyr = rng.normal(size=2)
        fx = o.hll(0, [h, qx, qy], [hr, qxr, qyr])
        fy = o.hll(1, [h, qy, qx], [hr, qyr, qxr])
        assert np.array_equal(fx, fy[[0, 2, 1]])
    assert np.array_equal(o.hll(0, [0.0, 0.0, 0.0], [1e-6, 0.0, 0.0]), np.zeros(3))


def test_roe_property_gives_the_upwind_flux():
    """All three waves right-going (supercritical to the right on both sides): the
    flux is F(UL); all left-going: F(UR)."""
    o = oracle.Oracle(2, 2, 1.0, 1.0, flux="roe")
    rng = np.random.default_rng(6)
    for _ in range(200):
        hl, hr = rng.uniform(0.1, 2.0, size=2)
        ul = np.sqrt(G * hl) * rng.uniform(1.5, 3.0)
        ur = np.sqrt(G * hr) * rng.uniform(1.5, 3.0)
        vl, vr = rng.normal(size=2)
        L = [hl, hl * ul, hl * vl]
        R = [hr, hr * ur, hr * vr]
        f = o.hll(0, L, R)
        assert np.allclose(f, _fx(*L), rtol=1e-12, atol=1e-12), (f, _fx(*L))
        Lm = [hl, -hl * ul, hl * vl]
        Rm = [hr, -hr * ur, hr * vr]
        f = o.hll(0, Lm, Rm)
        assert np.allclose(f, _fx(*Rm), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("limiter", [False, True])
def test_roe_lake_at_rest_and_mass(limiter):
    from paper_2010_02003_gb300 import inputs
    from conftest import make_oracle
    case = inputs.hump(eta=1.0)                      # fully wet hump
    o = make_oracle(case, limiter=limiter, flux="roe")
    m0 = o.mass()
    for _ in range(100):
        o.step()
    s = o.state()
    assert np.abs(s[3:]).max() <= 1e-12
    assert abs(o.mass() - m0) <= 1e-13 * m0
    blocks = inputs.wall_blocks()                    # still water against raised ground
    o = make_oracle(blocks, limiter=limiter, flux="roe")
    for _ in range(100):
        o.step()
    assert np.abs(o.state()[3:]).max() <= 1e-12


def test_roe_stoker_converges_with_the_limiter():
    """Across the Stoker hydraulic jump DG2-NL with Roe's (less dissipative) flux
    goes unstable (negative depths, then NaN at 200 cells) where HLL stays bounded;
    with the local limiter (DG2-LL, the paper's choice for shocks) it converges."""
    errs = []
    for nx in (100, 200, 400):
        dx = 100.0 / nx
        o = oracle.Oracle(nx, 3, dx, dx, cfl=0.3, flux="roe", limiter=True)
        o.set_dem(np.zeros((4, nx + 1)))
        o.set_state(riemann_planes(nx, 3, dx, 50.0, (1.0, 0, 0), (0.1, 0, 0)))
        o.run_to(4.0)
        e, s = l1_error(o, dx, lambda x: stoker_h(x, 4.0, 1.0, 0.1, 50.0))
        errs.append(e)
        assert s[0].min() > 0.0
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[2] > 2.5
    assert errs[2] < 0.1
