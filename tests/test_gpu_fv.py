"""GPU MUSCL-FV2 and FV1 comparators (Sec. 2.2, Eqs. 8-10) through the C ABI against
the FP64 oracle's FV schemes.

Bar (FP64), as for DG2: the averages h0, qx0, qy0 within 1e-12 of the scale of their
variable after 100 steps with the oracle's time steps forced, the slope planes zero,
and the mass and ledger within 1e-12 relative; every step from the oracle's own state
within 1e-12, or, on a step the oracle itself moves by more than 1e-14 under a 2e-16
perturbation of its input, within 100 times that sensitivity.
"""
import numpy as np
import pytest

from conftest import make_oracle
from paper_2010_02003_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12
AVG = [0, 3, 6]          # the planes an FV state uses
SLOPES = [1, 2, 4, 5, 7, 8]


def _binding():
    from paper_2010_02003_gb300 import binding
    return binding


def avg_err(a, b, g=9.80665):
    """max |a - b| over the average planes, relative to max|h0| (depth) and to
    max(max|q0|, max|h0| sqrt(g max|h0|)) (discharges)."""
    a = a.reshape(9, -1)
    b = b.reshape(9, -1)
    hs = max(np.abs(b[0]).max(), 1e-30)
    qs = max(np.abs(b[3]).max(), np.abs(b[6]).max(), hs * np.sqrt(g * hs))
    return max(np.abs(a[0] - b[0]).max() / hs, np.abs(a[3] - b[3]).max() / qs,
               np.abs(a[6] - b[6]).max() / qs)


def pair(case, scheme, flux="hll", **kw):
    B = _binding()
    o = make_oracle(case, scheme=scheme, flux=flux)
    s = B.solver_from_case(case, scheme=B.DG2_SCHEME_FV2 if scheme == "fv2" else B.DG2_SCHEME_FV1,
                           flux=B.DG2_ROE if flux == "roe" else B.DG2_HLL, **kw)
    return s, o


CASES = {
    "hump_dam_128": lambda: inputs.hump(eta=0.5, dam_eta=1.0),
    "hump_still_128": lambda: inputs.hump(eta=0.5),
    "terrain_77x53": lambda: inputs.random_terrain(77, 53, seed=5),
    "blocks_48x40": lambda: inputs.wall_blocks(),
    "floodplain_dry_96x64": lambda: inputs.floodplain(nx=96, ny=64, dx=2.0, q_peak=15.0,
                                                      t_peak=20.0, channel_width=12.0),
}


def _sensitivity(case, scheme, state, t, dt, flux="hll", seeds=3):
    """How far the oracle's own step moves when its input averages are perturbed by
    2e-16 of each variable's scale (max over a few seeds, in avg_err units)."""
    hs = np.abs(state[0]).max()
    qs = max(np.abs(state[3]).max(), np.abs(state[6]).max())
    scale = np.array([hs] * 3 + [qs] * 6)[:, None, None]
    ref = make_oracle(case, scheme=scheme, flux=flux)
    ref.set_state(state, t)
    ref.step(dt)
    base = ref.state()
    worst = 0.0
    for sd in range(seeds):
        rng = np.random.default_rng(sd)
        tw = make_oracle(case, scheme=scheme, flux=flux)
        tw.set_state(state + rng.standard_normal(state.shape) * 2e-16 * scale * (state != 0), t)
        tw.step(dt)
        worst = max(worst, avg_err(tw.state(), base))
    return worst


@pytest.mark.parametrize("scheme", ["fv2", "fv1"])
@pytest.mark.parametrize("name", list(CASES))
def test_fv_forced_dt_100_steps(name, scheme):
    case = CASES[name]()
    s, o = pair(case, scheme)
    assert avg_err(s.state(), o.state()) <= TOL
    for _ in range(100):
        s.step(o.step())
    st = s.state().reshape(9, -1)
    assert avg_err(st, o.state()) <= TOL
    assert np.abs(st[SLOPES]).max() == 0.0
    t_gpu, _ = s.time()
    assert abs(t_gpu - o.t) <= 1e-12 * o.t
    m, led = s.mass()
    assert abs(m - o.mass()) <= 1e-12 * abs(o.mass())
    assert abs(led - o.ledger()) <= 1e-12 * abs(o.ledger())


@pytest.mark.parametrize("scheme", ["fv2", "fv1"])
@pytest.mark.parametrize("name", list(CASES))
def test_fv_step_parity_along_oracle_trajectory(name, scheme):
    case = CASES[name]()
    s, o = pair(case, scheme)
    for k in range(100):
        st0, t0 = o.state(), o.t
        s.set_state(st0, t0)
        dt = o.step()
        s.step(dt)
        err = avg_err(s.state(), o.state())
        if err > TOL:
            sens = _sensitivity(case, scheme, st0, t0, dt)
            assert sens > 1e-14 and err <= 100.0 * sens, (k, err, sens)


@pytest.mark.parametrize("scheme", ["fv2", "fv1"])
def test_fv_self_dt(scheme):
    case = inputs.hump(eta=0.5, dam_eta=1.0)
    s, o = pair(case, scheme)
    odt, gdt = [], []
    for _ in range(100):
        odt.append(o.step())
        gdt.append(s.step(-1.0, want_dt=True))
    assert np.abs(np.array(gdt) - np.array(odt)).max() <= 1e-12 * max(odt)
    assert avg_err(s.state(), o.state()) <= TOL


@pytest.mark.parametrize("scheme", ["fv2", "fv1"])
def test_fv_sources_rain_and_point_inflow(scheme):
    """Rain that stops inside the run and a point inflow: the ledger of FV1 counts the
    rain of the step's start only (one forward-Euler stage)."""
    case = inputs.hump(nx=70, ny=45, eta=0.5)
    case.rain = (2e-3, 0.0, 0.6)
    case.point = (20.5, 10.5, 0.5)
    s, o = pair(case, scheme)
    for _ in range(60):
        s.step(o.step())
    assert avg_err(s.state(), o.state()) <= TOL
    m, led = s.mass()
    assert abs(m - led) <= 1e-12 * m
    assert abs(led - o.ledger()) <= 1e-12 * o.ledger()


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (41, 1), (33, 9), (31, 7), (65, 17)])
def test_fv_degenerate_and_ragged_grids(shape):
    nx, ny = shape
    case = inputs.random_terrain(nx, ny, seed=nx * 100 + ny, relief=0.5)
    for scheme in ("fv2", "fv1"):
        s, o = pair(case, scheme)
        for _ in range(40):
            s.step(o.step())
        assert avg_err(s.state(), o.state()) <= TOL


@pytest.mark.parametrize("scheme", ["fv2", "fv1"])
def test_fv_dry_tile_skipping_is_exact(scheme):
    """Skipping still, dry tiles leaves every bit of the FV result unchanged."""
    case = inputs.floodplain(nx=200, ny=120, dx=2.0, q_peak=15.0, t_peak=20.0,
                             channel_width=12.0)
    B = _binding()
    sch = B.DG2_SCHEME_FV2 if scheme == "fv2" else B.DG2_SCHEME_FV1
    a = B.solver_from_case(case, scheme=sch, skip_dry_tiles=True)
    b = B.solver_from_case(case, scheme=sch, skip_dry_tiles=False)
    for _ in range(150):
        dt = a.step(-1.0, want_dt=True)
        b.step(dt)
    assert np.array_equal(a.state(), b.state())
    nt, _, _, done = a.tile_stats()
    assert done < 150 * nt                    # tiles were skipped


def test_fv2_with_roe_flux():
    case = inputs.hump(eta=0.5, dam_eta=1.0)
    s, o = pair(case, "fv2", flux="roe")
    for _ in range(100):
        s.step(o.step())
    assert avg_err(s.state(), o.state()) <= TOL


def test_fv_full_size_floodplain_first_steps():
    """The 2000 x 1000 (2 m) floodplain from its channel start, FV2: 6 forced steps
    against the oracle, every cell compared."""
    case = inputs.floodplain(initial="channel")
    s, o = pair(case, "fv2")
    for _ in range(6):
        s.step(o.step())
    assert avg_err(s.state(), o.state()) <= TOL


def test_fv_parameter_rules():
    B = _binding()
    for kw in ({"precision": B.DG2_FP32}, {"variant": B.DG2_LL}, {"scheme": 3}):
        with pytest.raises(B.Dg2Error) as e:
            B.Solver(16, 16, 1.0, scheme=kw.pop("scheme", B.DG2_SCHEME_FV2), **kw)
        assert e.value.code == B.DG2_E_ARG
