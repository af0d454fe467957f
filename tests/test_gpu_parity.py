"""GPU path (through the C ABI) against the FP64 oracle.

Bar (FP64): for every one of the 9 coefficient planes,
    max|gpu - oracle| / (scale of the plane's variable) <= 1e-12
after 100 steps with the oracle's time-step sequence forced on the GPU, and
the self-computed Courant steps agree to 1e-12 relative.  The GPU evaluates
the same formulas in another order (fused multiply-adds, one face flux per
tile, reciprocal-free divisions kept), so agreement is to round-off, not bits.

Every case runs under both face revisions: the revision of Sec. 2.1.2 as
printed (h* = max(0, h), z* = z - max(0, -h); DG2_WD_PRINTED against the
oracle's wetdry="paper") and the positivity-consistent revision of partially
wet cells that is the library's default (DG2_WD_POSITIVE, wetdry="positive").
"""
import numpy as np
import pytest

from conftest import make_oracle
from paper_2010_02003_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _binding():
    from paper_2010_02003_gb300 import binding
    return binding


def plane_err(a, b, g=9.80665):
    """Per-plane max |a - b| relative to the scale of the plane's variable: max|h0| for
    the three h modes, max(max|q0|, max|h0| sqrt(g max|h0|)) for the discharge modes
    (a still lake's discharges are pure round-off, so their own maximum is no scale)."""
    a = a.reshape(9, -1)
    b = b.reshape(9, -1)
    hs = max(np.abs(b[0]).max(), 1e-30)
    qs = max(np.abs(b[3]).max(), np.abs(b[6]).max(), hs * np.sqrt(g * hs))
    scale = np.array([hs] * 3 + [qs] * 6)
    return np.abs(a - b).max(axis=1) / scale


def run_pair(case, limiter, nsteps, forced=True, wetdry="positive"):
    B = _binding()
    o = make_oracle(case, limiter=limiter, wetdry=wetdry)
    s = B.solver_from_case(case, variant=B.DG2_LL if limiter else B.DG2_NL,
                           wetdry=B.DG2_WD_POSITIVE if wetdry == "positive" else B.DG2_WD_PRINTED)
    # initial state and topography agree before any step
    assert plane_err(s.state(), o.state()).max() <= TOL
    gpu_dts, orc_dts = [], []
    for _ in range(nsteps):
        dt = o.step()
        orc_dts.append(dt)
        if forced:
            s.step(dt)
        else:
            gpu_dts.append(s.step(-1.0, want_dt=True))
    return s, o, np.array(orc_dts), np.array(gpu_dts)


CASES = {
    "hump_dam_128": lambda: inputs.hump(eta=0.5, dam_eta=1.0),
    "hump_still_128": lambda: inputs.hump(eta=0.5),
    "terrain_77x53": lambda: inputs.random_terrain(77, 53, seed=5),
    "blocks_48x40": lambda: inputs.wall_blocks(),
    # the floodplain recipe from its specified dry start, inflow hydrograph sped up
    "floodplain_dry_96x64": lambda: inputs.floodplain(nx=96, ny=64, dx=2.0, q_peak=15.0,
                                                      t_peak=20.0, channel_width=12.0),
}


WETDRY = ["paper", "positive"]
WD_IDS = ["printed", "positive"]

# Free-running horizon: 100 steps, except where the oracle's own trajectory
# amplifies round-off past the bar.  Measured by running the oracle twice, the
# second time from a state 2e-16 away (tests/test_oracle_conditioning.py): on the
# floodplain's dry start the thin channel front lifts that difference from ~2e-15
# at step 90 to 2e-11 (DG2-NL) / 6e-10 (DG2-LL) at step 100 under the default
# revision, and to 7e-12 at step 100 (DG2-LL) under the printed one, so no
# implementation with another rounding order can hold 1e-12 there.  Those runs
# are held over 85 / 90 steps, and every one of their 100 steps is checked from
# the oracle's own state below.
HORIZON = {("floodplain_dry_96x64", False, "positive"): 85,
           ("floodplain_dry_96x64", True, "positive"): 85,
           ("floodplain_dry_96x64", True, "paper"): 90}


@pytest.mark.parametrize("wetdry", WETDRY, ids=WD_IDS)
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
@pytest.mark.parametrize("name", list(CASES))
def test_parity_forced_dt_100_steps(name, limiter, wetdry):
    case = CASES[name]()
    s, o, _, _ = run_pair(case, limiter, HORIZON.get((name, limiter, wetdry), 100),
                          wetdry=wetdry)
    err = plane_err(s.state(), o.state())
    assert err.max() <= TOL, dict(enumerate(err))
    t_gpu, _ = s.time()
    assert abs(t_gpu - o.t) <= 1e-12 * o.t
    m, led = s.mass()
    assert abs(m - o.mass()) <= 1e-12 * abs(o.mass())
    assert abs(led - o.ledger()) <= 1e-12 * abs(o.ledger())


def _wd(B, wetdry):
    return B.DG2_WD_POSITIVE if wetdry == "positive" else B.DG2_WD_PRINTED


@pytest.mark.parametrize("wetdry", WETDRY, ids=WD_IDS)
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
@pytest.mark.parametrize("name", list(CASES))
def test_step_parity_along_oracle_trajectory(name, limiter, wetdry):
    """Each of 100 steps starts on the GPU from the oracle's own state and time and
    must land within 1e-12 of the oracle's step: the per-step arithmetic of every
    step of the run, without the round-off amplification of a long free run."""
    case = CASES[name]()
    B = _binding()
    o = make_oracle(case, limiter=limiter, wetdry=wetdry)
    s = B.solver_from_case(case, variant=B.DG2_LL if limiter else B.DG2_NL,
                           wetdry=_wd(B, wetdry))
    worst = 0.0
    for _ in range(100):
        s.set_state(o.state(), o.t)
        dt = o.step()
        s.step(dt)
        worst = max(worst, plane_err(s.state(), o.state()).max())
        m, _ = s.mass()
        assert abs(m - o.mass()) <= 1e-12 * abs(o.mass())
    assert worst <= TOL


@pytest.mark.parametrize("wetdry", WETDRY, ids=WD_IDS)
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_parity_self_dt(limiter, wetdry):
    case = inputs.hump(eta=0.5, dam_eta=1.0)
    s, o, odt, gdt = run_pair(case, limiter, 100, forced=False, wetdry=wetdry)
    assert np.abs(gdt - odt).max() <= 1e-12 * odt.max()
    assert plane_err(s.state(), o.state()).max() <= TOL


@pytest.mark.parametrize("wetdry", WETDRY, ids=WD_IDS)
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_violent_channel_start(limiter, wetdry):
    """Water dropped into the incised channel (not at rest) drains down steep banks into
    thin films.  Under the printed revision the partially wet bank cells amplify
    round-off (two oracle runs 2e-16 apart: 7e-13 (NL) / 3e-14 (LL) at step 70, 5e-12 /
    5e-13 at step 80), so the bar is held over 50 steps there; under the default
    revision the twin runs stay within 2e-14 over 100 steps, which are held."""
    case = inputs.floodplain(nx=96, ny=64, dx=2.0, q_peak=15.0, t_peak=60.0, initial="channel",
                             channel_width=12.0)
    s, o, _, _ = run_pair(case, limiter, 50 if wetdry == "paper" else 100, wetdry=wetdry)
    assert plane_err(s.state(), o.state()).max() <= TOL


@pytest.mark.parametrize("wetdry", WETDRY, ids=WD_IDS)
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_run_to_with_gauges_matches_oracle(limiter, wetdry):
    case = inputs.hump(eta=0.5, dam_eta=1.0)
    case.gauges = np.array([[64.0, 64.0], [30.5, 64.0], [64.0, 97.25], [10.0, 10.0], [100.2, 40.7]])
    case.sample_every = 0.75
    B = _binding()
    o = make_oracle(case, limiter=limiter, wetdry=wetdry)
    s = B.solver_from_case(case, variant=B.DG2_LL if limiter else B.DG2_NL,
                           wetdry=_wd(B, wetdry))
    steps_o, t_o, h_o = o.run_to(6.0, case.sample_every, case.gauges)
    steps_g = s.run_to(6.0)
    t_g, h_g, overflow = s.read_gauges()
    assert not overflow
    assert steps_g == steps_o
    assert np.array_equal(t_g, t_o)                     # landings are exact assignments
    assert np.abs(h_g - h_o).max() <= TOL * max(np.abs(h_o).max(), 1e-30)
    assert s.time()[0] == 6.0
    assert plane_err(s.state(), o.state()).max() <= TOL
    # a second run_to continues the sample sequence
    steps_o2, t_o2, h_o2 = o.run_to(10.0, case.sample_every, case.gauges)
    assert s.run_to(10.0) == steps_o2
    t_g2, h_g2, _ = s.read_gauges()
    assert np.array_equal(t_g2, t_o2)
    assert np.abs(h_g2 - h_o2).max() <= TOL * max(np.abs(h_o2).max(), 1e-30)
    assert plane_err(s.state(), o.state()).max() <= TOL


def test_run_to_lands_on_samples_and_keeps_the_ledger():
    """GPU-only properties of run_to on the floodplain: sample rows at exact multiples of
    the interval, t lands on t_end, the mass matches the ledger."""
    case = inputs.floodplain(nx=120, ny=60, dx=2.0, q_peak=10.0, t_peak=30.0, initial="channel",
                             channel_width=12.0, ngauge=6, sample_every=2.5)
    B = _binding()
    s = B.solver_from_case(case)
    n = s.run_to(30.0)
    t, h, overflow = s.read_gauges()
    assert n > 0 and not overflow
    assert np.array_equal(t, 2.5 * np.arange(1, 13))
    assert h.shape == (12, 6) and np.isfinite(h).all() and (h >= 0).all()
    assert s.time()[0] == 30.0
    m, led = s.mass()
    assert abs(m - led) <= 1e-12 * m


@pytest.mark.parametrize("wetdry", WETDRY, ids=WD_IDS)
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_sources_rain_and_point_inflow(limiter, wetdry):
    case = inputs.hump(nx=70, ny=45, eta=0.5)
    case.rain = (2e-3, 0.0, 0.6)
    case.point = (20.5, 10.5, 0.5)
    s, o, _, _ = run_pair(case, limiter, 60, wetdry=wetdry)
    assert plane_err(s.state(), o.state()).max() <= TOL
    m, led = s.mass()
    assert abs(m - led) <= 1e-12 * m
    assert abs(led - o.ledger()) <= 1e-12 * o.ledger()


@pytest.mark.parametrize("wetdry", WETDRY, ids=WD_IDS)
@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (41, 1), (33, 9), (31, 7), (65, 17)])
def test_degenerate_and_ragged_grids(shape, wetdry):
    nx, ny = shape
    case = inputs.random_terrain(nx, ny, seed=nx * 100 + ny, relief=0.5)
    for limiter in (False, True):
        s, o, _, _ = run_pair(case, limiter, 40, wetdry=wetdry)
        assert plane_err(s.state(), o.state()).max() <= TOL


def test_all_dry_grid_takes_dt_max_and_stays_dry():
    case = inputs.hump(nx=40, ny=24, eta=-1.0)          # free surface below the bed everywhere
    B = _binding()
    s = B.solver_from_case(case)
    assert np.abs(s.state()).max() == 0.0
    for _ in range(5):
        assert s.step(-1.0, want_dt=True) == 1.0         # dt_max
    assert np.abs(s.state()).max() == 0.0


@pytest.mark.parametrize("wetdry", WETDRY, ids=WD_IDS)
def test_full_size_floodplain_first_steps(wetdry):
    """The 2000 x 1000 (2 m) floodplain at full size, in the launch configuration the
    benchmark times: 6 forced steps against the oracle, every cell compared."""
    case = inputs.floodplain(initial="channel")
    s, o, _, _ = run_pair(case, False, 6, wetdry=wetdry)
    assert plane_err(s.state(), o.state()).max() <= TOL


def test_bad_arguments_are_rejected_on_the_host():
    B = _binding()
    import torch
    p = B.dg2_default_params()
    ws = torch.empty(B.dg2_workspace_bytes(8, 8, p) + 256, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_init_grid(8, 8, -1.0, 1.0, p, base, ws.numel() - 256, 0)
    assert e.value.code == B.DG2_E_ARG
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_init_grid(8, 8, 1.0, 1.0, p, base, 16, 0)
    assert e.value.code == B.DG2_E_NOMEM
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_init_grid(8, 8, 1.0, 1.0, p, base + 8, ws.numel() - 256, 0)
    assert e.value.code == B.DG2_E_ARG
    ctx = B.dg2_init_grid(8, 8, 1.0, 1.0, p, base, ws.numel() - 256, 0)
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_step(ctx, -1.0)
    assert e.value.code == B.DG2_E_STATE                 # no DEM yet
    z = np.zeros((9, 9))
    z[3, 3] = np.nan
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_set_dem(ctx, z)
    assert e.value.code == B.DG2_E_ARG
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_set_bc_inflow(ctx, 0, 100.0, 5.0, [0.0, 1.0], [1.0, 1.0])   # segment off the edge
    assert e.value.code == B.DG2_E_ARG
    B.dg2_destroy(ctx)


@pytest.mark.parametrize("wetdry", WETDRY, ids=WD_IDS)
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_urban_recipe_small(limiter, wetdry):
    """The urban recipe (buildings, roads, rain, point inflow) on a 192 x 160 grid."""
    case = inputs.urban(nx=192, ny=160, dx=0.5, nblocks=30)
    s, o, _, _ = run_pair(case, limiter, 100, wetdry=wetdry)
    assert plane_err(s.state(), o.state()).max() <= TOL
    m, led = s.mass()
    assert abs(m - led) <= 1e-12 * m


ROE_CASES = {
    "hump_dam_128": lambda: inputs.hump(eta=0.5, dam_eta=1.0),
    "terrain_77x53": lambda: inputs.random_terrain(77, 53, seed=5),
    "blocks_48x40": lambda: inputs.wall_blocks(),
    "floodplain_dry_96x64": lambda: inputs.floodplain(nx=96, ny=64, dx=2.0, q_peak=15.0,
                                                      t_peak=20.0, channel_width=12.0),
}


def _oracle_step_sensitivity(case, limiter, state, t, dt, seeds=3):
    """How far the oracle's own step moves when its input state is perturbed by
    2e-16 of each variable's scale (max over a few seeds, in plane_err units): the
    part of a GPU difference that rounding order alone explains."""
    hs = np.abs(state[0]).max()
    qs = max(np.abs(state[3]).max(), np.abs(state[6]).max())
    scale = np.array([hs] * 3 + [qs] * 6)[:, None, None]
    ref = make_oracle(case, limiter=limiter, flux="roe")
    ref.set_state(state, t)
    ref.step(dt)
    base = ref.state()
    worst = 0.0
    for sd in range(seeds):
        rng = np.random.default_rng(sd)
        tw = make_oracle(case, limiter=limiter, flux="roe")
        tw.set_state(state + rng.standard_normal(state.shape) * 2e-16 * scale * (state != 0), t)
        tw.step(dt)
        worst = max(worst, plane_err(tw.state(), base).max())
    return worst


@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
@pytest.mark.parametrize("name", list(ROE_CASES))
def test_roe_step_parity_along_oracle_trajectory(name, limiter):
    """The Roe flux option: each of 60 steps from the oracle's own state within
    1e-12, or, on a step whose result the oracle itself moves by more than 1e-14
    under a 2e-16 perturbation of its input (thin films at a wet-dry front, where
    q/h amplifies rounding), within 3 times that sensitivity (measured at most
    0.86 times, DG2-LL on the 77x53 terrain; every other case within 1e-12)."""
    case = ROE_CASES[name]()
    B = _binding()
    o = make_oracle(case, limiter=limiter, flux="roe")
    s = B.solver_from_case(case, variant=B.DG2_LL if limiter else B.DG2_NL, flux=B.DG2_ROE)
    worst = 0.0
    for k in range(60):
        st0, t0 = o.state(), o.t
        s.set_state(st0, t0)
        dt = o.step()
        s.step(dt)
        err = plane_err(s.state(), o.state()).max()
        if err > TOL:
            sens = _oracle_step_sensitivity(case, limiter, st0, t0, dt)
            worst = max(worst, err / sens)
            assert sens > 1e-14 and err <= 3.0 * sens, (k, err, sens)
    print(f"Roe {name} {'LL' if limiter else 'NL'}: worst error / oracle sensitivity {worst:.3g}")


@pytest.mark.parametrize("name", ["hump_dam_128", "blocks_48x40"])
def test_roe_free_run_100_steps(name):
    case = ROE_CASES[name]()
    B = _binding()
    o = make_oracle(case, limiter=True, flux="roe")
    s = B.solver_from_case(case, variant=B.DG2_LL, flux=B.DG2_ROE)
    for _ in range(100):
        s.step(o.step())
    assert plane_err(s.state(), o.state()).max() <= TOL
    m, led = s.mass()
    assert abs(m - o.mass()) <= 1e-12 * o.mass()


def test_roe_is_fp64_only():
    B = _binding()
    with pytest.raises(B.Dg2Error) as e:
        B.Solver(16, 16, 1.0, precision=B.DG2_FP32, flux=B.DG2_ROE)
    assert e.value.code == B.DG2_E_ARG


@pytest.mark.parametrize("wetdry", ["positive", "paper"])
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_planar_basin_at_rest(limiter, wetdry):
    """Still water in a basin whose bed rises 2 m across a cell, the surface crossing
    cells above their centres (partially wet cells on every side): at rest to
    round-off on the GPU, and equal to the oracle."""
    case = inputs.diamond_basin(level=16.5)
    s, o, _, _ = run_pair(case, limiter, 100, wetdry=wetdry)
    st = s.state()
    assert np.abs(st[3:]).max() <= 1e-12
    assert plane_err(st, o.state()).max() <= TOL


@pytest.mark.parametrize("wetdry", WETDRY, ids=WD_IDS)
def test_bench_workload_sampled_windows(wetdry):
    """The benchmark's workload in its launch configuration: the 2000 x 1000 (2 m)
    floodplain, DG2-LL, FP64, tile and warp-block skipping on, stepped once from a
    wet, flowing state (FP32 run from the channel start to t = 600 s).  A full-size
    oracle step takes minutes, so the oracle steps 48 x 48 windows cut around sampled
    wet cells with the GPU's dt; a step reads 4 cells around each cell (2 per stage,
    friction is pointwise), so window cells 6 or more cells from the cut must agree
    with the GPU's full-grid step.  Both face revisions step from the same state."""
    import oracle
    B = _binding()
    case = inputs.floodplain(initial="channel")
    warm = B.solver_from_case(case, variant=B.DG2_LL, precision=B.DG2_FP32)
    warm.run_to(600.0)
    st, t = warm.state(), warm.time()[0]
    warm.close()
    s = B.solver_from_case(case, variant=B.DG2_LL, wetdry=_wd(B, wetdry))
    s.set_state(st, t)
    dt = s.step(-1.0, want_dt=True)
    out = s.state()
    W, M = 48, 6
    hs = np.abs(out[0]).max()
    qs = max(np.abs(out[3]).max(), np.abs(out[6]).max(), hs * np.sqrt(9.80665 * hs))
    scale = np.array([hs] * 3 + [qs] * 6)[:, None, None]
    wet = np.argwhere(st[0] > 1e-5)
    wet = wet[(wet[:, 0] >= W) & (wet[:, 0] < case.ny - W) & (wet[:, 1] >= W) &
              (wet[:, 1] < case.nx - W)]
    assert len(wet) > 1000
    rng = np.random.default_rng(11)
    for j, i in wet[rng.choice(len(wet), 8, replace=False)]:
        j0, i0 = j - W // 2, i - W // 2
        o = oracle.Oracle(W, W, case.dx, case.dy, cfl=case.cfl, limiter=True,
                          dt_max=case.dt_max, wetdry=wetdry)
        man = None if case.manning is None else case.manning[j0:j0 + W, i0:i0 + W]
        o.set_dem(case.z_corner[j0:j0 + W + 1, i0:i0 + W + 1], man, case.n_uniform)
        o.set_state(st[:, j0:j0 + W, i0:i0 + W], t)
        o.step(dt)
        a = out[:, j0 + M:j0 + W - M, i0 + M:i0 + W - M]
        b = o.state()[:, M:W - M, M:W - M]
        err = (np.abs(a - b) / scale).max()
        assert err <= TOL, (j, i, err)
