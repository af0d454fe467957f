"""Ensembles (dg2_ens_*): FP32 members advanced together, each with its own time
step, through the C ABI.  Every member must end bit for bit where the same member
run alone ends (its states, time and step size), whatever the tile shape; the
autotuner must pick one of the shapes after timing each; the mass ledger holds."""
import numpy as np
import pytest

from paper_2010_02003_gb300 import inputs

pytestmark = pytest.mark.gpu


def _B():
    from paper_2010_02003_gb300 import binding
    return binding


def _cases(n=6, seed=77):
    # small members of the ensemble recipe: sizes, roughness and inflows all differ
    return inputs.ensemble(n=n, seed=seed, nx_range=(40, 160), ny_range=(24, 96), t_peak=60.0,
                           t_end=120.0, sample_every=5.0)


def _members(cases, variant):
    B = _B()
    return [B.solver_from_case(c, variant=variant, precision=B.DG2_FP32) for c in cases]


def _solo(cases, variant, t_end):
    out = []
    for s in _members(cases, variant):
        s.run_to(t_end)
        out.append((s.state(), s.time(), s.read_gauges()))
    return out


@pytest.mark.parametrize("variant", [0, 1], ids=["NL", "LL"])
def test_members_match_solo_runs_bit_for_bit(variant):
    B = _B()
    cases = _cases()
    solo = _solo(cases, variant, 40.0)
    mem = _members(cases, variant)
    ens = B.Ensemble(mem)
    steps = ens.run_to(40.0)
    assert steps > 0
    for k, s in enumerate(mem):
        st, tm, gauges = solo[k]
        assert np.array_equal(s.state(), st), k
        assert s.time() == tm, k                    # same t (landed) and same pending dt
        t_g, h_g, _ = s.read_gauges()
        assert np.array_equal(t_g, gauges[0]) and np.array_equal(h_g, gauges[1]), k
        m, led = s.mass()
        assert abs(m - led) <= 1e-6 * max(led, 1.0), k
    # a second leg continues every member exactly as a solo run_to would
    solo2 = []
    for s in _members(cases, variant):
        s.run_to(40.0)
        s.run_to(70.0)
        solo2.append(s.state())
    ens.run_to(70.0)
    for k, s in enumerate(mem):
        assert np.array_equal(s.state(), solo2[k]), k
        assert s.time()[0] == 70.0


def test_every_tile_shape_gives_the_same_members():
    B = _B()
    cases = _cases(n=4, seed=91)
    ref = None
    for shape in [(32, 8), (32, 4), (16, 8), (64, 4), (16, 16)]:
        mem = _members(cases, B.DG2_LL)
        ens = B.Ensemble(mem)
        ens.set_tile_shape(*shape)
        assert ens.tile_shape() == shape
        ens.run_to(30.0)
        states = [s.state() for s in mem]
        if ref is None:
            ref = states
        for a, b in zip(states, ref):
            assert np.array_equal(a, b), shape
        ens.close()


def test_autotune_times_every_shape_and_keeps_results_exact():
    B = _B()
    cases = _cases(n=5, seed=123)
    solo = _solo(cases, B.DG2_NL, 50.0)
    mem = _members(cases, B.DG2_NL)
    ens = B.Ensemble(mem)
    w, h = ens.autotune(50.0, steps_per_trial=8)
    assert (w, h) in [(32, 8), (32, 4), (16, 8), (64, 4), (16, 16)]
    assert ens.tile_shape() == (w, h)
    ms = ens.tune_times()
    assert len(ms) == 5 and (ms > 0).all()
    assert ms[[(32, 8), (32, 4), (16, 8), (64, 4), (16, 16)].index((w, h))] == ms.min()
    ens.run_to(50.0)
    for k, s in enumerate(mem):
        assert np.array_equal(s.state(), solo[k][0]), k
        assert s.time() == solo[k][1], k


def test_members_with_different_time_steps_all_land():
    """Members differ in dx (and so in dt); each lands on t_end with its own step
    count, and a member already at t_end does not move."""
    B = _B()
    cases = _cases(n=3, seed=5)
    # a member with four times smaller cells (and steps)
    cases[1] = inputs.floodplain(nx=60, ny=40, dx=0.5, q_peak=5.0, t_peak=60.0, t_end=120.0,
                                 ngauge=2, sample_every=5.0)
    mem = _members(cases, B.DG2_NL)
    mem[2].run_to(25.0)
    before = mem[2].state()
    ens = B.Ensemble(mem)
    ens.run_to(25.0)
    assert np.array_equal(mem[2].state(), before)
    for s in mem:
        assert s.time()[0] == 25.0
    n0 = mem[0].tile_stats()[3]
    assert n0 >= 0


def test_members_step_alone_after_the_ensemble():
    B = _B()
    cases = _cases(n=2, seed=8)
    mem = _members(cases, B.DG2_NL)
    ens = B.Ensemble(mem)
    ens.run_to(20.0)
    solo = _members(cases, B.DG2_NL)
    for s in solo:
        s.run_to(20.0)
    for a, b in zip(mem, solo):
        for _ in range(5):
            a.step(-1.0)
            b.step(-1.0)
        assert np.array_equal(a.state(), b.state())


def test_ensemble_arguments_are_checked():
    B = _B()
    cases = _cases(n=2, seed=9)
    f64 = B.solver_from_case(cases[0], precision=B.DG2_FP64)
    a, b = _members(cases, B.DG2_NL)
    ll = B.solver_from_case(cases[1], variant=B.DG2_LL, precision=B.DG2_FP32)
    assert B.dg2_ens_workspace_bytes([f64.ctx]) == 0
    for bad in ([a.ctx, f64.ctx], [a.ctx, ll.ctx], [a.ctx, a.ctx]):
        with pytest.raises(B.Dg2Error) as e:
            B.dg2_ens_create(bad, 0, 0, 0)
        assert e.value.code == B.DG2_E_ARG
    ens = B.Ensemble([a, b])
    with pytest.raises(B.Dg2Error):
        ens.set_tile_shape(8, 8)
    with pytest.raises(B.Dg2Error):
        ens.autotune(10.0, steps_per_trial=2)


def _fp32_errors(gpu, orc, g=9.80665):
    hs = max(np.abs(orc[0]).max(), 1e-30)
    qs = max(np.abs(orc[3]).max(), np.abs(orc[6]).max(), hs * np.sqrt(g * hs))
    return np.abs(gpu[:3] - orc[:3]).max() / hs, np.abs(gpu[3:] - orc[3:]).max() / qs


def _solo_dt_sequence(B, case, variant, t_end):
    """The Courant steps a member takes alone up to t_end, found by stepping an FP32 twin
    with dg2_step: each step the pending Courant step, the last one landing on t_end (the
    rule of dg2_run_to, which the ensemble follows for every member)."""
    s = B.solver_from_case(case, variant=variant, precision=B.DG2_FP32)
    dts = []
    while True:
        t, dt_next = s.time()
        if t + dt_next >= t_end:
            dts.append(t_end - t)
            s.step(t_end - t)
            break
        dts.append(s.step(-1.0, want_dt=True))
    st = s.state()
    s.close()
    return np.array(dts), st


# FP32 member error against the FP64 oracle over each member's own step sequence
# (depth / discharge, relative to the member's depth and discharge scales): measured
# NL 4.9e-6 / 2.2e-6, LL 4.2e-6 / 1.8e-6 at most over the six members; bars at 3x.
ENS_BAR = {0: (1.5e-5, 7e-6), 1: (1.3e-5, 6e-6)}


@pytest.mark.parametrize("variant", [0, 1], ids=["NL", "LL"])
def test_uneven_members_against_the_fp64_oracle(variant):
    """Six members of uneven sizes (33 x 17 to 96 x 64 cells), each with its own Manning
    n, inflow peak and Courant steps, advanced together to t = 8 s (37 to 51 steps); every
    member is compared with the FP64 oracle run alone through that member's own step
    sequence (the FP32 steps it takes alone, which the ensemble reproduces bit for bit).
    The window is where the members' dry-start inflow fronts are well conditioned: the
    oracle moves by 8e-8 there under a 1e-7 perturbation of its state, but by 0.2-0.6
    over 30 s, where FP32 and FP64 runs part at wet-dry decisions
    (tests/test_oracle_conditioning.py)."""
    from conftest import make_oracle
    B = _B()
    t_end = 8.0
    cases = inputs.ensemble(n=6, seed=4242, nx_range=(33, 96), ny_range=(17, 64), t_peak=3.0,
                            t_end=t_end, ngauge=2, sample_every=0.0)
    sizes = {(c.nx, c.ny) for c in cases}
    assert len(sizes) == 6
    mem = _members(cases, variant)
    ens = B.Ensemble(mem)
    ens.run_to(t_end)
    worst = (0.0, 0.0)
    nsteps = []
    for k, (case, s) in enumerate(zip(cases, mem)):
        dts, solo = _solo_dt_sequence(B, case, variant, t_end)
        got = s.state()
        assert np.array_equal(got, solo), k                # ensemble == the member alone
        assert s.time()[0] == t_end
        o = make_oracle(case, limiter=bool(variant))
        for dt in dts:
            o.step(dt)
        nsteps.append(len(dts))
        eh, eq = _fp32_errors(got, o.state())
        worst = (max(worst[0], eh), max(worst[1], eq))
        assert np.abs(o.state()[0]).max() > 1e-3, k        # water has entered the member
        m, led = s.mass()
        assert abs(m - led) <= 1e-6 * max(led, 1.0), k
    assert len(set(nsteps)) > 1                            # the members' steps differ
    print(f"ensemble members vs FP64 oracle ({'LL' if variant else 'NL'}): depth {worst[0]:.2e}, "
          f"discharge {worst[1]:.2e}, steps {nsteps}")
    bh, bq = ENS_BAR[variant]
    assert worst[0] < bh and worst[1] < bq, worst
