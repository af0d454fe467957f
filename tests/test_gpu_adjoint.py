"""Discrete adjoint of the FP64 DG2-NL step (dg2_adj_*) through the C ABI.

Checked against: the oracle's forward (misfit and sampled depths to 1e-12), the
oracle's own taped derivatives (tests/test_oracle_tape.py pins the tape against
its finite differences), central finite differences of the GPU forward, and
itself under every number of checkpoint slots (the gradient must not change a
bit).  The wet-dry, revision, HLL-regime and ghost branches are frozen from the
forward state, as the tape's are.  Both face revisions are checked (the default and
the printed one, the oracle's wetdry="positive" / "paper"); this channel case has
partially wet bank cells, where they differ."""
import numpy as np
import pytest

from paper_2010_02003_gb300 import inputs

pytestmark = pytest.mark.gpu


def _case():
    return inputs.floodplain(nx=14, ny=10, dx=2.0, q_peak=5.0, t_peak=20.0, t_end=60.0,
                             channel_width=8.0, inflow_len=8.0, ngauge=3, sample_every=5.0,
                             initial="channel")


DTS = np.full(30, 0.05)
SAMPLES = [10, 20, 30]
OBS = np.full((3, 3), 0.3)


WD = ["positive", "paper"]


def _setup(nsnap=8, wetdry="positive"):
    from paper_2010_02003_gb300 import binding as B
    case = _case()
    rng = np.random.default_rng(1)
    man = 0.03 + 0.02 * rng.random((case.ny, case.nx))
    case.manning = man
    a = B.Adjoint(case, nsnap=nsnap, max_steps=64,
                  wetdry=B.DG2_WD_POSITIVE if wetdry == "positive" else B.DG2_WD_PRINTED)
    a.set_schedule(DTS, SAMPLES, OBS)
    return case, man, a


@pytest.mark.parametrize("wetdry", WD)
def test_adjoint_forward_matches_the_oracle(wetdry):
    from conftest import make_oracle
    case, man, a = _setup(wetdry=wetdry)
    J, h = a.forward()
    o = make_oracle(case, wetdry=wetdry)
    hs = []
    for k in range(1, len(DTS) + 1):
        o.step(DTS[k - 1])
        if k in SAMPLES:
            hs.append([o.gauge_h(x, y) for x, y in case.gauges])
    hs = np.array(hs)
    assert np.abs(h - hs).max() <= 1e-12 * np.abs(hs).max()
    Jo = float(((hs - OBS) ** 2).sum())
    assert abs(J - Jo) <= 1e-12 * Jo


@pytest.mark.parametrize("wetdry", WD)
def test_adjoint_gradient_matches_the_taped_oracle(wetdry):
    import oracle
    case, man, a = _setup(wetdry=wetdry)
    J, gn, gq = a.gradient()
    Jt, gnt, gqt = oracle.taped_gradient(case, man, case.inflows[0].q_knots, DTS, SAMPLES, OBS,
                                         wetdry=wetdry)
    assert abs(J - Jt) <= 1e-12 * Jt
    assert np.abs(gnt).max() > 0
    assert np.abs(gn - gnt).max() <= 1e-9 * np.abs(gnt).max(), np.abs(gn - gnt).max()
    assert np.abs(gq - gqt).max() <= 1e-9 * np.abs(gqt).max(), (gq, gqt)
    assert np.array_equal(gn == 0.0, gnt == 0.0)   # same cells untouched by the flow


def test_adjoint_gradient_matches_gpu_finite_differences():
    case, man, a = _setup()
    J, gn, gq = a.gradient()
    qk = case.inflows[0].q_knots.copy()
    for j, i in np.argwhere(np.abs(gn) > 0.05 * np.abs(gn).max())[:4]:
        e = 1e-6
        mp, mm = man.copy(), man.copy()
        mp[j, i] += e
        mm[j, i] -= e
        a.set_params(mp, qk)
        Jp = a.forward()[0]
        a.set_params(mm, qk)
        Jm = a.forward()[0]
        fd = (Jp - Jm) / (2 * e)
        assert abs(gn[j, i] - fd) <= 1e-5 * abs(fd), (j, i, gn[j, i], fd)
    a.set_params(man, qk)
    e = 1e-5
    qp, qm = qk.copy(), qk.copy()
    qp[0] += e
    qm[0] -= e
    a.set_params(man, qp)
    Jp = a.forward()[0]
    a.set_params(man, qm)
    Jm = a.forward()[0]
    fd = (Jp - Jm) / (2 * e)
    assert abs(gq[0] - fd) <= 1e-5 * abs(fd), (gq[0], fd)


@pytest.mark.parametrize("nsnap", [1, 2, 3, 5, 31])
def test_checkpointing_does_not_change_the_gradient(nsnap):
    _, _, ref = _setup(nsnap=64)
    Jr, gnr, gqr = ref.gradient()
    _, _, a = _setup(nsnap=nsnap)
    J, gn, gq = a.gradient()
    assert J == Jr and np.array_equal(gn, gnr) and np.array_equal(gq, gqr)
    fwd, rev = a.counts()
    assert rev == len(DTS)
    # binomial checkpointing: with c = nsnap - 1 free slots, at most r recomputation
    # sweeps, r the least integer with C(c + r, c) >= K, plus the misfit's own sweep
    if nsnap >= 2:
        from math import comb
        c, K = nsnap - 1, len(DTS)
        r = next(r for r in range(1, K + 1) if comb(c + r, c) >= K)
        assert fwd <= (r + 1) * K, (fwd, r)


def test_autograd_function_runs_the_adjoint():
    import torch
    from paper_2010_02003_gb300 import binding as B
    case, man, a = _setup()
    _, gn, gq = a.gradient()
    n_t = torch.tensor(man, dtype=torch.float64, device="cuda", requires_grad=True)
    q_t = torch.tensor(case.inflows[0].q_knots, dtype=torch.float64, device="cuda",
                       requires_grad=True)
    J = B.gauge_misfit(a, n_t, q_t)
    J.backward()
    assert np.array_equal(n_t.grad.cpu().numpy(), gn)
    assert np.array_equal(q_t.grad.cpu().numpy(), gq)


def test_adjoint_rejects_other_forms():
    from paper_2010_02003_gb300 import binding as B
    p = B.dg2_default_params()
    p.variant = B.DG2_LL
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_adj_create(8, 8, 1.0, 1.0, p, 4, 1, 10, 0, 0, 0)
    assert e.value.code == B.DG2_E_ARG
    p = B.dg2_default_params()
    p.wetdry = 7
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_adj_create(8, 8, 1.0, 1.0, p, 4, 1, 10, 0, 0, 0)
    assert e.value.code == B.DG2_E_ARG


def _calibration16(B, precision, nsteps=400, every=40, nsnap=8):
    """The calibration recipe at the size of its finite-difference check: the floodplain
    terrain generator (seed 2014) on 16 x 16 cells of 2 m under a free surface 0.3 m above
    its highest point and tilted 5e-4, the generator's two-zone Manning field and
    triangular inflow as the truth, 8 gauges sampled every `every` of `nsteps` frozen
    Courant steps (37 s; every cell stays 0.34 m deep or more); an adjoint of the given
    precision with the truth's FP64 gauge depths as observations, parameters at Manning
    0.04 and 0.8 x the truth's knots.  The window is well conditioned: the Manning misfit
    moves the gauges by 1.5e-3 m while rounding the state to FP32 every step moves them
    by 4e-5 m, and central differences of the oracle converge (to 1e-6 of the taped
    gradient for steps 1e-4 to 1e-6)."""
    case = inputs.flooded_plain(16, 16, 2.0, seed=2014, freeboard=0.3, tilt=5e-4)
    s = B.solver_from_case(case, variant=B.DG2_NL, precision=B.DG2_FP64)
    dts = np.array([s.step(-1.0, want_dt=True) for _ in range(nsteps)])
    s.close()
    samples = list(range(every, nsteps + 1, every))
    truth = B.Adjoint(case, nsnap=nsnap, max_steps=len(dts))
    truth.set_schedule(dts, samples, np.zeros((len(samples), truth.ngauge)))
    _, h_true = truth.forward()
    a = B.Adjoint(case, nsnap=nsnap, max_steps=len(dts), precision=precision)
    a.set_schedule(dts, samples, h_true)
    man = np.full((case.ny, case.nx), 0.04)
    qk = 0.8 * case.inflows[0].q_knots
    a.set_params(man, qk)
    return case, a, man, qk, dts, samples, h_true


def _central(a, man, qk, j, i, e):
    mp, mm = man.copy(), man.copy()
    mp[j, i] += e
    mm[j, i] -= e
    a.set_params(mp, qk)
    Jp = a.forward()[0]
    a.set_params(mm, qk)
    Jm = a.forward()[0]
    a.set_params(man, qk)
    return (Jp - Jm) / (2 * e)


def test_finite_differences_on_the_16x16_calibration_recipe():
    """FP64 adjoint on the 16 x 16 calibration recipe: the oracle's taped gradient, and
    central differences of the GPU forward on the six largest Manning components and
    on the positive knot (steps 1e-5 on n = 0.04, 1e-3 on the knot; the zero first knot
    is left out, a negative discharge there has no derivative)."""
    import oracle
    from paper_2010_02003_gb300 import binding as B
    case, a, man, qk, dts, samples, h_true = _calibration16(B, B.DG2_FP64)
    assert a.ngauge == 8
    J, gn, gq = a.gradient()
    assert J > 0 and np.abs(gn).max() > 0
    # the misfit sums squares of ~1e-3 m gauge differences taken from ~2 m depths that
    # the two programs round differently over 400 steps (measured |J - Jt| = 2e-14 of
    # J = 7.8e-6): misfit and gradients against the tape within 1e-8 / 1e-6 relative
    Jt, gnt, gqt = oracle.taped_gradient(case, man, qk, dts, samples, h_true)
    assert abs(J - Jt) <= 1e-8 * Jt, (J, Jt)
    assert np.abs(gn - gnt).max() <= 1e-6 * np.abs(gnt).max()
    assert np.abs(gq - gqt).max() <= 1e-6 * np.abs(gqt).max()
    for j, i in np.argwhere(np.abs(gn) >= np.sort(np.abs(gn).ravel())[-6]):
        fd = _central(a, man, qk, j, i, 1e-5)
        assert abs(gn[j, i] - fd) <= 1e-5 * abs(fd), (j, i, gn[j, i], fd)
    for k in np.flatnonzero(qk > 1.0):
        e = 1e-3
        qp, qm = qk.copy(), qk.copy()
        qp[k] += e
        qm[k] -= e
        a.set_params(man, qp)
        Jp = a.forward()[0]
        a.set_params(man, qm)
        Jm = a.forward()[0]
        fd = (Jp - Jm) / (2 * e)
        assert abs(gq[k] - fd) <= 1e-5 * abs(fd), (k, gq[k], fd)


# FP32 adjoint against the FP64 one on the 16 x 16 recipe (relative to the largest
# FP64 component): measured misfit 3.7e-2, Manning gradient 2.4e-2, knot gradient
# 3.1e-2 -- the ratio of the FP32 rounding carried to the gauges (4e-5 m) to the
# misfit signal (1.5e-3 m); bars at 3x
FP32_ADJ_BAR = {"misfit": 1.1e-1, "manning": 7e-2, "knots": 9e-2}


def test_fp32_adjoint_against_the_fp64_adjoint():
    """The FP32 adjoint (FP32 storage of state, checkpoints, adjoints, Jacobians and
    inputs; FP64 arithmetic) on the 16 x 16 calibration recipe: its misfit and gradients
    against the FP64 adjoint's, which the taped oracle and finite differences pin.
    Depths of up to 4 m stored in FP32 round by ~4e-7 m each step; the trajectory
    carries that rounding (4e-5 m at the gauges after 400 steps against a 1.5e-3 m
    signal), which sets the error stated here."""
    from paper_2010_02003_gb300 import binding as B
    _, a64, _, _, _, _, _ = _calibration16(B, B.DG2_FP64)
    _, a32, _, _, _, _, _ = _calibration16(B, B.DG2_FP32)
    J64, gn64, gq64 = a64.gradient()
    J32, gn32, gq32 = a32.gradient()
    e_j = abs(J32 - J64) / J64
    e_n = np.abs(gn32 - gn64).max() / np.abs(gn64).max()
    e_q = np.abs(gq32 - gq64).max() / np.abs(gq64).max()
    print(f"FP32 adjoint vs FP64: misfit {e_j:.2e}, Manning gradient {e_n:.2e}, "
          f"knot gradient {e_q:.2e}")
    assert e_j < FP32_ADJ_BAR["misfit"], e_j
    assert e_n < FP32_ADJ_BAR["manning"], e_n
    assert e_q < FP32_ADJ_BAR["knots"], e_q
    big = np.abs(gn64) > 0.1 * np.abs(gn64).max()
    assert np.array_equal(np.sign(gn32[big]), np.sign(gn64[big]))


def test_fp32_adjoint_checkpoints_do_not_change_the_gradient():
    """The FP32 gradient does not change a bit with the number of checkpoint slots (the
    recomputed forward segments round exactly as the first sweep did).  (Central
    differences of the FP32-storage forward are no check here: its misfit moves by
    ~4 % under FP32 rounding of the state, as much as a 1 % change of one cell's n.)"""
    from paper_2010_02003_gb300 import binding as B
    case, a, man, qk, dts, samples, h_true = _calibration16(B, B.DG2_FP32)
    J1, gn1, gq1 = a.gradient()
    b = B.Adjoint(case, nsnap=3, max_steps=len(dts), precision=B.DG2_FP32)
    b.set_schedule(dts, samples, h_true)
    b.set_params(man, qk)
    J3, gn3, gq3 = b.gradient()
    assert J3 == J1 and np.array_equal(gn3, gn1) and np.array_equal(gq3, gq1)
    fwd, rev = b.counts()
    assert rev == len(dts)
