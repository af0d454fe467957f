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


def test_finite_differences_on_the_16x16_calibration_recipe():
    """The calibration recipe at the size of its finite-difference check: the floodplain
    terrain generator (seed 2014) on 16 x 16 cells of 2 m under a gently tilted free
    surface, the generator's two-zone Manning field and triangular inflow as the truth,
    8 gauges sampled every 10 steps over 120 frozen Courant steps; the misfit is taken
    at Manning 0.04 everywhere and the knots at 0.8 x truth.  The adjoint gradient must
    match central differences of the GPU forward on the largest Manning components
    and on two knots, and the oracle's taped gradient."""
    import oracle
    from paper_2010_02003_gb300 import binding as B
    case = inputs.flooded_plain(16, 16, 2.0, seed=2014)
    s = B.solver_from_case(case, variant=B.DG2_NL, precision=B.DG2_FP64)
    dts = np.array([s.step(-1.0, want_dt=True) for _ in range(120)])
    s.close()
    samples = list(range(10, 121, 10))
    a = B.Adjoint(case, nsnap=8, max_steps=len(dts))
    assert a.ngauge == 8
    a.set_schedule(dts, samples, np.zeros((len(samples), a.ngauge)))
    _, h_true = a.forward()
    a.set_schedule(dts, samples, h_true)
    man = np.full((case.ny, case.nx), 0.04)
    qk = 0.8 * case.inflows[0].q_knots
    a.set_params(man, qk)
    J, gn, gq = a.gradient()
    assert J > 0 and np.abs(gn).max() > 0
    # the misfit moves by ~1e-15 for a 1e-6 change of one cell's n while the depths are
    # ~2 m (round-off 4e-16), so the differences use steps whose truncation error
    # (relative ~e^2) stays far below the tolerance: 1e-4 on n = 0.04, 1e-3 on the knots
    for j, i in np.argwhere(np.abs(gn) >= np.sort(np.abs(gn).ravel())[-6]):
        e = 1e-4
        mp, mm = man.copy(), man.copy()
        mp[j, i] += e
        mm[j, i] -= e
        a.set_params(mp, qk)
        Jp = a.forward()[0]
        a.set_params(mm, qk)
        Jm = a.forward()[0]
        fd = (Jp - Jm) / (2 * e)
        assert abs(gn[j, i] - fd) <= 1e-4 * abs(fd), (j, i, gn[j, i], fd)
    for k in np.argsort(-np.abs(gq))[:2]:
        e = 1e-3
        qp, qm = qk.copy(), qk.copy()
        qp[k] += e
        qm[k] -= e
        a.set_params(man, qp)
        Jp = a.forward()[0]
        a.set_params(man, qm)
        Jm = a.forward()[0]
        fd = (Jp - Jm) / (2 * e)
        assert abs(gq[k] - fd) <= 1e-4 * abs(fd), (k, gq[k], fd)
    Jt, gnt, gqt = oracle.taped_gradient(case, man, qk, dts, samples, h_true)
    assert abs(J - Jt) <= 1e-12 * Jt
    assert np.abs(gn - gnt).max() <= 1e-9 * np.abs(gnt).max()
    assert np.abs(gq - gqt).max() <= 1e-9 * np.abs(gqt).max()
