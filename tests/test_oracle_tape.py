"""The oracle's taped derivatives (oracle/tape.cpp) against central finite
differences of the oracle itself (no GPU): the tape is the independent reference
the GPU adjoint is checked against, so it is pinned first."""
import numpy as np

from conftest import make_oracle
from paper_2010_02003_gb300 import inputs


def _case(**kw):
    return inputs.floodplain(nx=14, ny=10, dx=2.0, q_peak=5.0, t_peak=20.0, t_end=60.0,
                             channel_width=8.0, inflow_len=8.0, ngauge=3, sample_every=5.0,
                             initial="channel", **kw)


DTS = np.full(30, 0.05)
SAMPLES = [10, 20, 30]


def _misfit(man, qk, obs):
    c = _case()
    c.manning = man
    c.inflows[0].q_knots = qk
    o = make_oracle(c)
    hs = []
    for k in range(1, len(DTS) + 1):
        o.step(DTS[k - 1])
        if k in SAMPLES:
            hs.append([o.gauge_h(x, y) for x, y in c.gauges])
    return float(((np.array(hs) - obs) ** 2).sum())


def test_taped_gradient_matches_oracle_finite_differences():
    import oracle
    case = _case()
    rng = np.random.default_rng(1)
    man = 0.03 + 0.02 * rng.random((case.ny, case.nx))
    qk = case.inflows[0].q_knots.copy()
    obs = np.full((3, 3), 0.3)
    J, gn, gq = oracle.taped_gradient(case, man, qk, DTS, SAMPLES, obs)
    # the taped run is the oracle run (the C++ scalar type reproduces the misfit to the
    # last unit or so; its derivatives are the subject of the checks below)
    assert abs(J - _misfit(man, qk, obs)) <= 1e-15 * abs(J)
    checked = 0
    for j, i in [(5, 3), (4, 7), (6, 1), (3, 5)]:
        e = 1e-6
        mp, mm = man.copy(), man.copy()
        mp[j, i] += e
        mm[j, i] -= e
        fd = (_misfit(mp, qk, obs) - _misfit(mm, qk, obs)) / (2 * e)
        assert abs(gn[j, i] - fd) <= 1e-6 * max(abs(fd), 1e-3), (j, i, gn[j, i], fd)
        checked += abs(fd) > 1e-4
    assert checked >= 2
    for k in range(2):
        e = 1e-5
        qp, qm = qk.copy(), qk.copy()
        qp[k] += e
        qm[k] -= e
        fd = (_misfit(man, qp, obs) - _misfit(man, qm, obs)) / (2 * e)
        assert abs(gq[k] - fd) <= 1e-5 * max(abs(fd), 1e-4), (k, gq[k], fd)
    # cells the water never reaches carry no gradient
    assert gn[0, -1] == 0.0
