"""Long runs on the floodplain recipe's steep channel banks (GPU, default face
revision): the failure class that R25-R26 address.  Under the printed revision of
Sec. 2.1.2 partially wet bank cells drove averages to -0.45 m, cell speeds q0/h0
past 1000 m/s, Courant steps to 1e-4 s, and DG2-LL to a non-finite state at t = 1314 s
on the 2000x1000 grid.  Here a 400x200 grid of the same recipe (2 m cells, incised
channel, 1 m of water in it, inflow hydrograph) runs 15 minutes of simulated time in
FP64 (DG2-NL and DG2-LL) and FP32 (DG2-NL) through dg2_run_to."""
import numpy as np
import pytest

from paper_2010_02003_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _speeds(st):
    h0 = st[0]
    w = h0 > TOL
    hs = np.where(w, h0, 1.0)
    return np.where(w, np.maximum(np.abs(st[3] / hs), np.abs(st[6] / hs)), 0.0)


@pytest.mark.parametrize("variant,precision", [(0, 0), (1, 0), (0, 1)],
                         ids=["fp64-NL", "fp64-LL", "fp32-NL"])
def test_channel_start_runs_clean(variant, precision):
    from paper_2010_02003_gb300 import binding as B
    case = inputs.floodplain(nx=400, ny=200, dx=2.0, q_peak=20.0, t_peak=600.0,
                             initial="channel")
    s = B.solver_from_case(case, variant=variant, precision=precision)
    worst_h, worst_u, steps = 0.0, 0.0, 0
    for t_end in (300.0, 600.0, 900.0):
        steps += s.run_to(t_end)                 # raises on a non-finite state
        st = s.state()
        assert np.isfinite(st).all()
        worst_h = min(worst_h, float(st[0].min()))
        worst_u = max(worst_u, float(_speeds(st).max()))
    m, led = s.mass()
    assert abs(m - led) <= (1e-12 if precision == 0 else 1e-6) * m
    assert worst_h > -1e-3, worst_h              # averages stay (near) non-negative
    assert worst_u < 30.0, worst_u               # no artificial velocities
    # Courant steps set by the flow, not by films: well under one step per 0.02 s
    assert steps < 900.0 / 0.02, steps
    print(f"{'fp32' if precision else 'fp64'} {'LL' if variant else 'NL'}: {steps} steps to "
          f"900 s, min h0 {worst_h:.2e}, max |q0/h0| {worst_u:.2f}")
