"""Failure detection through the C ABI, with the failure made on the host.

A step far beyond the Courant limit (a forced dt of 50 s where the limit is
about 0.1 s, or a Courant number of 40 in an ensemble member's parameters)
drives the state to values that overflow or turn negative past -1 m.  The
device guards of the stage kernels (a block-wide OR of the per-cell checks) and
of the end of step (a step that is not positive and finite) raise the context's
non-finite flag, which the host reads as DG2_E_NONFINITE.  Further steps are
then refused without launching, until dg2_set_state restores a valid state.
Only floating-point arithmetic on finite inputs happens on the GPU: nothing here
can fault or hang it.
"""
import numpy as np
import pytest

from paper_2010_02003_gb300 import inputs

pytestmark = pytest.mark.gpu


def _B():
    from paper_2010_02003_gb300 import binding
    return binding


def _step_until_nonfinite(B, s, dt, max_steps):
    """Forces steps of size dt and returns the step count at which the guard fired."""
    for k in range(1, max_steps + 1):
        try:
            s.step(dt, want_dt=True)
        except B.Dg2Error as e:
            assert e.code == B.DG2_E_NONFINITE, (e.code, str(e))
            return k
    return None


@pytest.mark.parametrize("precision", [0, 1], ids=["FP64", "FP32"])
@pytest.mark.parametrize("variant", [0, 1], ids=["NL", "LL"])
def test_courant_violating_step_trips_the_guard_and_later_steps_are_refused(variant, precision):
    B = _B()
    case = inputs.hump(eta=0.5, dam_eta=1.0)           # wet dam break, dx = 1 m
    s = B.solver_from_case(case, variant=variant, precision=precision)
    good, t_good = s.state(), s.time()[0]
    fired = _step_until_nonfinite(B, s, 50.0, 60)
    assert fired is not None, "a 50 s step on a 1 m grid never raised DG2_E_NONFINITE"
    launches = s.launches()
    # refused without a launch, with or without a read of the step size
    for want in (False, True):
        with pytest.raises(B.Dg2Error) as e:
            s.step(-1.0, want_dt=want)
        assert e.value.code == B.DG2_E_NONFINITE
    with pytest.raises(B.Dg2Error) as e:
        s.run_to(100.0)
    assert e.value.code == B.DG2_E_NONFINITE
    assert s.launches() == launches
    # a valid state clears the flag and the context steps again
    s.set_state(good, t_good)
    dt = s.step(-1.0, want_dt=True)
    assert 0.0 < dt < 1.0
    assert np.isfinite(s.state()).all()


def test_ensemble_member_with_a_courant_number_of_40_is_reported_and_refused():
    B = _B()
    cases = inputs.ensemble(n=3, seed=5, nx_range=(40, 80), ny_range=(24, 48), t_peak=30.0,
                            t_end=60.0, sample_every=0.0)
    mem = [B.solver_from_case(c, variant=B.DG2_NL, precision=B.DG2_FP32,
                              cfl=40.0 if k == 1 else c.cfl)
           for k, c in enumerate(cases)]
    # water everywhere in the unstable member, so its first steps are violent
    flooded = inputs.flooded_plain(cases[1].nx, cases[1].ny, cases[1].dx, seed=9)
    mem[1].set_dem(flooded.z_corner, None, 0.03, flooded.eta_corner)
    ens = B.Ensemble(mem)
    with pytest.raises(B.Dg2Error) as e:
        ens.run_to(60.0)
    assert e.value.code == B.DG2_E_NONFINITE
    # the next run is refused at its start: no chunk is replayed
    l0 = ens.launches()
    with pytest.raises(B.Dg2Error) as e:
        ens.run_to(60.0)
    assert e.value.code == B.DG2_E_NONFINITE
    assert ens.launches() - l0 <= 3                  # the start-of-run kernels only
    # the other members' states stayed finite throughout
    for k in (0, 2):
        assert np.isfinite(mem[k].state()).all()
