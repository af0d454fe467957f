"""Conditioning of the oracle's own trajectories (no GPU).

The FP64 parity bar is a statement about rounding order: an implementation that
rounds differently starts ~1e-16 away and stays within 1e-12 only while the
discrete dynamics do not amplify round-off by more than ~1e4.  These tests measure
it on the oracle alone by running it twice, the second time from a state
perturbed by a few units in the last place.

On the floodplain's dry start, the thin front of water entering the channel
amplifies a 2e-16 perturbation within steps 88-100: measured 1.4e-10 (DG2-LL) and
1.8e-11 (DG2-NL) under the default face revision, 8.6e-13 (DG2-LL) under the
printed one.  Every earlier ten-step window stays below the 1e-12 bar (at most
1.8e-13).  The
perturbation is applied to the nonzero coefficients of a state that already
holds water (step 10 onwards; the dry initial state has nothing to perturb).
"""
import numpy as np
import pytest

from conftest import make_oracle
from paper_2010_02003_gb300 import inputs


def _scaled_err(a, b, g=9.80665):
    a = a.reshape(9, -1)
    b = b.reshape(9, -1)
    hs = max(np.abs(b[0]).max(), 1e-30)
    qs = max(np.abs(b[3]).max(), np.abs(b[6]).max(), hs * np.sqrt(g * hs))
    scale = np.array([hs] * 3 + [qs] * 6)
    return (np.abs(a - b).max(axis=1) / scale).max()


def _twin_growth(start, steps, seeds, wetdry, limiter=True, initial="dry"):
    if initial == "dry":
        case = inputs.floodplain(nx=96, ny=64, dx=2.0, q_peak=15.0, t_peak=20.0,
                                 channel_width=12.0)
    else:
        case = inputs.floodplain(nx=96, ny=64, dx=2.0, q_peak=15.0, t_peak=60.0,
                                 initial="channel", channel_width=12.0)
    o = make_oracle(case, limiter=limiter, wetdry=wetdry)
    for _ in range(start):
        o.step()
    s0, t0 = o.state(), o.t
    dts = [o.step() for _ in range(steps)]
    ref = o.state()
    hs = np.abs(s0[0]).max()
    qs = max(np.abs(s0[3]).max(), np.abs(s0[6]).max())
    scale = np.array([hs] * 3 + [qs] * 6)[:, None, None]
    out = []
    for seed in seeds:
        rng = np.random.default_rng(seed)
        p = s0 + rng.standard_normal(s0.shape) * 2e-16 * scale * (s0 != 0)
        tw = make_oracle(case, limiter=limiter, wetdry=wetdry)
        tw.set_state(p, t0)
        for dt in dts:
            tw.step(dt)
        out.append(_scaled_err(tw.state(), ref))
    return np.array(out)


@pytest.mark.parametrize("wetdry", ["positive", "paper"])
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_floodplain_windows_before_the_front_are_well_conditioned(limiter, wetdry):
    for start in (10, 40, 70):
        assert _twin_growth(start, 10, range(3), wetdry, limiter).max() < 1e-12, start


@pytest.mark.parametrize("wetdry", ["positive", "paper"])
def test_floodplain_ll_front_amplifies_roundoff(wetdry):
    assert _twin_growth(88, 12, range(6), wetdry, True).max() > 5e-13


# The free-running parity horizons of the GPU tests: from the first wet state, the
# twin runs stay well below the 1e-12 bar over the steps each case is held.
HELD = {("positive", False): 84, ("positive", True): 84, ("paper", False): 99,
        ("paper", True): 89}


@pytest.mark.parametrize("wetdry", ["positive", "paper"])
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_floodplain_start_is_well_conditioned_over_the_held_horizon(limiter, wetdry):
    assert _twin_growth(1, HELD[(wetdry, limiter)], range(2), wetdry, limiter).max() < 1e-13


@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_channel_start_under_the_default_revision_is_well_conditioned(limiter):
    assert _twin_growth(0, 100, range(2), "positive", limiter, "channel").max() < 1e-13


def test_channel_start_under_the_printed_revision_amplifies_roundoff():
    # partially wet bank cells offer their full planar face depth: held 50 steps on the GPU
    assert _twin_growth(0, 50, range(2), "paper", False, "channel").max() < 1e-12
    assert _twin_growth(0, 80, range(2), "paper", False, "channel").max() > 1e-13


def _member_twin(t_end, t_pert, limiter):
    """Largest FP32-size (1e-7 relative) twin difference over the six members of the
    GPU ensemble-against-oracle test, from t_pert to t_end on the same steps."""
    cases = inputs.ensemble(n=6, seed=4242, nx_range=(33, 96), ny_range=(17, 64), t_peak=3.0,
                            t_end=t_end, ngauge=2, sample_every=0.0)
    worst = 0.0
    for c in cases:
        o = make_oracle(c, limiter=limiter)
        while o.t < t_pert:
            o.step()
        s0, t0 = o.state(), o.t
        dts = []
        while o.t + o.cfl_dt() < t_end:
            dts.append(o.step())
        dts.append(t_end - o.t)
        o.step(dts[-1])
        tw = make_oracle(c, limiter=limiter)
        tw.set_state(s0 * (1 + 1e-7 * np.random.default_rng(1).standard_normal(s0.shape)), t0)
        for dt in dts:
            tw.step(dt)
        worst = max(worst, _scaled_err(tw.state(), o.state()))
    return worst


@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_ensemble_members_are_well_conditioned_to_8_s(limiter):
    assert _member_twin(8.0, 1.5, limiter) < 1e-6
