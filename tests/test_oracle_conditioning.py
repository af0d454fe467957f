"""Conditioning of the oracle's own trajectories (no GPU).

The FP64 parity bar is a statement about rounding order: an implementation that
rounds differently starts ~1e-16 away and stays within 1e-12 only while the
discrete dynamics do not amplify round-off by more than ~1e4.  These tests measure
it on the oracle alone by running it twice, the second time from a state
perturbed by a few units in the last place.

With the face revision of Sec. 2.1.2 as printed (``wetdry="paper"``), partially
wet cells on steep banks carry planar depths far above their average (a few mm
of average water, +-0.5 m at the faces), and the velocity q0/h0 of such a cell
amplifies round-off ~10^3-10^4 within a dozen steps at the channel front of the
floodplain start.  The positivity-consistent revision (the default) removes
that: the same start stays well-conditioned over all 100 steps.
"""
import numpy as np

from conftest import make_oracle
from paper_2010_02003_gb300 import inputs


def _scaled_err(a, b, g=9.80665):
    a = a.reshape(9, -1)
    b = b.reshape(9, -1)
    hs = max(np.abs(b[0]).max(), 1e-30)
    qs = max(np.abs(b[3]).max(), np.abs(b[6]).max(), hs * np.sqrt(g * hs))
    scale = np.array([hs] * 3 + [qs] * 6)
    return (np.abs(a - b).max(axis=1) / scale).max()


def _twin_growth(start, steps, seeds, wetdry):
    case = inputs.floodplain(nx=96, ny=64, dx=2.0, q_peak=15.0, t_peak=20.0, channel_width=12.0)
    o = make_oracle(case, limiter=True, wetdry=wetdry)
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
        tw = make_oracle(case, limiter=True, wetdry=wetdry)
        tw.set_state(p, t0)
        for dt in dts:
            tw.step(dt)
        out.append(_scaled_err(tw.state(), ref))
    return np.array(out)


def test_floodplain_ll_printed_revision_start_is_well_conditioned():
    # steps 0-80: a 2e-16 perturbation stays far below the 1e-12 bar
    assert _twin_growth(0, 80, range(3), "paper").max() < 1e-13


def test_floodplain_ll_printed_revision_front_amplifies_roundoff():
    # steps 88-100: the same perturbation grows by ~10^3-10^4 at the channel front
    assert _twin_growth(88, 12, range(6), "paper").max() > 1e-13


def test_floodplain_ll_positive_revision_is_well_conditioned():
    assert _twin_growth(0, 100, range(3), "positive").max() < 1e-13
    assert _twin_growth(88, 12, range(6), "positive").max() < 1e-13
