"""Skipping quiescent dry tiles is exact: a run with skipping equals, bit for bit,
the same run computing every tile (both precisions, both variants, with inflow,
rain and point-source tiles that must stay active)."""
import numpy as np
import pytest

from paper_2010_02003_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(case, variant, precision, skip, nsteps, **kw):
    from paper_2010_02003_gb300 import binding as B
    s = B.solver_from_case(case, variant=variant, precision=precision, skip_dry_tiles=skip, **kw)
    dts = [s.step(-1.0, want_dt=True) for _ in range(nsteps)]
    return s.state(), s.time(), s.mass(), dts


CASES = {
    "floodplain_dry_160x96": lambda: inputs.floodplain(nx=160, ny=96, dx=2.0, q_peak=15.0,
                                                       t_peak=20.0, channel_width=12.0),
    "floodplain_channel_200x120": lambda: inputs.floodplain(nx=200, ny=120, dx=2.0,
                                                            initial="channel", channel_width=12.0),
    "dam_128": lambda: inputs.hump(eta=-1.0 + 0.0, dam_eta=1.0, dam_radius=12.0),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["FP64", "FP32"])
@pytest.mark.parametrize("variant", [0, 1], ids=["NL", "LL"])
@pytest.mark.parametrize("name", list(CASES))
def test_skip_is_bit_identical(name, variant, precision):
    case = CASES[name]()
    a = _run(case, variant, precision, True, 150)
    b = _run(case, variant, precision, False, 150)
    assert np.array_equal(a[0], b[0])
    assert a[1] == b[1] and a[2] == b[2] and a[3] == b[3]


@pytest.mark.parametrize("precision", [0, 1], ids=["FP64", "FP32"])
def test_skip_with_point_source_and_rain(precision):
    case = inputs.hump(nx=150, ny=90, eta=-1.0)        # dry basin
    case.point = (100.5, 60.5, 2.0)
    case.rain = (1e-4, 5.0, 12.0)                       # rain starts later: all tiles then
    # the dry-domain step dt_max must respect the source's filling rate (2 m^3/s into 1 m^2)
    a = _run(case, 0, precision, True, 120, dt_max=0.02)
    b = _run(case, 0, precision, False, 120, dt_max=0.02)
    assert np.array_equal(a[0], b[0]) and a[2] == b[2]
    assert a[0][0].max() > 0.0
