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


@pytest.mark.parametrize("precision", [0, 1], ids=["FP64", "FP32"])
@pytest.mark.parametrize("variant", [0, 1], ids=["NL", "LL"])
def test_skip_on_ragged_grid_with_point_source(variant, precision):
    """A ragged grid (neither side a multiple of the tile or of the 8 x 4 warp
    block), a dam breaking into a dry basin from off-centre and a point source
    without rain: fronts cross tile and warp-block edges in every direction, and
    the source's tile is forced while its neighbours are not."""
    case = inputs.hump(nx=203, ny=117, eta=-1.0, dam_eta=1.0, dam_radius=14.0)
    case.eta_corner = np.roll(case.eta_corner, (9, -23), axis=(0, 1))
    case.point = (40.5, 90.5, 0.5)
    a = _run(case, variant, precision, True, 160, dt_max=0.05)
    b = _run(case, variant, precision, False, 160, dt_max=0.05)
    assert np.array_equal(a[0], b[0])
    assert a[1] == b[1] and a[2] == b[2] and a[3] == b[3]
    assert (a[0][0] > 1e-5).sum() > 500        # the flow has spread


def _expected_active(state, tol=1e-5, tx=32, ty=8):
    """Tiles within one tile (3 x 3 neighbourhood) of a tile holding a non-quiescent
    cell (h0 > tol or any other mode non-zero), from the FP64 state."""
    busy = (state[0] > tol) | (np.abs(state[1:]).max(axis=0) != 0)
    ny, nx = busy.shape
    nty, ntx = -(-ny // ty), -(-nx // tx)
    pad = np.zeros((nty * ty, ntx * tx), dtype=bool)
    pad[:ny, :nx] = busy
    t = pad.reshape(nty, ty, ntx, tx).any(axis=(1, 3))
    d = t.copy()
    d[1:] |= t[:-1]
    d[:-1] |= t[1:]
    d2 = d.copy()
    d2[:, 1:] |= d[:, :-1]
    d2[:, :-1] |= d[:, 1:]
    return int(d2.sum()), ntx * nty


def test_tile_lists_match_host_classification():
    """The device tile lists hold exactly the tiles of the 3 x 3 rule (dam in a dry basin,
    no forced tiles), and the running total counts every computed tile."""
    from paper_2010_02003_gb300 import binding as B
    case = inputs.hump(nx=200, ny=120, eta=-1.0 + 0.0, dam_eta=1.0, dam_radius=12.0)
    s = B.solver_from_case(case, variant=B.DG2_LL)
    nt, na, nf, done = s.tile_stats()
    assert na == nt and done == 0              # a new state computes every tile once
    total = 0
    for k in range(30):
        _, na, nf, done0 = s.tile_stats()
        s.step(-1.0)
        _, na1, nf1, done1 = s.tile_stats()
        assert done1 - done0 == na                # the step computed the listed tiles
        exp, ntiles = _expected_active(s.state(), tx=s.tile_shape()[0], ty=s.tile_shape()[1])
        assert ntiles == nt and na1 == exp, (k, na1, exp)
        assert 0 < na1 < nt and na1 + nf1 <= nt
        total += na
    assert done1 == total


def test_tile_stats_without_skipping_and_all_dry():
    from paper_2010_02003_gb300 import binding as B
    case = inputs.hump(nx=100, ny=50, eta=0.5)
    s = B.solver_from_case(case, skip_dry_tiles=False)
    for _ in range(3):
        s.step(-1.0)
    nt, na, nf, done = s.tile_stats()
    tw, th = s.tile_shape()
    assert nt == -(-100 // tw) * -(-50 // th) and na == nt and nf == 0 and done == 3 * nt
    dry = inputs.hump(nx=100, ny=50, eta=-1.0)
    s2 = B.solver_from_case(dry)
    for _ in range(3):
        s2.step(-1.0)
    nt, na, nf, done = s2.tile_stats()
    assert na == 0 and nf == 0 and done == nt   # only the first step after set-up computes
