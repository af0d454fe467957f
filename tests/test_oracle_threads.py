"""The oracle's OpenMP build (rows in parallel, used only to time the oracle on every
host core) gives the serial build's results bit for bit: each cell writes only its own
outputs and the edge-flux sum of the mass ledger is taken in cell order afterwards."""
import numpy as np
import pytest

from conftest import make_oracle
from paper_2010_02003_gb300 import inputs
import oracle


@pytest.mark.parametrize("wetdry", ["positive", "paper"])
@pytest.mark.parametrize("limiter", [False, True], ids=["NL", "LL"])
def test_threaded_oracle_equals_serial_oracle(limiter, wetdry):
    case = inputs.floodplain(nx=96, ny=64, dx=2.0, q_peak=15.0, t_peak=60.0, initial="channel",
                             channel_width=12.0)
    case.rain = (1e-5, 0.0, 10.0)
    case.point = (50.5, 30.5, 0.3)
    a = make_oracle(case, limiter=limiter, wetdry=wetdry)
    b = make_oracle(case, limiter=limiter, wetdry=wetdry, threads=True)
    n = oracle.set_threads(4)
    assert n == 4
    for _ in range(30):
        dt = a.step()
        assert b.step() == dt
    assert np.array_equal(a.state(), b.state())
    assert a.ledger() == b.ledger() and a.mass() == b.mass() and a.t == b.t
