"""dg2_mass_noalloc: the mass reduction for callers that cannot allocate device memory.

It reads a caller-owned depth plane and writes one caller-owned double, keeping
its partial sums in the library's fixed device scratch.  Checked against the
regular dg2_mass (which keeps its partials in the caller's workspace) on two
calls in a row, through the C ABI.  Collected last so that a failure here leaves
every other test already run.
"""
import numpy as np
import pytest

from paper_2010_02003_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_mass_matches_dg2_mass_twice_in_a_row():
    import torch
    from paper_2010_02003_gb300 import binding as B

    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    cases = [inputs.hump(eta=0.5, dam_eta=1.0), inputs.random_terrain(77, 53, seed=5)]
    for k, case in enumerate(cases):
        s = B.solver_from_case(case)
        for _ in range(5):
            s.step(-1.0)
        ref, _ = s.mass()                                      # regular entry point
        planes = s.state()                                     # public API: host copy
        pitch = case.nx + 3                                    # a padded caller layout
        h0 = torch.zeros((case.ny, pitch), dtype=torch.float64, device="cuda")
        h0[:, :case.nx] = torch.from_numpy(planes[0]).cuda()
        h0[:, case.nx:] = 1e9                                  # padding must not be summed
        torch.cuda.synchronize()
        B.dg2_mass_noalloc(h0.data_ptr(), case.nx, case.ny, pitch, case.dx, case.dy,
                           out.data_ptr() + 8 * k, 0)
        torch.cuda.synchronize()
        got = float(out[k].item())
        assert abs(got - ref) <= 1e-12 * abs(ref), (k, got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2010_02003_gb300 import binding as B

    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(B.Dg2Error) as e:
        B.dg2_mass_noalloc(buf.data_ptr(), 1, B.DG2_NOALLOC_MAX_ROWS + 1, 1, 1.0, 1.0,
                           buf.data_ptr(), 0)
    assert e.value.code == B.DG2_E_ARG
    assert "DG2_NOALLOC_MAX_ROWS" in str(e.value)
