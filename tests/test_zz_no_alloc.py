"""lbm_residual_noalloc, the convergence monitor for callers that cannot
allocate device memory, against lbm_residual.

Some callers hand all device memory to another framework's pool, or monitor
convergence at a point where an allocation would synchronise the device or
fail; they cannot let the library allocate scratch.  lbm_residual_noalloc
takes the two states and the solid mask as device arrays the caller already
holds and keeps its partial sums in a fixed array inside the library.  This
test checks it through the C ABI against lbm_residual on the same states,
twice in a row per case (the second call reuses the scratch the first one
left behind), within the parity tolerances of the other GPU tests.
"""
import math

import numpy as np
import pytest

from paper_2012_14707_gb300 import build as lbm_build
from paper_2012_14707_gb300 import cases, lbm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,precision,res_rtol", [
    ("cylinders", "fp32", 1e-5),
    ("couette", "fp64", 1e-10),
])
def test_noalloc_residual_matches_lbm_residual(name, precision, res_rtol):
    import torch

    lbm_build.build()
    lbm.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    if name == "cylinders":
        case = cases.cylinder_array(300, 150, 5, Kn=0.02, ax=1e-5)
    else:
        case = cases.annulus(64, 12.0, 28.0, 0.05, 0.05 * math.sqrt(1 / 3) / 12)
    g = lbm.Solver(case, precision=precision, stream=stream)
    solid = torch.from_numpy(np.ascontiguousarray(case.solid, np.uint8)).cuda()
    g.step(40)
    for call in range(2):
        f_prev = torch.from_numpy(g.get_f()).cuda()
        g.step(1)
        f_cur = torch.from_numpy(g.get_f()).cuda()
        want_res, want_mass = g.residual()
        torch.cuda.synchronize()
        res, mass = lbm.lbm_residual_noalloc(f_cur.data_ptr(), f_prev.data_ptr(), solid.data_ptr(),
                                             case.nx, case.ny, case.ax, case.ay, stream)
        assert want_res > 0.0
        assert res == pytest.approx(want_res, rel=res_rtol), call
        assert mass == pytest.approx(want_mass, rel=1e-13), call
        g.step(25)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    lbm.load()
    torch.cuda.set_device(0)
    f = torch.zeros(9, dtype=torch.float64, device="cuda")
    m = torch.zeros(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_residual_noalloc(f.data_ptr(), f.data_ptr(), m.data_ptr(), 1, 16385, 0.0, 0.0)
    assert ei.value.code == lbm.LBM_EINVAL
    assert "16384" in str(ei.value)


def test_noalloc_reports_a_nonfinite_previous_state():
    """A non-finite value in the previous state alone is reported, as
    lbm_residual reports it (both states are checked)."""
    import torch

    lbm.load()
    torch.cuda.set_device(0)
    case = cases.cylinder_array(120, 64, 3, Kn=0.02, ax=1e-5)
    f = cases.random_populations(case.nx, case.ny, 2)
    fl = np.argwhere(case.solid == 0)[17]
    f_prev = f.copy()
    f_prev[5, fl[0], fl[1]] = np.nan
    cur = torch.from_numpy(f).cuda()
    prev = torch.from_numpy(f_prev).cuda()
    solid = torch.from_numpy(np.ascontiguousarray(case.solid, np.uint8)).cuda()
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_residual_noalloc(cur.data_ptr(), prev.data_ptr(), solid.data_ptr(), case.nx,
                                 case.ny, case.ax, case.ay)
    assert ei.value.code == lbm.LBM_EUNSTABLE
    # the clean pair still reports normally afterwards
    res, mass = lbm.lbm_residual_noalloc(cur.data_ptr(), cur.data_ptr(), solid.data_ptr(), case.nx,
                                         case.ny, case.ax, case.ay)
    assert res == 0.0 and math.isfinite(mass)
