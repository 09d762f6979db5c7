"""Checkpoint and resume (lbm_save / lbm_load): a solve stopped and continued
from its file follows the uninterrupted solve bit for bit; files of another
case, precision or a damaged file are refused."""
import numpy as np
import pytest

from paper_2012_14707_gb300 import build as lbm_build
from paper_2012_14707_gb300 import cases, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm_build.build()
    lbm.load()


@pytest.mark.parametrize("precision,moving", [("fp32", False), ("bf16", False), ("fp16", False),
                                             ("fp64", False), ("fp32", True)])
def test_resume_from_checkpoint_is_bitwise(tmp_path, precision, moving):
    """16-bit storage rounds stochastically with random bits keyed by the
    step count, which the file restores; FP32 with a moving wall runs the
    exact-mass step, whose carries the file holds too."""
    if moving:
        c = cases.channel(37, 9, 0.2, 0.85, Kn=0.05, ax=1e-6, u_top=0.01)
    else:
        c = cases.cylinder_array(120, 80, 4, Kn=0.02, ax=1e-5)
    path = str(tmp_path / "state.bin")
    a = lbm.Solver(c, precision=precision)
    assert a.info().exact_mass == int(moving)
    a.step(300)
    a.save(path)
    a.step(200)
    want_f, want_res, want_fields = a.get_f(), a.residual(), a.fields()
    a.close()
    b = lbm.Solver(c, precision=precision)
    b.load(path)
    assert b.info().steps == 300
    b.step(200)
    np.testing.assert_array_equal(b.get_f(), want_f)
    assert b.residual() == want_res
    for x, y in zip(b.fields(), want_fields):
        np.testing.assert_array_equal(x, y)
    b.close()


def test_checkpoint_of_another_case_or_a_damaged_file_is_refused(tmp_path):
    c = cases.cylinder_array(120, 80, 4, Kn=0.02, ax=1e-5)
    path = str(tmp_path / "state.bin")
    a = lbm.Solver(c, precision="fp32")
    a.step(10)
    a.save(path)
    a.close()
    other = cases.cylinder_array(120, 80, 5, Kn=0.02, ax=1e-5)   # same size, other seed
    for case, prec, word in ((other, "fp32", "another case"), (c, "fp64", "precision")):
        s = lbm.Solver(case, precision=prec)
        with pytest.raises(lbm.LbmError) as ei:
            s.load(path)
        assert ei.value.code == lbm.LBM_EINVAL and word in str(ei.value)
        s.close()
    s = lbm.Solver(c, precision="fp32")
    with pytest.raises(lbm.LbmError) as ei:
        s.load(str(tmp_path / "missing.bin"))
    assert ei.value.code == lbm.LBM_EIO
    raw = open(path, "rb").read()
    open(tmp_path / "short.bin", "wb").write(raw[:len(raw) // 2])
    with pytest.raises(lbm.LbmError) as ei:
        s.load(str(tmp_path / "short.bin"))
    assert ei.value.code == lbm.LBM_EIO
    open(tmp_path / "magic.bin", "wb").write(b"XXXXXXXX" + raw[8:])
    with pytest.raises(lbm.LbmError) as ei:
        s.load(str(tmp_path / "magic.bin"))
    assert ei.value.code == lbm.LBM_EINVAL
    # a refused load leaves the solver usable
    s.step(5)
    assert np.isfinite(s.residual()[0])
    s.close()
