"""The compacted lattice's index arithmetic, checked on the host (no GPU):
tests/native/compact_layout_check.cu links the library, builds each case's
compacted layout with the library's own code, and compares the neighbour
indices the step kernels compute (compact_targets) and the
pull slots they gather from (pull_slots, the per-link f_jb slots) with the
dense neighbourhood and the link table, for every fluid node and
direction.  A wrong index would be a silent out-of-bounds access on the
GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2012_14707_gb300 import build as lbm_build
from paper_2012_14707_gb300 import cases

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _dump(c, path):
    with open(path, "wb") as f:
        np.array([c.nx, c.ny, int(c.periodic_x), int(c.periodic_y)], np.int32).tofile(f)
        c.solid.astype(np.uint8).tofile(f)


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc to build the host-side checker")
def test_compact_targets_match_the_dense_neighbourhood(tmp_path):
    lib = lbm_build.build()
    libdir = os.path.dirname(lib)
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "compact_layout_check")
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2012_14707_gb300", "csrc"),
                           "-o", exe, os.path.join(HERE, "native", "compact_layout_check.cu"),
                           "-L", libdir, "-llbm", "-Xlinker", f"-rpath={libdir}"])
    files = []
    for k, c in enumerate([cases.inclined_channel(120, 1.2, 16, Kn=0.0194),
                           cases.inclined_channel(120, 0.2, 4, Kn=0.0194),
                           cases.annulus(72, 20.0, 32.0, 0.05, 0.001),
                           cases.cylinder_array(1024, 512, 3, Kn=0.02, ax=1e-5),
                           cases.config_poiseuille(),
                           cases.periodic_box(1, 7, ax=1e-5)]):
        path = str(tmp_path / f"case{k}.bin")
        _dump(c, path)
        files.append(path)
    out = subprocess.run([exe, *files], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "ALL OK" in out.stdout
    print(out.stdout)
