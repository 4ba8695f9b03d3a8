"""Bounds-checked build as a sanitizer substitute: every walk kernel, the
voxelizer and its adjoint and full optimisation steps run once with the
default library and once with libdgr_checked.so (built with
-DDGR_CHECK_BOUNDS: the volume, integer-sum, gradient and record accesses test
their indices and set DGR_STATUS_BOUNDS, skipping the access, for an index
outside its buffer).  No status word may be set, and the outputs must be the
same bits: the checks only skip accesses that never happen."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2411_04844_b300 import build as B, dgr
from tests import _bounds_cases as C

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checked_build_reports_nothing_and_matches(tmp_path):
    B.build(checked=True)
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, DGR_CHECK_BOUNDS="1", PYTHONPATH=ROOT)
    subprocess.run([sys.executable, "-m", "tests._bounds_cases", path], cwd=ROOT, env=env, check=True,
                   timeout=600)
    with np.load(path) as z:
        chk = {k.replace("__", "/"): z[k] for k in z.files}
    assert any("libdgr_checked.so" in s for s in chk.pop("libs")), "the child did not load the checked library"
    ref = C.run_cases()
    assert set(ref) == set(chk)
    for k in sorted(ref):
        if k.split("/")[1].startswith("status"):
            assert int(chk[k]) == 0, (k, hex(int(chk[k])))
            assert int(ref[k]) == 0, (k, hex(int(ref[k])))
        else:
            assert np.array_equal(chk[k], ref[k]), k
            assert np.isfinite(ref[k]).all(), k
