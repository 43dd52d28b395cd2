"""The index-checked build (in place of a memory checker): libmhd_check.so, compiled with
-DMHD_CHECK, tests every computed cell and lattice index of its kernels against its array and
records a bad one (replacing it by an in-bounds index).  Small, ragged and degenerate boxes, FP64
and FP32, periodic and outflow, a batch, self-gravity and the ion network run through it in a child
process; the flags must stay 0."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu


def test_checked_build_sees_no_bad_index():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    here = os.path.dirname(os.path.abspath(__file__))
    out = subprocess.run([sys.executable, os.path.join(here, "gpu_selftest", "checked_run.py")],
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["runs"] >= 30 and res["flags"] == 0, res
