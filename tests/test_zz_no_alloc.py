"""mhd_diagnostics_noalloc: the diagnostics entry point for callers that cannot allocate device
memory (stream capture in global mode, a fully committed HBM budget, monitors inside another
application's time loop).  Its output must equal that of mhd_diagnostics, which uses scratch the
simulation allocated, on two calls in a row.

This file is collected last on purpose, so a run that stops at the first failure has already run
every other test."""
import ctypes as C
import os
import sys

import numpy as np
import pytest

from paper_1608_08748_gb300 import inputs as I

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu
TOL = 1e-12


def _noalloc_fn(M):
    fn = M.lib().mhd_diagnostics_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p] * 8 + [C.c_int] * 6 + [C.c_void_p, C.c_void_p]
    return fn


def _device_state(M, torch, sim, shape):
    """Caller-owned device copies of the cell fields and the face fields."""
    out = {"rho": torch.empty(shape, dtype=torch.float64, device="cuda"),
           "mom": torch.empty((3,) + shape, dtype=torch.float64, device="cuda"),
           "E": torch.empty(shape, dtype=torch.float64, device="cuda"),
           "B": torch.empty((3,) + shape, dtype=torch.float64, device="cuda"),
           "rho_h2": None}
    sim.get_state(out=out)
    faces = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(4)]
    rc = M.lib().mhd_get_full(sim.h, *[f.data_ptr() for f in faces], 1)
    assert rc == 0, M.lib().mhd_last_error()
    torch.cuda.synchronize()
    return out, faces[1:]


def test_noalloc_diagnostics_match_allocating_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_08748_gb300 import build as B
    B.build()
    import paper_1608_08748_gb300 as M

    shape = (20, 24, 28)
    ic = I.turbulence(8, mach=3.0, seed=11, shape=shape)
    sim = M.from_ic(ic)
    fn = _noalloc_fn(M)
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    keys = ["rho", "mx", "my", "mz", "E", "bx", "by", "bz", "max_div_b_h"]
    for call in range(2):
        sim.step(0.4)  # a different state for each call: stale partials would show
        want = sim.diagnostics()
        st, faces = _device_state(M, torch, sim, shape)
        out.fill_(float("nan"))
        args = [st["rho"].data_ptr(), st["mom"][0].data_ptr(), st["mom"][1].data_ptr(),
                st["mom"][2].data_ptr(), st["E"].data_ptr()] + [f.data_ptr() for f in faces]
        rc = fn(*args, shape[2], shape[1], shape[0], 0, 0, 0, out.data_ptr(), None)
        assert rc == 0, M.lib().mhd_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for q, k in enumerate(keys):
            scale = max(abs(want[k]), abs(want["rho"]) * 1e-12, 1e-300)
            assert abs(got[q] - want[k]) <= TOL * scale, (call, k, got[q], want[k])


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 1)], ids=["periodic", "outflow_xz"])
def test_noalloc_diagnostics_match_the_oracle(oracle_mod, bc):
    """The same nine values against the oracle's diagnostics of the same state (sums to 1e-12 of
    the sum of |terms|; max |div b| h, here of order the field's variation, to 1e-12 of max |b|),
    right after the load and after three steps, with periodic and with outflow upper faces."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_08748_gb300 import build as B
    B.build()
    import paper_1608_08748_gb300 as M
    import test_gpu_diagnostics as TD

    shape = (14, 17, 20)
    ic = TD.divergent_turbulence(shape)
    ic["options"] = dict(ic["options"], bc_x=bc[0], bc_y=bc[1], bc_z=bc[2])
    sim = M.from_ic(ic)
    o = oracle_mod.run(ic)
    fn = _noalloc_fn(M)
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    keys = ["rho", "mx", "my", "mz", "E", "bx", "by", "bz", "max_div_b_h"]
    for call in range(2):
        st, faces = _device_state(M, torch, sim, shape)
        out.fill_(float("nan"))
        args = [st["rho"].data_ptr(), st["mom"][0].data_ptr(), st["mom"][1].data_ptr(),
                st["mom"][2].data_ptr(), st["E"].data_ptr()] + [f.data_ptr() for f in faces]
        rc = fn(*args, shape[2], shape[1], shape[0], bc[0], bc[1], bc[2], out.data_ptr(), None)
        assert rc == 0, M.lib().mhd_last_error()
        torch.cuda.synchronize()
        got = dict(zip(keys, out.cpu().numpy().tolist()))
        TD.check(got, o.diag(), o, 1e-12)
        for _ in range(3):
            sim.step(0.4)
            o.step(0.4)


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_08748_gb300 import build as B
    B.build()
    import paper_1608_08748_gb300 as M
    fn = _noalloc_fn(M)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    rc = fn(p, p, p, p, p, p, p, p, 256, 256, 128, 0, 0, 0, p, None)  # 8.4M cells > 4,194,304
    assert rc == -1
    assert b"exceed the fixed maximum" in M.lib().mhd_last_error()
