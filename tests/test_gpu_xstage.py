"""The FP32-bulk x sweep with its rows staged in shared memory by bulk asynchronous copies
(kb_euler_x_staged, MHD_OPT_X_STAGE = 1) against the same sweep reading global memory (the default): the same
arithmetic on the same values, so the states agree bit for bit, on periodic and outflow boxes,
boxes whose tiles span many rows, and a box whose n_x is not a multiple of 4 (which the launcher
leaves on the direct kernel).  Also the copy and its bounded mbarrier wait on their own: a copy
arrives whole, and a phase that no copy can complete gives up after about a second with a status
the host reads, leaving the context usable."""
import numpy as np
import pytest

from paper_1608_08748_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_08748_gb300 import build as B
    B.build()
    import paper_1608_08748_gb300 as M
    return M


CASES = {
    "periodic_40x24x16": dict(shape=(16, 24, 40), opts={}),
    "outflow_x_36x20x12": dict(shape=(12, 20, 36), opts={"bc_x": 1}),
    "many_rows_16x8x8": dict(shape=(8, 8, 16), opts={"bc_y": 1}),
    "ragged_nx_42": dict(shape=(6, 10, 42), opts={}),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_x_staging_matches_direct_reads(M, case):
    c = CASES[case]
    ic = I.turbulence(8, mach=3.0, beta=1.0, seed=37, shape=c["shape"])
    states = []
    for stage in (1, 0):
        s = M.from_ic(ic, precision=1, x_stage=stage, **c["opts"])
        for _ in range(6):
            s.step(0.4)
        states.append(s.get_state())
        s.close()
    for k in ("rho", "mom", "E", "B", "rho_h2"):
        assert np.array_equal(states[0][k], states[1][k]), k


def test_x_staging_in_a_batch(M):
    """Two boxes stepped as one batch (both rows staged) equal the same boxes stepped alone."""
    ics = [I.turbulence(8, mach=2.0, beta=1.0, seed=41, shape=(12, 16, 24)),
           I.turbulence(8, mach=4.0, beta=0.5, seed=42, shape=(8, 20, 32))]
    solo = []
    for ic in ics:
        s = M.from_ic(ic, precision=1, x_stage=0)
        for _ in range(4):
            s.step(0.4)
        solo.append(s.get_state())
        s.close()
    sims = [M.from_ic(ic, precision=1, x_stage=1) for ic in ics]
    b = M.Batch(sims)
    for _ in range(4):
        b.step(0.4)
    b.sync()
    for s, ref in zip(sims, solo):
        st = s.get_state()
        for k in ("rho", "mom", "E", "B"):
            assert np.array_equal(st[k], ref[k]), k


@pytest.fixture(scope="module")
def bulk(tmp_path_factory):
    import ctypes
    import os
    import subprocess
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    lib = str(tmp_path_factory.mktemp("bulk") / "libbulk_selftest.so")
    subprocess.run([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                    "-I", os.path.join(root, "paper_1608_08748_gb300", "csrc"), "-I", os.path.join(root, "include"),
                    os.path.join(here, "gpu_selftest", "bulk_selftest.cu"), "-o", lib], check=True)
    L = ctypes.CDLL(lib)
    L.selftest_bulk.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return L


def _bulk(L, n, extra):
    import torch
    src = torch.arange(n, dtype=torch.float32, device="cuda") * 0.5 + 1.0
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = L.selftest_bulk(src.data_ptr(), n, extra, out.data_ptr(), status.data_ptr())
    assert rc == 0, rc
    return src.cpu().numpy(), out.cpu().numpy(), int(status.item())


def test_bulk_copy_arrives_whole(bulk):
    src, out, status = _bulk(bulk, 4096, 0)
    assert status == 1
    assert np.array_equal(src, out)


def test_bulk_copy_wait_is_bounded(bulk):
    import time
    t0 = time.perf_counter()
    _, out, status = _bulk(bulk, 1024, 16)  # 16 bytes announced that no copy delivers
    elapsed = time.perf_counter() - t0
    assert status == 2
    assert elapsed < 30.0
    assert not out.any()
    src, out, status = _bulk(bulk, 1024, 0)  # the context still works
    assert status == 1 and np.array_equal(src, out)


def test_x_stage_option_values(M):
    """MHD_OPT_X_STAGE takes 0 or 1; anything else is MHD_EINVAL and leaves the sim usable."""
    ic = I.turbulence(8, mach=1.0, beta=1.0, seed=43, shape=(8, 8, 16))
    s = M.from_ic(ic, precision=1)
    for bad in (2, -1, 0.5):
        with pytest.raises(M.MHDError) as e:
            s.set_option("x_stage", bad)
        assert "EINVAL" in str(e.value)
    s.set_option("x_stage", 1)
    s.step(0.4)
    s.set_option("x_stage", 0)
    s.step(0.4)
    s.close()
