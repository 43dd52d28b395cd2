"""GPU checks at the full sizes of the FP32-bulk, batched and largest configurations.

- Config 3 (256^3 turbulence with chemistry, FP32 bulk): per-field relative L1 against the FP64
  GPU path (itself within 1e-14 of the oracle at 128^3 after 50 steps) after 3 steps, <= 1e-4.
- Config 4 (the 64-box ensemble, FP32 bulk, one batched launch per kernel class): every member
  after 3 batched steps equals the same box stepped alone, bit for bit.
- The largest box (512^3, FP32, 1.35e8 lattice points, the limit of 32-bit indices is 2^31): a
  state that varies only along x stays the same in every (y, z) column and equals the 512 x 4 x 4
  box with the same x-profile bit for bit after 2 steps (index arithmetic at that size), and the
  FP64 mass sum is conserved to FP32 rounding."""
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


def test_config3_fp32_256_against_the_fp64_path(M):
    from test_gpu_parity import compare
    ic = I.turbulence(256, mach=5.0, beta=1.0, seed=1)
    s32 = M.from_ic(ic, precision=1)
    s64 = M.from_ic(ic, precision=0)
    for _ in range(3):
        s32.step(0.4, sync=False)
        s64.step(0.4, sync=False)
    s32.sync()
    s64.sync()
    errs = compare(s32.get_state(), s64.get_state(), tol=1e-4)
    print("config 3 FP32 vs FP64 rel L1:", {k: f"{v:.1e}" for k, v in errs.items()})


def test_config4_ensemble_batched_equals_solo(M):
    boxes = I.ensemble_boxes()
    ics = [I.turbulence(8, mach=b["mach"], beta=b["beta"], seed=b["seed"], shape=b["shape"]) for b in boxes]
    mixed = [M.from_ic(ic, precision=1) for ic in ics]
    batch = M.Batch(mixed)
    for _ in range(3):
        batch.step(0.4)
    batch.sync()
    for k in range(0, len(ics), 7):  # every seventh member, all sizes of the table among them
        solo = M.from_ic(ics[k], precision=1)
        for _ in range(3):
            solo.step(0.4, sync=False)
        solo.sync()
        a, b = solo.get_state(dtype=M.mhd.F32), mixed[k].get_state(dtype=M.mhd.F32)
        for f in ["rho", "E", "mom", "B", "rho_h2"]:
            assert np.array_equal(a[f], b[f]), (k, f)
    batch.close()


def _x_profile_state(nx):
    """A smooth state that varies only along x (periodic): density, velocity, field and H2 waves
    of the turbulence set-up's units (n = 100, T = 100 K, about Mach 2.5), chemistry on."""
    x = (np.arange(nx) + 0.5) / nx
    s = np.sin(2 * np.pi * x)[None, None, :]
    c = np.cos(2 * np.pi * x)[None, None, :]
    rho = 100.0 * (1.0 + 0.2 * s)
    p = 82.5 * (1.0 + 0.1 * c)
    v = np.stack([3.0 * s, 1.0 * c, 0.5 * s])
    B = np.stack([8.0 + 0 * s, 6.0 * s, 4.0 + 0 * s])
    ic = I.conserved(rho, v, p, B, 5.0 / 3.0, 0.01 * rho)
    return ic


def _broadcast(ic, shape, dtype):
    out = {}
    for k in ["rho", "E", "rho_h2"]:
        out[k] = np.ascontiguousarray(np.broadcast_to(ic[k].astype(dtype), shape))
    for k in ["mom", "B"]:
        out[k] = np.ascontiguousarray(np.broadcast_to(ic[k].astype(dtype), (3,) + shape))
    return out


def test_largest_box_512_fp32_columns_and_profile(M):
    nx = 512
    ic1 = _x_profile_state(nx)
    opts = dict(bc_x=0, bc_y=0, bc_z=0, chem=1, precision=1)
    dx = 256.0 / nx
    small_f = _broadcast(ic1, (4, 4, nx), np.float32)
    small = M.Sim(nx, 4, 4, 5.0 / 3.0, dx, **opts)
    small.set_state(small_f["rho"], small_f["mom"], small_f["E"], small_f["B"], small_f["rho_h2"])
    big_f = _broadcast(ic1, (nx, nx, nx), np.float32)
    big = M.Sim(nx, nx, nx, 5.0 / 3.0, dx, **opts)
    big.set_state(big_f["rho"], big_f["mom"], big_f["E"], big_f["B"], big_f["rho_h2"])
    del big_f
    m0 = big.diagnostics()["rho"]
    for _ in range(2):
        ds, db = small.step(0.4), big.step(0.4)
        assert ds == db
    m1 = big.diagnostics()["rho"]
    assert abs(m1 - m0) <= 1e-6 * abs(m0), (m0, m1)
    a = small.get_state(dtype=M.mhd.F32)
    b = big.get_state(dtype=M.mhd.F32)
    for f in ["rho", "E", "rho_h2", "mom", "B"]:
        prof = a[f][..., 0:1, 0:1, :]
        assert np.array_equal(a[f], np.broadcast_to(prof, a[f].shape)), f
        assert np.array_equal(b[f], np.broadcast_to(prof, b[f].shape)), f
        del prof
