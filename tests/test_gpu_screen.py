"""Two pieces of the post kernel's arithmetic on the GPU, under the compile flags of both paths (the
FP64 translation unit's, and the FP32-bulk one's: flush to zero, approximate division and square
root), built from tests/gpu_selftest/screen_selftest.cu:

- the chemistry's table-driven exponential (Tang's method, Sec. 2.7 / App. D rates) within 2 ulp
  of the library exp on the GPU and of numpy's on the host, over the rates' argument range;
- the FP32 estimate of the CFL screen (Sec. 2.3) within 64 u (u = 2^-24) of the FP64 denominator
  of the same cell wherever its guards pass.  tau takes the largest FP64 denominator over the cells,
  and the post kernel skips the FP64 evaluation of a cell only where its estimate raised by 2^-12
  stays below an FP64 denominator already reached; with the estimate this close, no skipped cell
  can hold the maximum, so tau equals that of evaluating every cell.  Flushed subnormal squares,
  densities and internal energies over many decades, zero components and unphysical abundances
  are among the inputs;
- end to end, tau of steps whose maximum is held by one cell and falls fast equal to the oracle's
  (FP64 within 1e-11, FP32 within 1e-4), and a batch holding that box stepping as its boxes do
  alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
FLAGS = {"fp64": ["--fmad=true"],
         "fp32": ["--fmad=true", "-prec-div=false", "-prec-sqrt=false", "-ftz=true"]}


class _Selftest:
    def __init__(self, path):
        import ctypes
        self.L = ctypes.CDLL(path)
        for f in (self.L.selftest_exp, self.L.selftest_screen):
            f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]

    def _run(self, f, a, cols_out):
        import torch
        d = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()
        n = d.shape[0]
        out = torch.empty((n, cols_out), dtype=torch.float64, device=d.device)
        rc = f(d.data_ptr(), n, out.data_ptr())
        assert rc == 0, rc
        return out.cpu().numpy()

    def exp(self, x):
        return self._run(self.L.selftest_exp, x, 2)

    def screen(self, w):
        return self._run(self.L.selftest_screen, w, 2)


@pytest.fixture(scope="module", params=sorted(FLAGS))
def S(request, tmp_path_factory):
    import os
    import subprocess
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    lib = str(tmp_path_factory.mktemp("screen_" + request.param) / "libscreen_selftest.so")
    subprocess.run([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    "-std=c++17", *FLAGS[request.param], "-Xcompiler", "-fPIC", "-shared",
                    "-I", os.path.join(root, "paper_1608_08748_gb300", "csrc"), "-I", os.path.join(root, "include"),
                    os.path.join(here, "gpu_selftest", "screen_selftest.cu"), "-o", lib], check=True)
    return _Selftest(lib)


def _ulp_distance(a, b):
    """Distance in units in the last place between doubles of one sign (by their ordered bits)."""
    ia, ib = a.view(np.int64), b.view(np.int64)
    return np.abs(ia - ib)


def test_exp_tang_within_two_ulp(S):
    rng = np.random.default_rng(1608)
    x = np.concatenate([
        -746.0 * rng.random(200000), -rng.random(100000), -20.0 * rng.random(100000),
        -np.ldexp(1.0 + rng.random(100000), -rng.integers(0, 60, 100000)),
        np.array([0.0, -0.0, -5e-324, -1e-300, -707.0, -706.9999999999999, -707.0000000000001, -708.0,
                  -708.4, -745.0, -745.13, -746.0]),
    ])
    o = S.exp(x)
    ours, lib = o[:, 0], o[:, 1]
    host = np.exp(x)
    assert np.all(_ulp_distance(ours, lib) <= 2)
    assert np.all(_ulp_distance(ours, host) <= 2)


def _screen_inputs(n, seed):
    rng = np.random.default_rng(seed)

    def logu(lo, hi, size):
        return np.exp(rng.uniform(np.log(lo), np.log(hi), size))

    kind = np.arange(n) % 4
    chem = (np.arange(n) // 4) % 2
    rho = np.where(kind == 0, logu(1e-13, 1e13, n), logu(1e-3, 1e3, n))
    w = np.zeros((n, 12))
    w[:, 0] = rho
    for d in range(3):
        mag_m = np.where(kind == 1, logu(1e-30, 1e10, n), logu(1e-3, 1e3, n))
        mag_b = np.where(kind == 2, logu(1e-30, 1e10, n), logu(1e-3, 1e3, n))
        w[:, 1 + d] = np.where(rng.random(n) < 0.1, 0.0, rng.uniform(-1, 1, n) * mag_m)
        w[:, 4 + d] = np.where(rng.random(n) < 0.2, 0.0, rng.uniform(-1, 1, n) * mag_b)
    w[:, 7] = rho * np.where(kind == 3, logu(1e-16, 1e8, n), logu(1e-4, 1e4, n))
    fhp = np.where(np.arange(n) % 3 == 0, 0.0, 0.1 * rng.random(n))
    rh2 = rho * rng.random(n) * (1.0 - fhp)
    odd = np.arange(n) % 97 == 0
    rh2[odd] = rho[odd] * (1.0 + 0.5 * rng.random(odd.sum()))  # more H2 than gas
    w[:, 8], w[:, 9] = rh2, rho * fhp
    w[:, 10] = np.where(chem == 1, 5.0 / 3.0, 1.0 + logu(1e-4, 0.67, n))
    w[:, 11] = chem
    # half the cells as the FP32 path holds them (float values widened)
    half = np.arange(n) % 2 == 1
    w[half, :10] = w[half, :10].astype(np.float32).astype(np.float64)
    return w


def test_cfl_screen_estimate_within_64u(S):
    w = _screen_inputs(400000, 2016)
    o = S.screen(w)
    est, exact = o[:, 0], o[:, 1]
    screened = est <= 3.0e38
    assert screened.mean() > 0.5
    assert np.all(np.isfinite(exact[screened]) & (exact[screened] > 0))
    rel = np.abs(est[screened] - exact[screened]) / exact[screened]
    assert rel.max() <= 64 * U, rel.max()


# ------------------------------------------------------------------------------------------------
# The screened maximum end to end (Sec. 2.3), where one cell holds it and it falls fast.  A
# low-density cell at the background's pressure and velocity sets the maximum (its sound speed is
# 10 times the background's) and fills with denser fluid within a few steps: the oracle's tau grows
# by 1.79, 1.41, 1.25 and 1.17 over the first four steps.  One warp holds the maximum, every other
# warp's estimates lie far below it, and the box's running maximum starts from zero each step.

@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_08748_gb300 import build as B
    B.build()
    import paper_1608_08748_gb300 as M
    return M


def _low_density_cell(n=16, v=3.0, rlow=0.01):
    from paper_1608_08748_gb300 import inputs as I
    B = (0.5, 0.3, 0.2)
    ic = I.uniform(n, n, n, rho=1.0, p=1.0, v=(v, 0.0, 0.0), B=B, dx=1.0 / n)
    g = ic["gamma"]
    k = (n // 2, n // 2, n // 2)
    ic["rho"][k] = rlow
    ic["mom"][0][k] = rlow * v
    ic["E"][k] = 1.0 / (g - 1.0) + 0.5 * rlow * v * v + 0.5 * sum(b * b for b in B)
    return ic


def test_cfl_maximum_held_by_one_falling_cell(M, oracle_mod):
    from test_gpu_parity import compare
    ic = _low_density_cell()
    o = oracle_mod.run(ic)
    g = M.from_ic(ic)
    taus = []
    for _ in range(5):
        dg, do = g.step(0.4), o.step(0.4)
        assert abs(dg - do) <= 1e-11 * do, (dg, do)
        taus.append(do)
    assert all(taus[i + 1] / taus[i] > 8.0 / 7.0 for i in range(3)), taus
    compare(g.get_state(), o.get_state())


def test_cfl_maximum_of_one_cell_fp32_and_batched(M, oracle_mod):
    ic = _low_density_cell()
    o = oracle_mod.run(ic)
    g32 = M.from_ic(ic, precision=1)
    for _ in range(5):
        dg, do = g32.step(0.4), o.step(0.4)
        assert abs(dg - do) <= 1e-4 * do, (dg, do)
    # per-box maxima in a batch: the box with the falling maximum beside a uniform box, both as they
    # step alone
    from paper_1608_08748_gb300 import inputs as I
    from paper_1608_08748_gb300.mhd import Batch
    ics = [ic, I.uniform(12, 10, 8, rho=1.0, p=2.0, v=(0.5, 0.1, 0.0), B=(0.2, 0.0, 0.1), dx=1.0 / 12)]
    solo = [M.from_ic(x) for x in ics]
    for s in solo:
        for _ in range(5):
            s.step(0.4)
    sims = [M.from_ic(x) for x in ics]
    b = Batch(sims)
    for _ in range(5):
        b.step(0.4)
    b.sync()
    for a, s in zip(sims, solo):
        sa, ss = a.get_state(), s.get_state()
        for k in ("rho", "mom", "E", "B"):
            assert np.array_equal(sa[k], ss[k]), k
        assert a.diagnostics()["t"] == s.diagnostics()["t"]
