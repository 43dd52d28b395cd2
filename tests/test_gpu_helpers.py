"""The FP64 path's arithmetic helpers on the GPU (inline PTX on the integer pipes and Newton-Raphson
steps from the hardware seeds), checked element by element against their definitions on special and
random doubles over the whole exponent range: |x| and -x bit for bit; x/2 and x/4 equal to the
product where it is normal, zero, infinite or NaN, else the zero of the sign of x; the ordered keys
sort the values in their order (-0 below +0); 1/x, 1/sqrt(x) and sqrt(x) within 2 ulp of the
correctly rounded values for normal arguments."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TINY = np.finfo(np.float64).tiny  # smallest normal double


class _Selftest:
    """The helpers run over an array on the device: an (n, 8) float64 array of |x|, -x, x/2, x/4,
    the ordered key of x (its bits), 1/x, 1/sqrt|x|, sqrt|x| (tests/gpu_selftest/helpers_selftest.cu,
    built here with nvcc for sm_103a; not part of libmhd.so)."""

    def __init__(self, path):
        import ctypes
        self.L = ctypes.CDLL(path)
        self.L.selftest_helpers.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]

    def selftest_helpers(self, x):
        import torch
        xd = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64).ravel()).cuda()
        out = torch.empty((xd.numel(), 8), dtype=torch.float64, device=xd.device)
        rc = self.L.selftest_helpers(xd.data_ptr(), xd.numel(), out.data_ptr())
        assert rc == 0, rc
        return out.cpu().numpy()


@pytest.fixture(scope="module")
def M(tmp_path_factory):
    import os
    import subprocess
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    lib = str(tmp_path_factory.mktemp("selftest") / "libhelpers_selftest.so")
    subprocess.run([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    "-std=c++17", "--fmad=true", "-Xcompiler", "-fPIC", "-shared",
                    "-I", os.path.join(root, "paper_1608_08748_gb300", "csrc"), "-I", os.path.join(root, "include"),
                    os.path.join(here, "gpu_selftest", "helpers_selftest.cu"), "-o", lib], check=True)
    return _Selftest(lib)


def inputs():
    rng = np.random.default_rng(71)
    special = [0.0, -0.0, 1.0, -1.0, TINY, -TINY, 2 * TINY, 4 * TINY, 3 * TINY, TINY / 2, -TINY / 3,
               5e-324, -5e-324, np.finfo(np.float64).max, -np.finfo(np.float64).max, np.inf, -np.inf,
               np.nan, 2.0 ** -1020, 2.0 ** -1021, -(2.0 ** -1021), 0.1, 1e-300, 1e300]
    mant = rng.uniform(1.0, 2.0, 20000)
    expo = rng.integers(-1074, 1024, 20000)
    rand = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], 20000)
    return np.concatenate([np.array(special), rand, rng.normal(size=2000)])


def bits(a):
    return np.asarray(a, dtype=np.float64).view(np.int64)


def test_sign_and_magnitude_bit_for_bit(M):
    x = inputs()
    o = M.selftest_helpers(x)
    fin = ~np.isnan(x)
    assert np.array_equal(bits(o[fin, 0]), bits(np.abs(x[fin])))
    assert np.array_equal(bits(o[fin, 1]), bits(-x[fin]))
    assert np.isnan(o[~fin, 0]).all() and np.isnan(o[~fin, 1]).all()


@pytest.mark.parametrize("col,k", [(2, 1), (3, 2)])
def test_power_of_two_scaling(M, col, k):
    x = inputs()
    o = M.selftest_helpers(x)[:, col]
    with np.errstate(under="ignore"):
        prod = x / 2.0 ** k
    nan = np.isnan(x)
    assert np.isnan(o[nan]).all()
    exact = ~nan & ((np.abs(prod) >= TINY) | (x == 0) | np.isinf(x))
    assert np.array_equal(bits(o[exact]), bits(prod[exact]))
    flushed = ~nan & ~exact
    assert flushed.any()
    assert np.array_equal(bits(o[flushed]), bits(np.copysign(0.0, x[flushed])))


def test_ordered_keys_sort_like_the_values(M):
    x = inputs()
    x = x[~np.isnan(x)]
    keys = M.selftest_helpers(x)[:, 4].view(np.int64)
    # value order with -0 below +0: sort by (value, sign bit set first)
    order_vals = np.lexsort((~np.signbit(x), x))
    order_keys = np.argsort(keys, kind="stable")
    assert np.array_equal(x[order_vals].view(np.int64), x[order_keys].view(np.int64))
    assert keys[np.flatnonzero(bits(x) == bits(np.array(0.0)))[0]] == 0
    assert keys[np.flatnonzero(bits(x) == bits(np.array(-0.0)))[0]] == -1


def test_newton_raphson_forms_within_two_ulp(M):
    x = inputs()
    o = M.selftest_helpers(x)
    a = np.abs(x)
    with np.errstate(all="ignore"):
        normal = np.isfinite(x) & (a >= TINY) & (1.0 / a >= TINY) & np.isfinite(1.0 / a)
        # references rounded once from extended precision
        xl, al = x.astype(np.longdouble), a.astype(np.longdouble)
        r = (1 / xl).astype(np.float64)
        rs = (1 / np.sqrt(al)).astype(np.float64)
        sq = np.sqrt(a)
    for got, ref in [(o[:, 5], r), (o[:, 6], rs), (o[:, 7], sq)]:
        err = np.abs(got[normal] - ref[normal]) / np.spacing(np.abs(ref[normal]))
        assert err.max() <= 2.0, err.max()
    assert normal.sum() > 15000
