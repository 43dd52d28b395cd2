"""The C-ABI library builds, loads and exports every function include/mhd.h declares (no GPU
needed: nothing here calls into the device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(mhd_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libmhd():
    from paper_1608_08748_gb300 import build as B
    try:
        path = B.build()
    except FileNotFoundError:
        pytest.skip("nvcc not available")
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mhd_create", "mhd_destroy", "mhd_set_state", "mhd_get_state", "mhd_step",
                     "mhd_advance", "mhd_diagnostics", "mhd_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libmhd):
    missing = [n for n in declared_functions() if not hasattr(libmhd, n)]
    assert not missing, missing


def test_bytes_needed_is_host_only(libmhd):
    f = libmhd.mhd_bytes_needed
    f.restype = ctypes.c_size_t
    f.argtypes = [ctypes.c_int] * 5
    small, big = f(16, 16, 16, 0, 1), f(32, 32, 32, 0, 1)
    assert 7.0 < big / small < 8.5
    assert f(64, 64, 64, 1, 1) < f(64, 64, 64, 0, 1)


def test_argument_errors_are_reported_without_a_device(libmhd):
    """Bad arguments are rejected on the host, before any CUDA call: the calls return MHD_EINVAL (or
    NULL) and mhd_last_error names the call."""
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    libmhd.mhd_last_error.restype = ctypes.c_char_p
    err = lambda: libmhd.mhd_last_error().decode()
    EINVAL = -1

    libmhd.mhd_create.restype = vp
    libmhd.mhd_create.argtypes = [i, i, i, d, d]
    for args in [(0, 4, 4, 1.4, 1.0), (4, 4, 4, 1.0, 1.0), (4, 4, 4, 1.4, 0.0), (2048, 2048, 1024, 1.4, 1.0)]:
        assert libmhd.mhd_create(*args) is None
        assert "mhd_create" in err()

    libmhd.mhd_set_option.argtypes = [vp, i, d]
    assert libmhd.mhd_set_option(None, 4, 1.0) == EINVAL and "mhd_set_option" in err()
    libmhd.mhd_step.argtypes = [vp, d, vp]
    assert libmhd.mhd_step(None, 0.4, None) == EINVAL and "mhd_step" in err()
    libmhd.mhd_set_ions.argtypes = [vp, vp, i]
    assert libmhd.mhd_set_ions(None, None, 0) == EINVAL and "mhd_set_ions" in err()
    libmhd.mhd_get_ions.argtypes = [vp, vp, i]
    assert libmhd.mhd_get_ions(None, None, 0) == EINVAL and "mhd_get_ions" in err()
    libmhd.mhd_batch_create.restype = vp
    libmhd.mhd_batch_create.argtypes = [vp, i]
    assert libmhd.mhd_batch_create(None, 0) is None and "mhd_batch_create" in err()
    libmhd.mhd_server_set_policy.argtypes = [vp, i]
    assert libmhd.mhd_server_set_policy(None, 0) == EINVAL and "mhd_server_set_policy" in err()


def test_binding_option_keys_match_the_header():
    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    enum = re.search(r"enum mhd_option\s*\{(.*?)\};", src, flags=re.S).group(1)
    header = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"MHD_OPT_([A-Z0-9_]+)\s*=\s*(\d+)", enum)}
    from paper_1608_08748_gb300 import mhd
    assert mhd.OPT == header
