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
