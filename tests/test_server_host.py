"""Host-side logic of the request server (no device work happens in these paths): argument
checks and admission refusal of a request that can never fit the HBM budget."""
import numpy as np
import pytest

from paper_1608_08748_gb300 import inputs as I


@pytest.fixture(scope="module")
def M():
    from paper_1608_08748_gb300 import build as B
    try:
        B.build()
    except FileNotFoundError:
        pytest.skip("nvcc not available")
    import paper_1608_08748_gb300 as M
    return M


def test_bad_server_arguments(M):
    with pytest.raises(M.MHDError):
        M.Server(0, 4)
    with pytest.raises(M.MHDError):
        M.Server(1 << 20, 0)


def test_request_checks_and_capacity(M):
    srv = M.Server(64 << 20, 4)  # 64 MiB
    ic = I.uniform(8, 8, 8)
    with pytest.raises(M.MHDError) as e:
        srv.submit(ic, nsteps=0)
    assert e.value.code == -1
    big = I.uniform(128, 128, 64)
    with pytest.raises(M.MHDError) as e:
        srv.submit(big, nsteps=10)
    assert e.value.code == -7  # MHD_ECAPACITY: needs more than the whole budget
    rc, _ = srv.poll(12345)
    assert rc == -6  # MHD_ENOTFOUND
    srv.close()
