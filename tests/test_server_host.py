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


def test_pause_cancel_budget_and_drain_timeout(M):
    """Fault and control paths of the server that need no device work: with admission paused the
    queue holds, so drain gives up with MHD_ETIMEOUT; a cancelled waiting request ends with
    MHD_ECANCELED (a second cancel is refused, an unknown id is not found); shrinking the budget
    below a waiting request's need fails that request with MHD_ECAPACITY and leaves the others
    waiting; once the rest are cancelled, drain returns MHD_OK."""
    srv = M.Server(1 << 30, 4)
    srv.pause(True)
    ids = [srv.submit(I.uniform(8, 8, 8), nsteps=5) for _ in range(3)]
    big = srv.submit(I.uniform(16, 16, 16), nsteps=5)
    assert srv.drain_rc(0.05) == -5  # MHD_ETIMEOUT
    srv.cancel(ids[0])
    rc, res = srv.poll(ids[0])
    assert rc == -8 and res["status"] == -8  # MHD_ECANCELED
    with pytest.raises(M.MHDError) as e:
        srv.cancel(ids[0])
    assert e.value.code == -1  # already finished
    with pytest.raises(M.MHDError) as e:
        srv.cancel(987654)
    assert e.value.code == -6  # MHD_ENOTFOUND
    srv.set_budget(M.bytes_needed(8, 8, 8, 1, 0))  # the 8^3 requests still fit, the 16^3 one not
    assert srv.poll(big)[0] == -7  # MHD_ECAPACITY
    assert srv.poll(ids[1])[0] == 1 and srv.poll(ids[2])[0] == 1  # MHD_PENDING: still queued
    with pytest.raises(M.MHDError) as e:
        srv.set_budget(0)
    assert e.value.code == -1
    for rid in ids[1:]:
        srv.cancel(rid)
    assert srv.drain_rc(1.0) == 0
    with pytest.raises(M.MHDError) as e:
        srv.fetch(ids[1], (8, 8, 8))
    assert e.value.code == -8
    srv.close()
