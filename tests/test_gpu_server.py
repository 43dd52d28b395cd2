"""Serving: requests of different sizes and precisions arrive while others run; they are admitted
by HBM budget and stepped together (continuous batching).  Every result equals the same request
run alone, bit for bit."""
import time

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


REQS = [((16, 16, 16), 1, 7, 0.0), ((24, 20, 12), 1, 12, 0.0), ((8, 9, 10), 0, 5, 0.05),
        ((32, 16, 16), 1, 9, 0.1), ((12, 12, 12), 0, 8, 0.1), ((20, 20, 20), 1, 6, 0.2),
        ((16, 8, 24), 1, 11, 0.25)]


def request_ic(k):
    shape, prec, steps, delay = REQS[k]
    return I.turbulence(8, mach=2.0 + k, beta=0.5 + 0.2 * k, seed=100 + k, shape=shape)


def solo(M, k):
    shape, prec, steps, delay = REQS[k]
    s = M.from_ic(request_ic(k), precision=prec)
    for _ in range(steps):
        s.step(0.4, sync=False)
    s.sync()
    return s.get_state()


@pytest.mark.parametrize("policy", ["fifo", "smallest_work"])
def test_served_results_equal_solo_runs(M, policy):
    budget = sum(M.bytes_needed(*s[::-1], p, 1) for s, p, _, _ in REQS[:3])  # ~3 at a time
    srv = M.Server(budget, max_active=3)
    srv.set_policy(policy)
    ids = []
    t0 = time.time()
    for k, (shape, prec, steps, delay) in enumerate(REQS):
        while time.time() - t0 < delay:
            time.sleep(0.005)
        ids.append(srv.submit(request_ic(k), nsteps=steps, precision=prec))
    srv.drain(300)
    stats = srv.stats()
    assert stats["peak_bytes"] <= budget and stats["peak_active"] <= 3
    for k, rid in enumerate(ids):
        rc, res = srv.poll(rid)
        assert rc == 0, (k, rc)
        assert res["steps_done"] == REQS[k][2]
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]
        got = srv.fetch(rid, REQS[k][0])
        want = solo(M, k)
        for f in ["rho", "E", "mom", "B", "rho_h2"]:
            assert np.array_equal(got[f], want[f]), (k, f)
    srv.close()


def test_failed_device_allocation_and_running_cancel(M):
    """A request whose device memory cannot be had when it is admitted ends with MHD_ENOMEM and
    gives its budget back, and the server carries on: here the GPU's memory is first taken by the
    test (about 1.5 GB left), and a 192^3 request (2.2 GB) is admitted against a budget that would
    allow it.  Then a long request is cancelled while it runs: it ends with MHD_ECANCELED at the
    end of a batched step, and a request behind it completes."""
    import torch
    srv = M.Server(1 << 40, 8)
    free, _ = torch.cuda.mem_get_info()
    filler = torch.empty(max(free - (3 << 29), 1), dtype=torch.uint8, device="cuda")
    rid = srv.submit(I.turbulence(8, mach=2.0, seed=3, shape=(192, 192, 192)), nsteps=2)
    srv.drain(120)
    rc, res = srv.poll(rid)
    assert rc == -2, rc  # MHD_ENOMEM
    del filler
    torch.cuda.empty_cache()
    long_id = srv.submit(request_ic(0), nsteps=100000)
    t0 = time.time()
    while srv.poll(long_id)[1]["steps_done"] < 3 and time.time() - t0 < 60:
        time.sleep(0.01)
    srv.cancel(long_id)
    after = srv.submit(request_ic(1), nsteps=3)
    srv.drain(120)
    rc, res = srv.poll(long_id)
    assert rc == -8 and 3 <= res["steps_done"] < 100000
    assert srv.poll(after)[0] == 0
    srv.close()
