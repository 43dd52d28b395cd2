"""Checkpoint / resume and failure detection through the C-ABI (no GPU fault is involved: a
non-physical value is reported by the kernels' checks as MHD_ENONPHYS)."""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resume_is_bitwise(M, precision):
    ic = I.turbulence(8, mach=3.0, seed=61, shape=(12, 10, 14))
    straight = M.from_ic(ic, precision=precision)
    for _ in range(9):
        straight.step(0.4)
    first = M.from_ic(ic, precision=precision)
    for _ in range(4):
        first.step(0.4)
    st, full = first.get_state(), first.get_full()
    resumed = M.Sim(14, 10, 12, ic["gamma"], ic["dx"], precision=precision, chem=1)
    resumed.set_state(st["rho"], st["mom"], st["E"], st["B"], st["rho_h2"])
    resumed.set_full(full["eint"], full["bface"])  # exact rho eps and face fields
    for _ in range(5):
        resumed.step(0.4)
    a, b = straight.get_state(), resumed.get_state()
    for k in ["rho", "E", "mom", "B", "rho_h2"]:
        assert np.array_equal(a[k], b[k]), k


def test_nan_input_is_reported_not_faulted(M):
    ic = I.turbulence(8, mach=2.0, seed=62, shape=(8, 8, 8))
    ic["rho"][3, 4, 5] = np.nan
    s = M.from_ic(ic)
    with pytest.raises(M.MHDError) as e:
        s.step(0.4)
    assert e.value.code in (-4, -1)  # MHD_ENONPHYS, or MHD_EINVAL when tau itself is not finite
    assert s.diagnostics()["error_flags"] != 0
    # the context stays usable: a fresh simulation runs normally afterwards
    ok = M.from_ic(I.turbulence(8, mach=2.0, seed=63, shape=(8, 8, 8)))
    assert ok.step(0.4) > 0


def test_bad_arguments_are_rejected(M):
    with pytest.raises(M.MHDError):
        M.Sim(0, 4, 4, 1.4, 0.1)
    s = M.Sim(4, 4, 4, 1.4, 0.1)
    with pytest.raises(M.MHDError):
        s.step(0.4)  # no state loaded
    with pytest.raises(M.MHDError):
        s.set_option("precision", 7)


def test_enqueue_only_step_reports_an_earlier_flagged_step(M):
    """mhd_step with dt = NULL does not synchronise, but once a flagged step has finished on the
    device the next such call returns the error (host-mapped copy of the step's flags)."""
    import torch
    ic = I.turbulence(8, mach=2.0, seed=64, shape=(8, 8, 8))
    ic["rho"][2, 3, 4] = np.nan
    s = M.from_ic(ic)
    st = torch.cuda.Stream()
    s.set_stream(st.cuda_stream)
    s.step(0.4, sync=False)  # nothing has run yet when it is enqueued
    st.synchronize()
    with pytest.raises(M.MHDError) as e:
        s.step(0.4, sync=False)
    assert e.value.code in (-4, -1)
    ok = M.from_ic(I.turbulence(8, mach=2.0, seed=65, shape=(8, 8, 8)))
    ok.set_stream(st.cuda_stream)
    for _ in range(3):
        ok.step(0.4, sync=False)
    st.synchronize()
    ok.step(0.4, sync=False)  # a healthy sim keeps stepping
    ok.sync()


@pytest.mark.parametrize("precision", [0, 1])
def test_page_locked_host_buffers_equal_pageable(M, precision):
    """set_state and get_state with page-locked host arrays (read and written in place by the
    kernels) give the same bits as with pageable arrays (copied through the staging buffer)."""
    import torch
    ic = I.turbulence(8, mach=3.0, seed=66, shape=(10, 12, 14))
    a = M.from_ic(ic, precision=precision)
    b = M.Sim(14, 12, 10, ic["gamma"], ic["dx"], precision=precision, chem=1)
    pinned = {k: torch.from_numpy(np.ascontiguousarray(ic[k])).pin_memory()
              for k in ["rho", "mom", "E", "B", "rho_h2"]}
    b.set_state(*[pinned[k].numpy() for k in ["rho", "mom", "E", "B", "rho_h2"]])
    for s in (a, b):
        s.step(0.4)
    out = {k: torch.empty(tuple(v.shape), dtype=torch.float64).pin_memory() for k, v in pinned.items()}
    got = b.get_state(out={k: v.numpy() for k, v in out.items()})
    want = a.get_state()
    for k in ["rho", "mom", "E", "B", "rho_h2"]:
        assert np.array_equal(np.asarray(got[k]), want[k]), k


def test_per_step_log(M, tmp_path):
    """log_steps writes one JSON line per step with t, tau, the FP64 sums, max |div b| h, the
    velocity-branch count and the error flags; mass is conserved to rounding along the log."""
    import json
    ic = I.turbulence(8, mach=2.0, seed=67, shape=(8, 10, 12))
    s = M.from_ic(ic)
    path = tmp_path / "steps.jsonl"
    M.log_steps(s, 0.4, 3, str(path))
    recs = [json.loads(x) for x in path.read_text().splitlines()]
    assert [r["step"] for r in recs] == [1, 2, 3]
    assert all(r["tau"] > 0 and r["error_flags"] == 0 for r in recs)
    assert recs[0]["t"] < recs[1]["t"] < recs[2]["t"]
    assert abs(recs[2]["rho"] - recs[0]["rho"]) <= 1e-12 * recs[0]["rho"]
