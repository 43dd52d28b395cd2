"""The three directional sweeps of each stage run on side streams forked from the sim's stream. The
result must not depend on how the step is launched: a captured CUDA graph, direct launches, and
the per-class profiler (which runs the sweeps in order on one stream) all give the same state bit
for bit, in FP64 and FP32, for a box with every per-cell stage on and for a plain box."""
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


def ic_of(kind):
    ic = dict(I.turbulence(20, mach=3.0, seed=61, shape=(18, 20, 22), T_K=2000.0))
    if kind == "full":
        ic["rho_h2"] = 0.05 * ic["rho"]
        ic["rho_hp"] = 0.01 * ic["rho"]
        ic["options"] = dict(ic["options"], ions=1, heatcool=1)
    return ic


@pytest.mark.parametrize("kind", ["plain", "full"])
@pytest.mark.parametrize("precision", [0, 1])
def test_launch_modes_agree_bitwise(M, kind, precision):
    ic = ic_of(kind)
    graph = M.from_ic(ic, precision=precision, graph=1)
    direct = M.from_ic(ic, precision=precision, graph=0)
    prof = M.from_ic(ic, precision=precision)
    for _ in range(4):
        graph.step(0.4, sync=False)
        direct.step(0.4, sync=False)
    graph.sync()
    direct.sync()
    M.profile(prof, 0.4, 4)
    a, b, c = graph.get_state(), direct.get_state(), prof.get_state()
    for k in ["rho", "E", "mom", "B", "rho_h2"]:
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a[k], c[k]), k
    assert graph.diagnostics()["t"] == direct.diagnostics()["t"] == prof.diagnostics()["t"]
