"""FP32-bulk path (reconstruction, fluxes, updates and state in float; CFL reduction, chemistry and
diagnostics sums in FP64) against the FP64 oracle.

Tolerances: relative L1 <= 1e-4 per field on smooth flows; on the Brio-Wu tube (config 1) the
positions of the compound wave, the contact and the slow shock within one cell."""
import numpy as np
import pytest

from paper_1608_08748_gb300 import inputs as I
from test_gpu_parity import compare

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


def run32(M, ic, steps=None, t_end=None, cfl=0.4):
    g = M.from_ic(ic, precision=1)
    if t_end is not None:
        g.advance(cfl, t_end)
    else:
        for _ in range(steps):
            g.step(cfl)
    return g


def test_fp32_smooth_turbulence(M, oracle_mod):
    """Subsonic (Mach 0.5) smooth turbulence with chemistry, 24^3, 20 steps."""
    ic = I.turbulence(24, mach=0.5, beta=1.0, seed=21)
    g = run32(M, ic, steps=20)
    o = oracle_mod.run(ic, steps=20)
    errs = compare(g.get_state(), o.get_state(), tol=1e-4)
    assert g.diagnostics()["t"] == pytest.approx(o.t, rel=1e-5)
    print("fp32 smooth turbulence rel L1:", {k: f"{v:.2e}" for k, v in errs.items()})


def test_fp32_linear_wave(M, oracle_mod):
    from test_oracle_physics import wave_ic
    ic, speed = wave_ic(64, "fast", amp=1e-3)
    t_end = 1.0 / abs(speed)
    g = run32(M, ic, t_end=t_end)
    o = oracle_mod.run(ic, t_end=t_end)
    compare(g.get_state(), o.get_state(), tol=1e-4)


def test_fp32_brio_wu_wave_positions(M, oracle_mod):
    ic = I.brio_wu(128, 4, 4)
    g = run32(M, ic, t_end=0.1)
    o = oracle_mod.run(ic, t_end=0.1)
    rg, ro = g.get_state()["rho"][0, 0], o.get_state()["rho"][0, 0]

    def position(r, lo, hi):
        # the |d rho| - weighted centroid of the interfaces lo .. hi - 1: the largest single jump is
        # ill-posed at the slow shock, where the oracle's two largest jumps differ by 5 % and the
        # post-shock state oscillates (beta = 0.13)
        j = np.abs(np.diff(r))[lo:hi]
        return lo + float(np.sum(np.arange(hi - lo) * j) / np.sum(j))

    for lo, hi in [(55, 66), (66, 76), (76, 92)]:  # compound wave, contact, slow shock at t = 0.1
        pg, po = position(rg, lo, hi), position(ro, lo, hi)
        assert abs(pg - po) <= 1.0, (lo, hi, pg, po, np.round(rg[lo:hi + 1], 4), np.round(ro[lo:hi + 1], 4))


def test_fp32_accepts_float32_inputs(M):
    ic = I.turbulence(8, mach=1.0, seed=3, shape=(6, 8, 10))
    g = M.Sim(10, 8, 6, ic["gamma"], ic["dx"], precision=1, chem=1)
    f32 = {k: None if v is None else np.asarray(v, np.float32) for k, v in ic.items()
           if k in ("rho", "mom", "E", "B", "rho_h2")}
    g.set_state(f32["rho"], f32["mom"], f32["E"], f32["B"], f32["rho_h2"], dtype=1)
    st = g.get_state(dtype=1)
    assert np.array_equal(st["rho"], f32["rho"])
    g.step(0.4)
    assert np.isfinite(g.get_state()["E"]).all()
