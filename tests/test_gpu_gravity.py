"""GPU self-gravity (Sec. 2.10 Poisson solution by cuFFT; gravity terms of the Eulerian stage)
against the FP64 oracle: the potential itself, the Eulerian stage, full FP64 steps (relative L1
<= 1e-10 per field, tau within 1e-11) and FP32-bulk steps (<= 1e-4); and the refusals (outflow
boundaries, batching)."""
import numpy as np
import pytest

from paper_1608_08748_gb300 import inputs as I

pytestmark = pytest.mark.gpu
G = 6.6743e-8 * 1.6735575e-24 * (3.0856775814913673e18 / 1e5) ** 2  # G in pc, km/s, m_H cm^-3


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_08748_gb300 import build as B
    B.build()
    import paper_1608_08748_gb300 as M
    return M


def gravity_ic(n, mach, seed, shape=None):
    """The turbulence set-up with the density perturbed by up to 30 % (same velocity, pressure and
    field), self-gravity on."""
    ic = I.turbulence(n, mach=mach, seed=seed, shape=shape)
    rng = np.random.default_rng(seed)
    v = ic["mom"] / ic["rho"][None]
    kin = 0.5 * ic["rho"] * (v ** 2).sum(0)
    p = (ic["gamma"] - 1.0) * (ic["E"] - kin - 0.5 * (ic["B"] ** 2).sum(0))
    rho = ic["rho"] * (1.0 + 0.3 * rng.random(ic["rho"].shape))
    out = I.conserved(rho, v, p, ic["B"], ic["gamma"], np.zeros_like(rho))
    out.update(gamma=ic["gamma"], dx=ic["dx"], options=dict(ic["options"], grav_g=G))
    return out


@pytest.mark.parametrize("shape", [(16, 16, 16), (8, 10, 12), (5, 7, 9)])
@pytest.mark.parametrize("precision", [0, 1])
def test_potential_matches_the_oracle(M, oracle_mod, shape, precision):
    ic = gravity_ic(8, 2.0, 41, shape=shape)
    g = M.from_ic(ic, precision=precision)
    o = oracle_mod.run(ic)
    pg, po = g.potential(), o.potential()
    tol = 1e-12 if precision == 0 else 1e-5
    assert np.abs(pg - po).max() <= tol * np.abs(po).max()


def test_eulerian_stage_with_gravity_matches_the_oracle(M, oracle_mod):
    from test_gpu_parity import compare
    ic = gravity_ic(16, 3.0, 42)
    g = M.from_ic(ic)
    o = oracle_mod.run(ic)
    g.stage(1, 0.02)
    o.stage(1, 0.02)
    compare(g.get_state(), o.get_state(), tol=1e-12)


def test_full_steps_fp64_match_the_oracle(M, oracle_mod):
    from test_gpu_parity import compare, run_pair
    ic = gravity_ic(24, 3.0, 43)
    g, o = run_pair(M, oracle_mod, ic, steps=10)
    errs = compare(g.get_state(), o.get_state())
    print("self-gravity 10 steps rel L1:", {k: f"{v:.1e}" for k, v in errs.items()})


def test_full_steps_fp32_within_tolerance(M, oracle_mod):
    from test_gpu_parity import compare
    ic = gravity_ic(24, 0.5, 44)
    g = M.from_ic(ic, precision=1)
    o = oracle_mod.run(ic)
    for _ in range(10):
        g.step(0.4, sync=False)
        o.step(0.4)
    g.sync()
    compare(g.get_state(), o.get_state(), tol=1e-4)


def test_gravity_refusals(M):
    ic = gravity_ic(8, 1.0, 45)
    out = dict(ic)
    out["options"] = dict(ic["options"], bc_x=1)
    s = M.from_ic(out)
    with pytest.raises(M.MHDError):
        s.step(0.4)
    a = M.from_ic(ic)
    with pytest.raises(M.MHDError):
        M.Batch([a])
