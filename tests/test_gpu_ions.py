"""GPU ionisation network (reactions 5-8 with H+ and e; App. D k5-k8, Gamma_5, Lambda_6-8; gamma_eff
with electrons) against the FP64 oracle: the chemistry stage alone, full FP64 steps with heating and
cooling (relative L1 <= 1e-10 per field, rho_H+ included; tau within 1e-11), FP32-bulk steps
(<= 1e-4), the set/get round trip, and the Lagrangian stage's exact transport of a power-of-two ion
fraction."""
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


def ionised_ic(n, mach, seed, T_K=100.0, heatcool=0):
    """Turbulence with 5 % of the hydrogen molecular and a random ion fraction 1e-4 .. 0.3 per cell."""
    ic = dict(I.turbulence(n, mach=mach, seed=seed, T_K=T_K))
    rng = np.random.default_rng(seed)
    ic["rho_h2"] = 0.05 * ic["rho"]
    ic["rho_hp"] = ic["rho"] * 10 ** rng.uniform(-4, np.log10(0.3), ic["rho"].shape)
    ic["options"] = dict(ic["options"], ions=1, heatcool=heatcool)
    return ic


def compare_ions(g, o, tol):
    a, b = g.get_ions(), o.get_ions()
    err = np.abs(a - b).sum() / max(np.abs(b).sum(), b.size * o.get_state()["rho"].mean() * 1e-6)
    assert err <= tol, err
    return err


@pytest.mark.parametrize("T_K", [100.0, 1.2e4])
def test_chemistry_stage_alone_matches_the_oracle(M, oracle_mod, T_K):
    from test_gpu_parity import compare
    ic = ionised_ic(16, 2.0, 41, T_K=T_K)
    g = M.from_ic(ic)
    o = oracle_mod.run(ic)
    for tau in (1e-3, 0.05):
        g.stage(3, tau)
        o.stage(3, tau)
    compare(g.get_state(), o.get_state(), tol=1e-12)
    err = compare_ions(g, o, 1e-12)
    print(f"ion chemistry stage at {T_K} K: rho_H+ rel L1 {err:.1e}")


def test_full_steps_fp64_match_the_oracle(M, oracle_mod):
    from test_gpu_parity import compare, run_pair
    ic = ionised_ic(24, 3.0, 42, T_K=8000.0, heatcool=1)
    g, o = run_pair(M, oracle_mod, ic, steps=10)
    errs = compare(g.get_state(), o.get_state())
    errs["rho_hp"] = compare_ions(g, o, 1e-10)
    print("ions + heating/cooling, 10 steps rel L1:", {k: f"{v:.1e}" for k, v in errs.items()})


def test_full_steps_fp32_within_tolerance(M, oracle_mod):
    from test_gpu_parity import compare
    ic = ionised_ic(24, 0.5, 43, T_K=8000.0, heatcool=1)
    g = M.from_ic(ic, precision=1)
    o = oracle_mod.run(ic)
    for _ in range(10):
        g.step(0.4, sync=False)
        o.step(0.4)
    g.sync()
    compare(g.get_state(), o.get_state(), tol=1e-4)
    compare_ions(g, o, 1e-4)


def test_set_get_round_trip_and_set_state_zeroes(M):
    ic = ionised_ic(12, 2.0, 44)
    g = M.from_ic(ic)
    assert np.array_equal(g.get_ions(), ic["rho_hp"])
    g.set_state(ic["rho"], ic["mom"], ic["E"], ic["B"], ic["rho_h2"])
    assert not g.get_ions().any()


@pytest.mark.parametrize("precision", [0, 1])
def test_lagrangian_stage_carries_an_exact_ion_fraction(M, precision):
    ic = ionised_ic(16, 3.0, 45)
    ic["rho_h2"] = 0.125 * ic["rho"]
    ic["rho_hp"] = 0.25 * ic["rho"]
    g = M.from_ic(ic, precision=precision)
    tau = 0.5 * g.diagnostics()["tau_next"] * 0.4
    g.stage(2, tau)
    st = g.get_state()
    assert np.array_equal(g.get_ions(), 0.25 * st["rho"])
    assert np.array_equal(st["rho_h2"], 0.125 * st["rho"])
