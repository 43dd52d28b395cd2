"""GPU heating/cooling stage (Sec. 2.8, App. D Gamma_1, Lambda_2, Lambda_3, Gamma_4) against the FP64
oracle: the stage alone, full FP64 steps (relative L1 <= 1e-10 per field, tau within 1e-11) and
FP32-bulk steps (<= 1e-4), on turbulence boxes with molecular hydrogen present."""
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


def molecular_ic(n, mach, seed, frac=0.05):
    ic = I.turbulence(n, mach=mach, seed=seed)
    ic["rho_h2"] = frac * ic["rho"]
    ic["options"] = dict(ic["options"], heatcool=1)
    return ic


def test_stage_alone_matches_the_oracle(M, oracle_mod):
    from test_gpu_parity import compare
    ic = molecular_ic(16, 4.0, 31)
    g = M.from_ic(ic)
    o = oracle_mod.run(ic)
    for tau in (0.01, 0.2):  # the second tau drives hot cells onto the rho eps / 2 limit
        g.stage(5, tau)
        o.stage(5, tau)
    errs = compare(g.get_state(), o.get_state(), tol=1e-12)
    print("heating/cooling stage rel L1:", {k: f"{v:.1e}" for k, v in errs.items()})


def test_full_steps_fp64_match_the_oracle(M, oracle_mod):
    from test_gpu_parity import compare, run_pair
    ic = molecular_ic(24, 3.0, 32)
    g, o = run_pair(M, oracle_mod, ic, steps=10)
    errs = compare(g.get_state(), o.get_state())
    print("heating/cooling 10 steps rel L1:", {k: f"{v:.1e}" for k, v in errs.items()})


def test_full_steps_fp32_within_tolerance(M, oracle_mod):
    from test_gpu_parity import compare
    ic = molecular_ic(24, 0.5, 33)
    g = M.from_ic(ic, precision=1)
    o = oracle_mod.run(ic)
    for _ in range(10):
        g.step(0.4, sync=False)
        o.step(0.4)
    g.sync()
    compare(g.get_state(), o.get_state(), tol=1e-4)


def test_stage_changes_the_energy_by_heating_minus_cooling(M, oracle_mod):
    ic = molecular_ic(16, 2.0, 34)
    g = M.from_ic(ic)
    e0 = g.diagnostics()["E"]
    g.stage(5, 0.05)
    d = g.get_state()
    e1 = g.diagnostics()["E"]
    o = oracle_mod.run(ic)
    a = o.get_state()
    kin = 0.5 * (a["mom"] ** 2).sum(0) / a["rho"]
    eint = a["E"] - kin - 0.5 * (a["B"] ** 2).sum(0)
    pred = sum(o.heatcool_cell(r, e, h, 0.05)["delta"] for r, e, h in
               zip(a["rho"].ravel(), eint.ravel(), a["rho_h2"].ravel()))
    assert e1 - e0 == pytest.approx(pred, rel=1e-9, abs=0)
    for k in ["rho", "mom", "B", "rho_h2"]:  # only rho E and rho eps change
        assert np.array_equal(d[k], ic[k]), k
