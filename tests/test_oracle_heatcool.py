"""Pins of the oracle's heating/cooling stage (Sec. 2.8; App. D Gamma_1, Lambda_2, Lambda_3, Gamma_4).

The physics of the App. D fits is parity unpinned beyond what the paper itself fixes. Pinned here:
- the printed two-branch fits of Lambda_2 join continuously at their switch temperatures (1087 K
  for L_H, 4031 K for L_L), as the paper's fits do;
- the limits of the L_H / (1 + L_H / L_L) form: n_H2 L_H at high density, n_H2 L_L at low density;
- the critical-density limits of Gamma_1: 7.2e-12 erg per formed molecule (the formation rate C of
  the chemistry) far above n_cr, and that times n / n_cr far below;
- Gamma_4 = 6.4e-13 erg per photodissociation (k4 n_H2);
- no H2: no Lambda_2, Lambda_3 or Gamma_4;
- the Euler step of Sec. 2.8: rho E and rho eps change by the same amount, linear in tau, and the
  change never removes more than half of rho eps;
- in a box: the stage changes only rho E and rho eps, and the total change of rho E is the sum of
  the per-cell changes."""
import numpy as np
import pytest

from paper_1608_08748_gb300 import inputs as I

KB, MH = 1.380649e-16, 1.6735575e-24
P0 = MH * 1e10


def eint_of(T, rho, rh2):
    """rho eps (code units) with temperature T: T = (gamma_eff - 1) rho eps P0 / ((n_H + n_H2) k_B)."""
    nH, nH2 = rho - rh2, 0.5 * rh2
    g = (5 * nH + 7 * nH2) / (3 * nH + 5 * nH2)
    return T * (nH + nH2) * KB / ((g - 1.0) * P0)


@pytest.fixture(scope="module")
def sim(oracle_mod):
    return oracle_mod.Sim(4, 4, 4, 5.0 / 3.0, 2.0, chem=1, heatcool=1)


def terms(sim, T, rho, rh2, tau=1e-3):
    return sim.heatcool_cell(rho, eint_of(T, rho, rh2), rh2, tau)


@pytest.mark.parametrize("Tsw,rho", [(1087.0, 1e8), (4031.0, 1e-6)])
def test_lambda2_branches_join(sim, Tsw, rho):
    # high density: Lambda_2 -> n_H2 L_H (probes L_H at 1087 K); low density: -> n_H2 L_L (L_L at 4031 K)
    rh2 = 0.5 * rho
    lo = terms(sim, Tsw * (1 - 1e-9), rho, rh2)["L2"]
    hi = terms(sim, Tsw * (1 + 1e-9), rho, rh2)["L2"]
    assert abs(hi - lo) <= 0.02 * abs(lo), (lo, hi)


def test_lambda2_density_limits(sim):
    T = 2000.0
    hi = [terms(sim, T, r, 0.5 * r)["L2"] / (0.25 * r) for r in (1e10, 1e12)]
    assert hi[1] == pytest.approx(hi[0], rel=1e-3, abs=0)  # per-molecule rate saturates: n_H2 L_H
    lo = [terms(sim, T, r, 0.5 * r)["L2"] for r in (1e-8, 1e-7)]
    # n_H2 L_L with L_L ~ n^0.77: Lambda_2 ~ n^1.77
    assert lo[1] / lo[0] == pytest.approx(10 ** 1.77, rel=1e-3, abs=0)


def test_gamma1_critical_density_limits(oracle_mod, sim):
    T = 300.0
    for rho, rel in [(1e12, 1e-6)]:
        rh2 = 1e-3 * rho
        h = terms(sim, T, rho, rh2)
        C = sim.chem_cell(rho, eint_of(T, rho, rh2), rh2, 1e-3)["C"]
        assert h["G1"] == pytest.approx(7.2e-12 * C, rel=rel, abs=0)
    # far below n_cr: Gamma_1 ~ 7.2e-12 C n / n_cr, so Gamma_1 / C grows linearly with n
    a, b = [terms(sim, T, r, 1e-3 * r)["G1"] / sim.chem_cell(r, eint_of(T, r, 1e-3 * r), 1e-3 * r, 1e-3)["C"]
            for r in (1e-4, 1e-3)]
    assert b / a == pytest.approx(10.0, rel=1e-3, abs=0)


def test_gamma4_per_photodissociation(sim):
    rho, rh2, T = 50.0, 20.0, 500.0
    h = terms(sim, T, rho, rh2)
    k4 = sim.chem_rates(T, rho - rh2, 0.5 * rh2)["k4"]
    assert h["G4"] == pytest.approx(6.4e-13 * k4 * 0.5 * rh2, rel=1e-14, abs=0)


def test_no_molecules_no_molecular_cooling(sim):
    h = terms(sim, 800.0, 100.0, 0.0)
    assert h["L2"] == 0.0 and h["L3"] == 0.0 and h["G4"] == 0.0
    assert h["G1"] > 0.0 and h["net"] == h["G1"]


def test_euler_step_is_linear_and_limited(sim):
    rho, rh2, T = 100.0, 10.0, 60.0
    e = eint_of(T, rho, rh2)
    d1 = sim.heatcool_cell(rho, e, rh2, 1e-4)["delta"]
    d2 = sim.heatcool_cell(rho, e, rh2, 2e-4)["delta"]
    assert d2 == pytest.approx(2 * d1, rel=1e-12, abs=0)
    assert abs(d1) < 0.01 * e
    # a cooling time far below tau: the step removes exactly half of rho eps
    hot = eint_of(5000.0, rho, rh2)
    h = sim.heatcool_cell(rho, hot, rh2, 1.0)
    assert h["net"] < 0 and h["delta"] == -0.5 * hot


def test_box_stage_changes_only_the_energies(oracle_mod):
    ic = I.turbulence(8, mach=3.0, seed=9)
    ic["rho_h2"] = 0.02 * ic["rho"]
    ic["E"] = ic["E"] + 0.0
    s = oracle_mod.run(ic, heatcool=1)
    a = s.get_state()
    eps0 = None
    tau = 0.01
    # per-cell changes predicted from the unit entry
    rho, rh2 = a["rho"], a["rho_h2"]
    kin = 0.5 * (a["mom"] ** 2).sum(0) / rho
    mag = 0.5 * (a["B"] ** 2).sum(0)
    eint = a["E"] - kin - mag
    pred = np.array([s.heatcool_cell(r, e, h, tau)["delta"] for r, e, h in
                     zip(rho.ravel(), eint.ravel(), rh2.ravel())]).reshape(rho.shape)
    s.stage(5, tau)
    b = s.get_state()
    for k in ["rho", "mom", "B", "rho_h2"]:
        assert np.array_equal(a[k], b[k]), k
    assert np.allclose(b["E"] - a["E"], pred, rtol=1e-10, atol=1e-12 * np.abs(a["E"]).max())
    assert (b["E"] - a["E"]).sum() == pytest.approx(pred.sum(), rel=1e-10, abs=0)
