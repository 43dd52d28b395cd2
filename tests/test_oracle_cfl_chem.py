"""Pins of the CFL rule (Sec. 2.3), the H/H2 chemistry (Sec. 2.7, App. D) and gamma_eff (Sec. 4.3).

Checked against: the identity c_f + c_s = sqrt(c^2 + b^2 + 2 c c_a) (not the form the oracle
uses), hand-reduced App. D rates (tests/golden/app_d_rates.txt), the exact solution of
dn/dt = C - D n with frozen rates, and the limits of the backward-Euler formula."""
import os

import numpy as np
import pytest

from paper_1608_08748_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden", "app_d_rates.txt")


def cfl_closed_form(rho, v, B, p, gam):
    c = np.sqrt(gam * p / rho)
    b = np.sqrt(np.dot(B, B) / rho)
    best = 0.0
    for d in range(3):
        ca = abs(B[d]) / np.sqrt(rho)
        best = max(best, np.linalg.norm(v) + b + c + ca + np.sqrt(c * c + b * b + 2 * c * ca))
    return best


@pytest.mark.parametrize("state", [
    (1.0, [0, 0, 0], [0.75, 1.0, 0.0], 1.0, 2.0),        # Brio-Wu left
    (0.125, [0, 0, 0], [0.75, -1.0, 0.0], 0.1, 2.0),     # Brio-Wu right
    (0.18405, [3.8964, 0.5361, 2.4866], [4.0, 2.394, 1.197], 0.3541, 1.4),  # Sec. 3.1 left
    (1.0, [0.3, -2, 1], [0, 0, 0], 0.6, 5 / 3),
])
def test_cfl_denominator_closed_form(oracle_mod, state):
    rho, v, B, p, g = state
    assert oracle_mod.cfl_denominator(rho, v, B, p, g) == pytest.approx(
        cfl_closed_form(rho, np.array(v, float), np.array(B, float), p, g), rel=1e-13)


def test_tau_of_uniform_state(oracle_mod):
    ic = I.uniform(6, 5, 4, rho=1.3, p=0.7, v=(0.3, -0.2, 0.1), B=(0.5, 0.4, -0.3), dx=0.1)
    s = oracle_mod.run(ic)
    D = cfl_closed_form(1.3, np.array([0.3, -0.2, 0.1]), np.array([0.5, 0.4, -0.3]), 0.7, 5 / 3)
    assert s.tau(0.4) == pytest.approx(0.4 * 0.1 / D, rel=1e-13)


def test_gamma_eff_limits(oracle_mod):
    assert oracle_mod.gamma_eff(3.0, 0.0) == pytest.approx(5 / 3, rel=1e-15)
    assert oracle_mod.gamma_eff(3.0, 3.0) == pytest.approx(7 / 5, rel=1e-15)
    # n_H = 1, n_H2 = 1: (5 + 7) / (3 + 5)
    assert oracle_mod.gamma_eff(3.0, 2.0) == pytest.approx(12 / 8, rel=1e-15)


def _golden():
    rows = []
    for line in open(GOLD):
        line = line.split("#")[0].strip()
        if line:
            name, T, nH, nH2, val, tol = line.split()
            rows.append((name, float(T), float(nH), float(nH2), float(val), float(tol)))
    return rows


@pytest.mark.parametrize("row", _golden())
def test_app_d_rates_golden(oracle_mod, row):
    name, T, nH, nH2, val, tol = row
    s = oracle_mod.Sim(4, 4, 4, 5 / 3, 1.0, chem=1)
    r = s.chem_rates(T, nH, nH2)
    assert r[name] == pytest.approx(val, rel=tol, abs=0)




def test_temperature_of_the_turbulence_gas(oracle_mod):
    """p = n k_B T with n = 100 cm^-3 and T = 100 K (the initial state of the turbulence box)."""
    ic = I.turbulence(8, mach=1.0)
    s = oracle_mod.Sim(8, 8, 8, 5 / 3, ic["dx"], chem=1)
    p0 = 100.0 * I.KB_CGS * 100.0 / I.P_UNIT_CGS
    out = s.chem_cell(100.0, p0 / (5 / 3 - 1), 0.0, 1e-3)
    assert out["T"] == pytest.approx(100.0, rel=1e-12)


def test_chemistry_update_limits_and_exact_solution(oracle_mod):
    s = oracle_mod.Sim(4, 4, 4, 5 / 3, 2.0, chem=1)
    rho, rh2 = 100.0, 20.0
    eint = 300.0
    T0 = 3.0856775814913673e18 / 1e5  # code time unit in s
    base = s.chem_cell(rho, eint, rh2, 1e-30)
    C, D = base["C"], base["D"]
    n0 = 0.5 * rh2
    # tau -> 0: the update approaches explicit Euler, dn = tau (C - D n)
    for tau in [1e-6, 1e-7]:
        out = s.chem_cell(rho, eint, rh2, tau)
        dn = 0.5 * out["rho_h2"] - n0
        assert dn == pytest.approx(tau * T0 * (C - D * n0), rel=1e-3 * (1 + 1e6 * tau), abs=0)
    # tau -> infinity: the fixed point C / D
    out = s.chem_cell(rho, eint, rh2, 1e12)
    assert 0.5 * out["rho_h2"] == pytest.approx(min(C / D, 0.5 * rho), rel=1e-9, abs=0)
    # frozen-rate exact solution n(t) = C/D + (n0 - C/D) exp(-D t); the local error of one
    # backward-Euler step is O(tau^2)
    errs = []
    for tau in [1e-4, 5e-5, 2.5e-5]:
        ts = tau * T0
        exact = C / D + (n0 - C / D) * np.exp(-D * ts)
        got = 0.5 * s.chem_cell(rho, eint, rh2, tau)["rho_h2"]
        errs.append(abs(got - exact))
    assert errs[0] > errs[1] > errs[2]
    assert 3.2 < errs[0] / errs[1] < 4.8 and 3.2 < errs[1] / errs[2] < 4.8


def test_chemistry_conserves_nuclei_and_stays_in_range(oracle_mod):
    """n_H + 2 n_H2 = rho is untouched (rho is not updated) and 0 <= rho_H2 <= rho."""
    s = oracle_mod.Sim(4, 4, 4, 5 / 3, 2.0, chem=1)
    rng = np.random.default_rng(11)
    for _ in range(200):
        rho = 10 ** rng.uniform(0, 3)
        rh2 = rho * rng.uniform(0, 1)
        eint = rho * 10 ** rng.uniform(-1, 3)
        tau = 10 ** rng.uniform(-4, 1)
        out = s.chem_cell(rho, eint, rh2, tau)
        assert 0.0 <= out["rho_h2"] <= rho
        nH = rho - out["rho_h2"]
        assert nH + out["rho_h2"] == pytest.approx(rho, rel=1e-15)
