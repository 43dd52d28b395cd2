"""Pins of the oracle's self-gravity (Sec. 2.10 Poisson solution; gravity terms of the Sec. 2
momentum and energy equations, evaluated by central differences as Sec. 2.4 states).

Checked against:
- the real-space 27-point operator whose harmonic symbol Sec. 2.10 prints: with A the product of
  (1/6, 2/3, 1/6) averages along the three axes, (6 / h^2)(A Phi - Phi) = 4 pi G (rho - mean rho)
  to rounding (rolls in numpy, no Fourier transform);
- the continuum solution of the Poisson equation for one smooth mode, Phi = -4 pi G a / k^2 cos(k x),
  approached at second order in k h;
- the Eulerian stage of a nearly cold gas at rest (p = 1e-16, no field) whose density varies along
  one axis, where gravity is the only force to 1e-10: rho v = tau rho g and rho E rises by
  rho |g|^2 tau^2 / 2 (SSP-RK3 integrates the quadratic energy exactly), g = -grad Phi by central
  differences;
- a mutation-sensitive sign: gas falls towards the density peak."""
import numpy as np
import pytest

from paper_1608_08748_gb300 import inputs as I

G = 0.7


def A27(phi):
    out = phi
    for ax in range(3):
        out = (np.roll(out, 1, axis=ax) + 4.0 * out + np.roll(out, -1, axis=ax)) / 6.0
    return out


def gas(oracle_mod, rho, dx=0.5, p=1.0):
    nz, ny, nx = rho.shape
    v = np.zeros((3,) + rho.shape)
    B = np.zeros((3,) + rho.shape)
    ic = I.conserved(rho, v, np.full(rho.shape, p), B, 5.0 / 3.0)
    s = oracle_mod.Sim(nx, ny, nz, 5.0 / 3.0, dx, grav_g=G)
    s.set_state(ic["rho"], ic["mom"], ic["E"], ic["B"])
    return s, ic


@pytest.mark.parametrize("shape", [(8, 10, 12), (16, 16, 16), (5, 7, 9)])
def test_potential_satisfies_the_27_point_equation(oracle_mod, shape):
    rng = np.random.default_rng(11)
    rho = 1.0 + 0.3 * rng.random(shape)
    dx = 0.25
    s, _ = gas(oracle_mod, rho, dx)
    phi = s.potential()
    lhs = (6.0 / dx ** 2) * (A27(phi) - phi)
    rhs = 4 * np.pi * G * (rho - rho.mean())
    assert np.abs(lhs - rhs).max() <= 1e-11 * np.abs(rhs).max()
    assert abs(phi.mean()) <= 1e-12 * np.abs(phi).max()  # the mean mode is zero


def test_smooth_mode_converges_to_the_continuum_solution(oracle_mod):
    errs = []
    for n in (16, 32, 64):
        L = 1.0
        x = (np.arange(n) + 0.5) / n * L
        k = 2 * np.pi / L
        a = 0.1
        rho = np.broadcast_to(1.0 + a * np.cos(k * x), (4, 4, n)).copy()
        s, _ = gas(oracle_mod, rho, L / n)
        phi = s.potential()[0, 0]
        exact = -4 * np.pi * G * a / k ** 2 * np.cos(k * x)
        errs.append(np.abs(phi - exact).max() / np.abs(exact).max())
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05, abs=0)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05, abs=0)


def test_eulerian_stage_with_gravity_only(oracle_mod):
    # density varying along x only: gravity drives normal flow only, so no face sees a tangential
    # velocity jump, and the near-cold gas feels no pressure response
    rng = np.random.default_rng(12)
    n = 24
    dx = 0.5
    rho = np.broadcast_to(1.0 + 0.2 * rng.random(n), (4, 4, n)).copy()
    s, ic = gas(oracle_mod, rho, dx, p=1e-16)
    phi = s.potential()
    g = np.stack([-(np.roll(phi, -1, axis=2 - d) - np.roll(phi, 1, axis=2 - d)) / (2 * dx) for d in range(3)])
    assert np.abs(g[1:]).max() <= 1e-12 * np.abs(g[0]).max()
    tau = 0.01
    s.stage(1, tau)
    st = s.get_state()
    ref = tau * rho * g
    assert np.abs(st["mom"] - ref).max() <= 1e-8 * np.abs(ref).max()
    dE = st["E"] - ic["E"]
    refE = 0.5 * rho * (g ** 2).sum(0) * tau ** 2
    assert np.abs(dE - refE).max() <= 1e-8 * np.abs(refE).max()
    assert np.array_equal(st["rho"], ic["rho"])


def test_gas_falls_towards_the_density_peak(oracle_mod):
    n = 32
    x = (np.arange(n) + 0.5) / n
    rho = np.broadcast_to(1.0 + 0.5 * np.exp(-((x - 0.5) / 0.1) ** 2), (4, 4, n)).copy()
    s, _ = gas(oracle_mod, rho, 1.0 / n)
    s.stage(1, 0.01)
    mx = s.get_state()["mom"][0, 0, 0]
    assert (mx[: n // 2 - 2] > 0).all() and (mx[n // 2 + 2:] < 0).all()
