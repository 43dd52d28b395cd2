"""Pins of the Eulerian eigensystem (Sec. 2.4, App. A) and characteristic Riemann solver.

Checked against: the matrix B of Sec. 2.4 (retyped here; the oracle never uses it) through
L R = I and R Omega L = B, numpy's eigenvalues of B, an independent linear Riemann solution built
from numpy's eigenvectors, the acoustic (B = 0) closed form, and the expanded solution of App. B."""
import numpy as np
import pytest


def Bmat(rho, p, gam, Bn, Bt1, Bt2):
    """Sec. 2.4: dq/dt + B dq/dx = 0 for q = (v_n, v_t1, v_t2, B_t1, B_t2, p)."""
    return np.array([
        [0, 0, 0, Bt1 / rho, Bt2 / rho, 1 / rho],
        [0, 0, 0, -Bn / rho, 0, 0],
        [0, 0, 0, 0, -Bn / rho, 0],
        [Bt1, -Bn, 0, 0, 0, 0],
        [Bt2, 0, -Bn, 0, 0, 0],
        [gam * p, 0, 0, 0, 0, 0]], dtype=float)


def random_states(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        rho = 10 ** rng.uniform(-2, 2)
        p = 10 ** rng.uniform(-2, 2)
        gam = rng.choice([5 / 3, 1.4, 2.0])
        B = rng.normal(size=3) * 10 ** rng.uniform(-1, 1)
        out.append((rho, p, gam, *B))
    return out


DEGENERATE = [
    (1.0, 1.0, 5 / 3, 1.0, 0.0, 0.0),          # B_perp = 0, c != c_a
    (1.0, 0.6, 5 / 3, 1.0, 0.0, 0.0),          # B_perp = 0, gamma p = B_n^2 (triple point)
    (1.0, 1.0, 5 / 3, 0.0, 0.7, -0.2),         # B_n = 0
    (1.0, 1.0, 1.4, 0.0, 0.0, 0.0),            # B = 0
    (2.0, 0.5, 2.0, -0.75, 1.0, 0.0),          # B_n < 0
]


@pytest.mark.parametrize("st,tol", [(st, 1e-11) for st in random_states(200, 7)] +
                         [(st, 1e-11) for st in DEGENERATE])
def test_eigen_identities(oracle_mod, st, tol):
    """Also at the degenerate states (B_perp = 0, B_n = 0, B = 0): the speeds are evaluated without
    cancellation, so alpha_s is exactly 0 where the printed formula gives sqrt(0)."""
    R, L, lam, info = oracle_mod.eigen(*st)
    assert np.abs(L @ R - np.eye(6)).max() < tol
    Bm = Bmat(*st)
    scale = np.abs(Bm).max()
    assert np.abs(R @ np.diag(lam) @ L - Bm).max() < tol * scale


@pytest.mark.parametrize("st", random_states(100, 8) + DEGENERATE[:3] + DEGENERATE[4:])
def test_eigenvalues_match_numpy(oracle_mod, st):
    _, _, lam, _ = oracle_mod.eigen(*st)
    ev = np.sort(np.linalg.eigvals(Bmat(*st)).real)
    assert np.allclose(np.sort(lam), ev, rtol=1e-7, atol=1e-7 * np.abs(ev).max())


def linear_riemann_numpy(st, qL, qR):
    """Exact solution at x = 0 of the linear Riemann problem dq/dt + B dq/dx = 0 with constant
    left/right states: right-moving waves carry the left state's characteristic amplitudes."""
    Bm = Bmat(*st)
    w, V = np.linalg.eig(Bm)
    w, V = w.real, V.real
    Vi = np.linalg.inv(V)
    s = np.where(w > 0, Vi @ qL, Vi @ qR)
    return V @ s


def flat_stencils(q):
    return np.repeat(np.asarray(q, float)[:, None], 5, axis=1)


@pytest.mark.parametrize("seed", range(40))
def test_flat_riemann_matches_numpy_linear_solution(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    rho, p, gam = 10 ** rng.uniform(-1, 1), 10 ** rng.uniform(-1, 1), 5 / 3
    Bn = rng.choice([-1, 1]) * 10 ** rng.uniform(-0.5, 0.5)
    Bt = rng.normal(size=2)
    # left/right cells share rho, p, gamma, B so the face average is this state exactly
    st = (rho, p, gam, Bn, *Bt)
    wl = wr = [rho, p, gam, Bt[0], Bt[1]]
    qL = np.array([*rng.normal(size=3), *(Bt + 0.1 * rng.normal(size=2)), p * (1 + 0.1 * rng.normal())])
    qR = np.array([*rng.normal(size=3), *(Bt + 0.1 * rng.normal(size=2)), p * (1 + 0.1 * rng.normal())])
    got = oracle_mod.face_solve(wl, wr, Bn, flat_stencils(qL), flat_stencils(qR), 0.3, edge=False)
    want = linear_riemann_numpy(st, qL, qR)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


@pytest.mark.parametrize("seed", range(20))
def test_acoustic_limit(oracle_mod, seed):
    """B = 0: P* = (pL+pR)/2 + rho c (vL - vR)/2, V* = (vL+vR)/2 + (pL - pR)/(2 rho c), and the
    transverse velocity is the mean of the two sides (zero-speed waves, one from each side)."""
    rng = np.random.default_rng(200 + seed)
    rho, p, gam = 10 ** rng.uniform(-1, 1), 10 ** rng.uniform(-1, 1), 1.4
    w = [rho, p, gam, 0.0, 0.0]
    qL = np.array([*rng.normal(size=3), 0.0, 0.0, p * 1.1])
    qR = np.array([*rng.normal(size=3), 0.0, 0.0, p * 0.9])
    got = oracle_mod.face_solve(w, w, 0.0, flat_stencils(qL), flat_stencils(qR), 0.2)
    c = np.sqrt(gam * p / rho)
    assert got[5] == pytest.approx(0.5 * (qL[5] + qR[5]) + 0.5 * rho * c * (qL[0] - qR[0]), rel=1e-12)
    assert got[0] == pytest.approx(0.5 * (qL[0] + qR[0]) + (qL[5] - qR[5]) / (2 * rho * c), rel=1e-12, abs=1e-12)
    assert got[1] == pytest.approx(0.5 * (qL[1] + qR[1]), rel=1e-12, abs=1e-12)
    assert got[2] == pytest.approx(0.5 * (qL[2] + qR[2]), rel=1e-12, abs=1e-12)


def appB_Vx_P(e, q):
    """App. B expanded V_x and P.  q[name](s) is the parabola average of variable `name` for the
    wave of speed s: s > 0 means +lambda tau (right cell), s < 0 means -lambda tau (left cell).
    The slow-wave cross terms are printed with the opposite sign of what the eigenvectors of
    App. A give (those satisfy L R = I and R Omega L = B and reproduce numpy's exact linear
    solution, both pinned above): in V_x the B_t terms alpha_f c_s alpha_s beta (b(c_s tau) -
    b(-c_s tau)), in P the v_t terms rho alpha_f alpha_s c_f beta sign (v(-c_s tau) - v(c_s tau)).
    Those four terms are written here in the App. A order; every other term is as printed."""
    c, cf, cs, af, as_, by, bz, sg = e["c"], e["cf"], e["cs"], e["af"], e["as"], e["by"], e["bz"], e["sg"]
    rho = e["rho"]
    sr = np.sqrt(rho)
    vx, vy, vz, Byq, Bzq, pq = (q[k] for k in ["vx", "vy", "vz", "by", "bz", "p"])
    Vx = (as_ ** 2 * cs ** 2 * (vx(cs) + vx(-cs)) / (2 * c ** 2)
          + af * cf * as_ * cs * by * sg * (vy(cs) + vy(-cs) - vy(cf) - vy(-cf)) / (2 * c ** 2)
          + af ** 2 * cf ** 2 * (vx(cf) + vx(-cf)) / (2 * c ** 2)
          + af * cf * as_ * cs * bz * sg * (vz(cs) + vz(-cs) - vz(cf) - vz(-cf)) / (2 * c ** 2)
          + af * cf * as_ * by * (Byq(-cf) - Byq(cf)) / (2 * c * sr)
          + af * cf * as_ * bz * (Bzq(-cf) - Bzq(cf)) / (2 * c * sr)
          + af ** 2 * cf * (pq(-cf) - pq(cf)) / (2 * rho * c ** 2)
          + af * cs * as_ * by * (Byq(cs) - Byq(-cs)) / (2 * c * sr)
          + af * cs * as_ * bz * (Bzq(cs) - Bzq(-cs)) / (2 * c * sr)
          + as_ ** 2 * cs * (pq(-cs) - pq(cs)) / (2 * rho * c ** 2))
    P = (rho * af ** 2 * cf * (vx(-cf) - vx(cf)) / 2
         + sr * af * as_ * by * c * (Byq(cf) + Byq(-cf) - Byq(cs) - Byq(-cs)) / 2
         + rho * as_ ** 2 * cs * (vx(-cs) - vx(cs)) / 2
         + sr * af * as_ * bz * c * (Bzq(cf) + Bzq(-cf) - Bzq(cs) - Bzq(-cs)) / 2
         + rho * af * as_ * cs * by * sg * (vy(cf) - vy(-cf)) / 2
         + rho * af * as_ * cf * by * sg * (vy(-cs) - vy(cs)) / 2
         + af ** 2 * (pq(cf) + pq(-cf)) / 2
         + rho * af * as_ * cs * bz * sg * (vz(cf) - vz(-cf)) / 2
         + rho * af * as_ * cf * bz * sg * (vz(-cs) - vz(cs)) / 2
         + as_ ** 2 * (pq(cs) + pq(-cs)) / 2)
    return Vx, P


@pytest.mark.parametrize("seed", range(30))
def test_appendix_B_expansion(oracle_mod, seed):
    rng = np.random.default_rng(300 + seed)
    rho, p, gam = 10 ** rng.uniform(-0.5, 0.5), 10 ** rng.uniform(-0.5, 0.5), 5 / 3
    Bn = rng.choice([-1, 1]) * 10 ** rng.uniform(-0.5, 0.5)
    Bt = rng.normal(size=2)
    w = [rho, p, gam, Bt[0], Bt[1]]
    base = np.array([0.0, 0.0, 0.0, Bt[0], Bt[1], p])
    stl = base[:, None] + 0.05 * rng.normal(size=(6, 5)) * np.maximum(np.abs(base), 1.0)[:, None]
    str_ = base[:, None] + 0.05 * rng.normal(size=(6, 5)) * np.maximum(np.abs(base), 1.0)[:, None]
    # the face average uses the cell centres, so make those equal on both sides
    stl[:, 2] = base
    str_[:, 2] = base
    tau_h = 0.15
    got = oracle_mod.face_solve(w, w, Bn, stl, str_, tau_h)
    _, _, _, e = oracle_mod.eigen(rho, p, gam, Bn, *Bt)
    e["rho"] = rho
    PL = [oracle_mod.ppm(stl[v]) for v in range(6)]
    PR = [oracle_mod.ppm(str_[v]) for v in range(6)]

    def fn(v):
        def f(s):
            y = abs(s) * tau_h
            return oracle_mod.avg(PR[v], y, False) if s > 0 else oracle_mod.avg(PL[v], y, True)
        return f
    q = dict(zip(["vx", "vy", "vz", "by", "bz", "p"], [fn(v) for v in range(6)]))
    Vx, P = appB_Vx_P(e, q)
    assert got[0] == pytest.approx(Vx, rel=1e-9, abs=1e-11)
    assert got[5] == pytest.approx(P, rel=1e-9, abs=1e-11)
