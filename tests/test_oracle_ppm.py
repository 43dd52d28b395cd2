"""Pins of the oracle's local parabola (Sec. 2.1) and domain-of-dependence averages (Sec. 2.4).

Checked against: the parabola's own definition (endpoints, cell average), exactness on linear
data, mirror symmetry, monotonicity bounds, and numerical quadrature of the parabola."""
import numpy as np
import pytest

_GX, _GW = np.polynomial.legendre.leggauss(4)  # exact for the quadratic parabola


def quad(f, a, b, **_):
    x = 0.5 * (b - a) * _GX + 0.5 * (a + b)
    return (0.5 * (b - a) * sum(w * f(xx) for w, xx in zip(_GW, x)),)


def parabola(P, xi):
    """q(xi) = q^L + xi (Delta q + q6 (1 - xi)) on xi in [0, 1] (Sec. 2.1, with Delta q = q^R - q^L)."""
    qL, qR, dq, q6 = P
    return qL + xi * (dq + q6 * (1.0 - xi))


def test_constant_stays_constant(oracle_mod):
    for c in [0.0, 1.0, -3.5, 1e-7]:
        P = oracle_mod.ppm([c] * 5)
        assert P[0] == c and P[1] == c and P[2] == 0.0 and P[3] == 0.0


def test_linear_data_exact_edges(oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(50):
        a, b = rng.normal(size=2) * [1.0, 0.3]
        a += 10.0  # keep the 1/100 contact-detector gate inactive
        q = a + b * np.arange(-2, 3)
        qL, qR, dq, q6 = oracle_mod.ppm(q)
        assert qL == pytest.approx(a - 0.5 * b, rel=1e-14, abs=1e-14)
        assert qR == pytest.approx(a + 0.5 * b, rel=1e-14, abs=1e-14)
        assert abs(q6) < 1e-13


def test_linear_data_as_written_step4_flattens(oracle_mod):
    """With the weights of Step 4 as printed, smooth data gets q +- delta_m q / 4 (half slope)."""
    q = 10.0 + 0.2 * np.arange(-2, 3)
    qL, qR, _, _ = oracle_mod.ppm(q, step4_as_written=True)
    assert qL == pytest.approx(10.0 - 0.05, rel=1e-14)
    assert qR == pytest.approx(10.0 + 0.05, rel=1e-14)


def test_cell_average_and_endpoints(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(500):
        q = rng.normal(size=5) * rng.choice([1e-3, 1.0, 10.0]) + rng.normal()
        P = oracle_mod.ppm(q)
        avg = quad(lambda x: parabola(P, x), 0.0, 1.0, epsabs=0, epsrel=1e-13)[0]
        assert avg == pytest.approx(q[2], rel=1e-12, abs=1e-12 * np.abs(q).max())
        assert parabola(P, 0.0) == pytest.approx(P[0], abs=1e-14 * np.abs(q).max())
        assert parabola(P, 1.0) == pytest.approx(P[1], abs=1e-13 * np.abs(q).max())


def test_monotone_and_bounded(oracle_mod):
    """Edge values lie between the neighbouring cell values and the parabola has no interior
    extremum (|q6| <= |Delta q|), for random data (Steps 1-5)."""
    rng = np.random.default_rng(2)
    for _ in range(2000):
        q = rng.normal(size=5)
        qL, qR, dq, q6 = oracle_mod.ppm(q)
        eps = 1e-12
        assert min(q[1], q[2]) - eps <= qL <= max(q[1], q[2]) + eps
        assert min(q[2], q[3]) - eps <= qR <= max(q[2], q[3]) + eps
        assert abs(q6) <= abs(dq) + eps


def test_mirror_symmetry(oracle_mod):
    rng = np.random.default_rng(3)
    for _ in range(500):
        q = rng.normal(size=5)
        a = oracle_mod.ppm(q)
        b = oracle_mod.ppm(q[::-1])
        assert a[0] == pytest.approx(b[1], abs=1e-14)
        assert a[1] == pytest.approx(b[0], abs=1e-14)
        assert a[3] == pytest.approx(b[3], abs=1e-13)


def test_extremum_is_flattened(oracle_mod):
    qL, qR, dq, q6 = oracle_mod.ppm([0.0, 1.0, 3.0, 1.0, 0.0])
    assert qL == 3.0 and qR == 3.0 and dq == 0.0 and q6 == 0.0


def test_domain_of_dependence_averages_match_quadrature(oracle_mod):
    """Sec. 2.4 closed forms q(-nu t) and q(nu t) equal the mean of the parabola over the last /
    first fraction y of the cell."""
    rng = np.random.default_rng(4)
    for _ in range(300):
        P = oracle_mod.ppm(rng.normal(size=5))
        for y in [1e-3, 0.1, 0.37, 0.8, 1.0]:
            right = quad(lambda x: parabola(P, x), 1.0 - y, 1.0, epsrel=1e-13)[0] / y
            left = quad(lambda x: parabola(P, x), 0.0, y, epsrel=1e-13)[0] / y
            assert oracle_mod.avg(P, y, True) == pytest.approx(right, abs=1e-13)
            assert oracle_mod.avg(P, y, False) == pytest.approx(left, abs=1e-13)
        assert oracle_mod.avg(P, 0.0, True) == P[1]
        assert oracle_mod.avg(P, 0.0, False) == P[0]
