"""Pins of the Step 4 discontinuity detector of Sec. 2.1 (readings A2, A3, A4).

The detector is checked on discrete profiles whose second differences are known by hand, so that
eta and the weight hbar have closed forms that do not come from the oracle's own code:

  * the cubic q_j = a j - j^3 (j = -2..2, unit spacing) has undivided second differences
    D_j = -6 j, so D_{+1} = -6, D_{-1} = +6 (an inflection at j = 0) and q_{+1} - q_{-1} = 2a - 2;
    with A2 (delta_m^2 q = D / (3 h^2)) eta = -h^2 (delta^2 q_{+1} - delta^2 q_{-1}) /
    (q_{+1} - q_{-1}) = 12 / (3 (2a - 2)) = 2 / (a - 1);
  * adding b j^2 moves both second differences by 2b: for |b| > 3 they share a sign (no
    inflection) and A3 zeroes eta, for |b| <= 3 eta stays 2 / (a - 1);
  * adding a constant C leaves every difference alone but raises min(|q_{+1}|, |q_{-1}|) =
    C - a + 1: A3 zeroes eta once |q_{+1} - q_{-1}| = 2a - 2 <= (C - a + 1) / 100.

For a >= 10 Steps 1-3 of the cubic are also known by hand: the limited slopes are
delta_m q_0 = a - 1 and delta_m q_{+-1} = a - 4, so q^L = -a/2, q^R = a/2 (monotone, no Step 2
fix), and the flattened values of Step 4 are q^{L,+} = -(a - 1)/4, q^{R,+} = (a - 1)/4.  With the
weights of reading A4 the final edges are q^L = hbar q^{L,+} + (1 - hbar)(-a/2) and q^R = -q^L.
"""
import numpy as np
import pytest




def cubic(a, b=0.0, C=0.0):
    j = np.arange(-2, 3, dtype=np.float64)
    return C + a * j - j ** 3 + b * j ** 2


def hbar_of(eta):
    return min(max(20.0 * (eta - 0.05), 0.0), 1.0)


A_VALUES = [10.0, 12.0, 18.0, 21.0, 23.5, 27.0, 31.0, 36.0, 41.0, 45.0, 80.0]


@pytest.mark.parametrize("a", A_VALUES)
def test_eta_and_weight_closed_form_on_a_cubic(oracle_mod, a):
    """eta = 2 / (a - 1) and hbar = clamp(20 (eta - 1/20), 0, 1); the ramp runs from a = 41
    (eta = 1/20, hbar = 0) to a = 21 (eta = 1/10, hbar = 1)."""
    eta, hb = oracle_mod.step4(cubic(a))
    assert abs(eta - 2.0 / (a - 1.0)) <= 1e-15 * (1.0 + abs(eta))
    assert abs(hb - hbar_of(2.0 / (a - 1.0))) <= 1e-13


@pytest.mark.parametrize("a", [12.0, 27.0, 36.0])
def test_detector_invariances(oracle_mod, a):
    """eta is unchanged by q -> s q (any nonzero scale, either sign), by a small offset and by
    mirroring the stencil (j -> -j with q -> -q maps the cubic onto itself)."""
    ref = oracle_mod.step4(cubic(a))
    for s in [1e-9, -1.0, 3.7, 1e12]:
        got = oracle_mod.step4(s * cubic(a))
        assert abs(got[0] - ref[0]) <= 1e-14 * abs(ref[0]) and abs(got[1] - ref[1]) <= 1e-12
    got = oracle_mod.step4(-cubic(a)[::-1].copy())
    assert abs(got[0] - ref[0]) <= 1e-15 * abs(ref[0])
    got = oracle_mod.step4(cubic(a, C=1.0))
    assert abs(got[0] - ref[0]) <= 1e-13 * abs(ref[0])


@pytest.mark.parametrize("a", A_VALUES)
def test_parabola_edges_follow_the_weight(oracle_mod, a):
    """The Step 5 parabola of the cubic: q^L = hbar (-(a - 1)/4) + (1 - hbar)(-a/2), q^R = -q^L,
    Delta q = q^R - q^L, q^(6) = 6 (q_0 - (q^L + q^R)/2) = 0 (A1, A4)."""
    hb = hbar_of(2.0 / (a - 1.0))
    qL = hb * (-(a - 1.0) / 4.0) + (1.0 - hb) * (-a / 2.0)
    P = oracle_mod.ppm(cubic(a))
    assert abs(P[0] - qL) <= 1e-13 * a
    assert abs(P[1] + qL) <= 1e-13 * a
    assert abs(P[2] - (-2.0 * qL)) <= 1e-13 * a
    assert abs(P[3]) <= 1e-13 * a


def test_printed_weights_flatten_smooth_cells_and_keep_discontinuities(oracle_mod):
    """With the weights as printed (flag step4_as_written) the roles swap: hbar weighs the Step 3
    edges and 1 - hbar the flattened ones, so at a = 80 (hbar = 0) the edges are the flattened
    -+(a - 1)/4 and at a = 12 (hbar = 1) they are the Step 3 values -+a/2."""
    P = oracle_mod.ppm(cubic(80.0), step4_as_written=True)
    assert abs(P[0] + 79.0 / 4.0) <= 1e-12 and abs(P[1] - 79.0 / 4.0) <= 1e-12
    P = oracle_mod.ppm(cubic(12.0), step4_as_written=True)
    assert abs(P[0] + 6.0) <= 1e-12 and abs(P[1] - 6.0) <= 1e-12


@pytest.mark.parametrize("b,active", [(0.0, True), (2.9, True), (-2.9, True), (3.0, True), (-3.0, True),
                                      (3.1, False), (-3.1, False), (20.0, False)])
def test_no_inflection_zeroes_eta(oracle_mod, b, active):
    """A3, second condition: eta := 0 where D_{+1} D_{-1} > 0 (no inflection), here |b| > 3; at
    |b| = 3 one second difference is 0 and the strict test keeps eta."""
    a = 28.0
    eta, hb = oracle_mod.step4(cubic(a, b=b))
    if active:
        assert abs(eta - 2.0 / 27.0) <= 1e-14
        assert abs(hb - hbar_of(2.0 / 27.0)) <= 1e-12 and hb > 0.4
    else:
        assert eta == 0.0 and hb == 0.0


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("frac,active", [(0.5, True), (0.98, True), (1.02, False), (3.0, False)])
def test_small_jumps_zero_eta(oracle_mod, sign, frac, active):
    """A3, first condition: eta := 0 where |q_{+1} - q_{-1}| <= min(|q_{+1}|, |q_{-1}|) / 100.  For
    the cubic offset by C (C > a) that is C >= C* = 100 (2a - 2) + a - 1; the sign of the offset
    does not matter (absolute values)."""
    a = 28.0
    Cstar = 100.0 * (2.0 * a - 2.0) + a - 1.0
    q = cubic(a, C=frac * Cstar)
    if sign < 0:
        q = -q[::-1].copy()  # offset -C, the same cubic mirrored
    eta, hb = oracle_mod.step4(q)
    if active:
        assert abs(eta - 2.0 / (a - 1.0)) <= 1e-11
        assert hb > 0.4
    else:
        assert eta == 0.0 and hb == 0.0


def test_sampled_sine_closed_form(oracle_mod):
    """On samples of a sine, q_j = sin(phi + k h j), every second difference is D_j = -2 (1 - cos kh)
    q_j, so wherever q_{+1} and q_{-1} differ in sign (the stencil straddles a zero of the sine) eta
    = 2 (1 - cos kh) / 3 exactly, whatever the phase; where they share a sign D_{+1} D_{-1} > 0
    zeroes it.  The weight therefore stays 0 for waves of 17 or more cells (eta < 1/20) and turns
    on below (16 cells: eta = 0.0507)."""
    for cells in [6, 8, 12, 16, 17, 24, 64]:
        kh = 2.0 * np.pi / cells
        eta_x = 2.0 * (1.0 - np.cos(kh)) / 3.0
        for phase in np.linspace(0.0, 2.0 * np.pi, 41)[:-1]:
            q = np.sin(phase + kh * np.arange(-2, 3))
            eta, hb = oracle_mod.step4(q)
            if q[3] * q[1] < 0.0 and abs(q[3] - q[1]) > 0.01 * min(abs(q[3]), abs(q[1])):
                assert abs(eta - eta_x) <= 1e-13, (cells, phase, eta, eta_x)
                assert abs(hb - hbar_of(eta_x)) <= 1e-11
            elif q[3] * q[1] > 0.0:
                assert eta == 0.0 and hb == 0.0
        if cells >= 17:
            assert eta_x < 0.05
