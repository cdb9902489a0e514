"""Pins of the oracle's cardinal Z-spline basis (Sec. 2.1 properties (a)-(c), Appendix).

Each property is fixed by the paper's definition, not by the oracle's own formula:
interpolation at the integers, compact support, the discrete-moment conditions, C^m continuity
with piecewise degree 2m+1 (eqs. zcontin, zpolynom), and the construction itself -- a Hermite
interpolant whose node derivatives are centered finite differences of 2m+1 points (eq. matchder);
and the piecewise polynomials the Appendix prints (tests/golden/zspline_appendix.txt).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

M_ALL = (0, 1, 2)


@pytest.mark.parametrize("m", M_ALL)
def test_interpolates_at_integers(oracle_mod, m):
    k = np.arange(-5, 6, dtype=float)
    z = oracle_mod.zspline(m, k)
    expect = (k == 0).astype(float)
    assert np.max(np.abs(z - expect)) <= 1e-13


@pytest.mark.parametrize("m", M_ALL)
def test_compact_support_and_symmetry(oracle_mod, m):
    rng = np.random.default_rng(1)
    x = rng.uniform(m + 1, m + 6, 200)
    assert np.all(oracle_mod.zspline(m, x) == 0.0)
    assert np.all(oracle_mod.zspline(m, -x) == 0.0)
    y = rng.uniform(-m - 1, m + 1, 200)
    assert np.array_equal(oracle_mod.zspline(m, y), oracle_mod.zspline(m, -y))


def _discrete_moment(oracle_mod, m, x, n):
    j = np.arange(np.floor(x) - m - 2, np.floor(x) + m + 3)
    return float(np.sum((x - j) ** n * oracle_mod.zspline(m, x - j)))


@pytest.mark.parametrize("m", M_ALL)
def test_discrete_moments(oracle_mod, m):
    """sum_j (x-j)^n Z~_m(x-j) = delta_0n.  The reading of the garbled range "first 2m+1 moments,
    n = 0..m" adopted here is n = 0..2m (Z~_0 also keeps n = 1); degree 2m+1 is NOT kept."""
    rng = np.random.default_rng(2)
    top = max(2 * m, 1)
    for x in rng.uniform(-3, 3, 25):
        for n in range(top + 1):
            assert abs(_discrete_moment(oracle_mod, m, x, n) - (1.0 if n == 0 else 0.0)) <= 1e-13 * (m + 2) ** n
    worst = max(abs(_discrete_moment(oracle_mod, m, x, top + 1)) for x in rng.uniform(0.1, 0.9, 25))
    assert worst > 1e-3


def _piece_poly(oracle_mod, m, a, b, deg):
    """Fit the exact polynomial of one piece [a, b] from deg+1 interior samples."""
    xs = np.linspace(a + 0.1 * (b - a), b - 0.1 * (b - a), deg + 1)
    ys = oracle_mod.zspline(m, xs)
    return np.polynomial.Polynomial.fit(xs, ys, deg).convert()


@pytest.mark.parametrize("m", (1, 2))
def test_piecewise_degree_and_continuity(oracle_mod, m):
    """Each piece between integers is a polynomial of degree 2m+1 and Z~_m is C^m at the knots."""
    deg = 2 * m + 1
    rng = np.random.default_rng(3)
    for knot in range(-m - 1, m + 2):
        left = _piece_poly(oracle_mod, m, knot - 1, knot, deg)
        right = _piece_poly(oracle_mod, m, knot, knot + 1, deg)
        # the fitted polynomial reproduces the piece elsewhere (degree is not higher than 2m+1)
        xs = rng.uniform(knot + 0.05, knot + 0.95, 7)
        assert np.max(np.abs(right(xs) - oracle_mod.zspline(m, xs))) <= 1e-11
        for p in range(m + 1):
            tol = 1e-8 if p else 1e-10
            assert abs(left.deriv(p)(knot) - right.deriv(p)(knot)) <= tol
        # and not C^(m+1) everywhere: some knot must break the next derivative
    jumps = []
    for knot in range(-m - 1, m + 2):
        left = _piece_poly(oracle_mod, m, knot - 1, knot, deg)
        right = _piece_poly(oracle_mod, m, knot, knot + 1, deg)
        jumps.append(abs(left.deriv(m + 1)(knot) - right.deriv(m + 1)(knot)))
    assert max(jumps) > 1e-3


def _hermite_cubic(h, x):
    i = int(np.floor(x))
    t = x - i
    d0 = (h[i + 1] - h[i - 1]) / 2.0
    d1 = (h[i + 2] - h[i]) / 2.0
    return ((2 * t ** 3 - 3 * t ** 2 + 1) * h[i] + (t ** 3 - 2 * t ** 2 + t) * d0
            + (-2 * t ** 3 + 3 * t ** 2) * h[i + 1] + (t ** 3 - t ** 2) * d1)


def _fd5(h, i):
    d1 = (h[i - 2] - 8 * h[i - 1] + 8 * h[i + 1] - h[i + 2]) / 12.0
    d2 = (-h[i - 2] + 16 * h[i - 1] - 30 * h[i] + 16 * h[i + 1] - h[i + 2]) / 12.0
    return d1, d2


def _hermite_quintic(h, x):
    i = int(np.floor(x))
    t = x - i
    v0, a0 = _fd5(h, i)
    v1, a1 = _fd5(h, i + 1)
    H0 = 1 - 10 * t ** 3 + 15 * t ** 4 - 6 * t ** 5
    H1 = t - 6 * t ** 3 + 8 * t ** 4 - 3 * t ** 5
    H2 = 0.5 * t ** 2 - 1.5 * t ** 3 + 1.5 * t ** 4 - 0.5 * t ** 5
    H3 = 0.5 * t ** 3 - t ** 4 + 0.5 * t ** 5
    H4 = -4 * t ** 3 + 7 * t ** 4 - 3 * t ** 5
    H5 = 10 * t ** 3 - 15 * t ** 4 + 6 * t ** 5
    return H0 * h[i] + H1 * v0 + H2 * a0 + H3 * a1 + H4 * v1 + H5 * h[i + 1]


@pytest.mark.parametrize("m", (1, 2))
def test_equals_hermite_construction(oracle_mod, m):
    """Z_m(x) = sum_i h_i Z~_m(x - i) is the piecewise Hermite polynomial of degree 2m+1 that
    matches h and its first m derivatives taken from centered finite differences of 2m+1 points
    (eqs. zcontin, matchder, zpolynom); the Appendix calls Z~_1 cubic Bessel interpolation."""
    rng = np.random.default_rng(4)
    h = rng.standard_normal(40)
    k = np.arange(40)
    for x in rng.uniform(8, 30, 20):
        zsum = float(np.sum(h * oracle_mod.zspline(m, x - k)))
        ref = _hermite_cubic(h, x) if m == 1 else _hermite_quintic(h, x)
        assert abs(zsum - ref) <= 1e-12 * max(1.0, abs(ref))


def test_hat_is_linear_interpolation(oracle_mod):
    rng = np.random.default_rng(5)
    h = rng.standard_normal(20)
    k = np.arange(20)
    for x in rng.uniform(2, 17, 20):
        assert abs(float(np.sum(h * oracle_mod.zspline(0, x - k))) - np.interp(x, k, h)) <= 1e-14


def test_sinpi_cospi_exact_points(oracle_mod):
    for k in range(-6, 7):
        assert oracle_mod.sinpi(float(k)) == 0.0
        assert oracle_mod.cospi(k + 0.5) == 0.0
        assert abs(oracle_mod.sinpi(k + 0.5)) == 1.0
        assert abs(oracle_mod.cospi(float(k))) == 1.0
    rng = np.random.default_rng(6)
    for x in rng.uniform(-5, 5, 100):
        assert abs(oracle_mod.sinpi(x) - np.sin(np.pi * x)) <= 4e-15
        assert abs(oracle_mod.cospi(x) - np.cos(np.pi * x)) <= 4e-15


GOLDEN_APPENDIX = os.path.join(os.path.dirname(__file__), "golden", "zspline_appendix.txt")


def _appendix_pieces():
    pieces = []
    with open(GOLDEN_APPENDIX) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            m, a, b, *coef = line.split()
            pieces.append((int(m), int(a), int(b), [float(Fraction(c)) for c in coef]))
    return pieces


def test_matches_the_printed_appendix_polynomials(oracle_mod):
    """Every piece of Z~_1 and Z~_2 equals the polynomial the Appendix prints for it (both signs
    of x, interior points and the knots)."""
    pieces = _appendix_pieces()
    assert sorted((m, a) for m, a, _, _ in pieces) == [(1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
    for m, a, b, coef in pieces:
        s = np.concatenate([np.linspace(a, b, 41), np.random.default_rng(m * 10 + a).uniform(a, b, 50)])
        printed = np.polynomial.polynomial.polyval(s, coef)
        for sign in (1.0, -1.0):
            got = oracle_mod.zspline(m, sign * s)
            assert np.max(np.abs(got - printed)) <= 1e-13, (m, a, b, sign)
    # the cubic's second piece is printed factored
    s = np.linspace(1.0, 2.0, 11)
    cubic2 = [c for m, a, _, c in pieces if (m, a) == (1, 1)][0]
    assert np.max(np.abs(np.polynomial.polynomial.polyval(s, cubic2) - 0.5 * (2 - s) ** 2 * (1 - s))) <= 1e-15
