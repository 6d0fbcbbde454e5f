"""Pins of the oracle's Gauss-Hermite rules (Sec. IV.B) against textbook facts."""
import math

import numpy as np
import pytest

from oracle import quadrature as qd


def half_gauss_moment(k):
    # int_0^inf x^k exp(-x^2/2)/sqrt(2 pi) dx = 2^{(k-1)/2} Gamma((k+1)/2) / sqrt(2 pi)
    return 2.0 ** ((k - 1) / 2.0) * math.gamma((k + 1) / 2.0) / math.sqrt(2.0 * math.pi)


def full_gauss_moment(k):
    return 0.0 if k % 2 else float(math.prod(range(k - 1, 0, -2)))


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 8, 12, 16])
def test_half_range_exact_on_polynomials(Q):
    p, w = qd.rule("HH", Q)
    assert p.shape == (2 * Q,) and np.all(p[:Q] > 0) and np.allclose(p[Q:], -p[:Q])
    for k in range(2 * Q):
        got = float(np.sum(w[:Q] * p[:Q] ** k))
        assert got == pytest.approx(half_gauss_moment(k), rel=2e-14, abs=1e-16)
    # the same rule on the negative semi-axis
    for k in range(2 * Q):
        got = float(np.sum(w[Q:] * np.abs(p[Q:]) ** k))
        assert got == pytest.approx(half_gauss_moment(k), rel=2e-14, abs=1e-16)


def test_half_range_Q1_by_hand():
    # h_1 has its root at the mean of the half-Gaussian, sqrt(2/pi); Eq. (w_hh) gives w = 1/2
    p, w = qd.rule("HH", 1)
    assert p[0] == pytest.approx(math.sqrt(2.0 / math.pi), rel=1e-15)
    assert w[0] == pytest.approx(0.5, rel=1e-15)


@pytest.mark.parametrize("Q", [3, 4, 5, 12, 20])
def test_full_range_matches_golub_welsch(Q):
    p, w = qd.rule("H", Q)
    x, ww = np.polynomial.hermite_e.hermegauss(Q)
    np.testing.assert_allclose(p, x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(w, ww / math.sqrt(2.0 * math.pi), rtol=1e-12, atol=1e-18)
    for k in range(2 * Q):
        scale = float(np.sum(np.abs(w * p ** k)))
        assert abs(float(np.sum(w * p ** k)) - full_gauss_moment(k)) <= 1e-14 * scale


def test_half_range_polynomials_orthonormal():
    # h_l orthonormal on [0, inf) under omega: check with an independent float64
    # scipy integration of the Decimal coefficients
    from scipy.integrate import quad
    coeffs, _, _, _ = qd.half_range_family(6)
    c = [[float(x) for x in row] for row in coeffs]
    om = lambda x: math.exp(-x * x / 2) / math.sqrt(2 * math.pi)
    for a in range(6):
        for b in range(a + 1):
            f = lambda x: om(x) * np.polyval(c[a][::-1], x) * np.polyval(c[b][::-1], x)
            val, _ = quad(f, 0, np.inf, epsabs=1e-13, epsrel=1e-13)
            assert val == pytest.approx(1.0 if a == b else 0.0, abs=1e-10)
        assert c[a][a] > 0
    assert c[0][0] == pytest.approx(math.sqrt(2.0), rel=1e-15)
