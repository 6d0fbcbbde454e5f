"""Pins of the oracle's truncated equilibrium (Sec. IV.D) against Gaussian moments.

The truncated expansion of order N recovers every moment of order <= N exactly
(Sec. IV.D): full range against the moments of N(u, T); half range against the
half-line moments int_0^inf p^a N(p; u, T) dp, integrated here numerically.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import lbmodel as lb


def gauss(p, u, T):
    return math.exp(-(p - u) ** 2 / (2 * T)) / math.sqrt(2 * math.pi * T)


def full_line_moment(a, u, T):
    # E[X^a] for X ~ N(u, T): sum over even k of C(a, k) u^{a-k} T^{k/2} (k-1)!!
    return sum(math.comb(a, k) * u ** (a - k) * T ** (k // 2) * math.prod(range(k - 1, 0, -2))
               for k in range(0, a + 1, 2))


def half_line_moments(amax, u, T):
    # M_a = int_0^inf p^a N(p; u, T) dp by integration by parts:
    # M_0 = (1 + erf(u / sqrt(2T))) / 2,  M_a = u M_{a-1} + (a-1) T M_{a-2} + [a == 1] T N(0; u, T)
    M = [0.5 * (1.0 + math.erf(u / math.sqrt(2.0 * T)))]
    for a in range(1, amax + 1):
        M.append(u * M[a - 1] + ((a - 1) * T * M[a - 2] if a >= 2 else T * gauss(0.0, u, T)))
    return M


@pytest.mark.parametrize("spec", ["H(2;3)", "H(4;5)", "H(4;12)", "H(4;20)", "H(3;4)"])
@pytest.mark.parametrize("u,T", [(0.0, 1.0), (0.3, 1.2), (-0.45, 0.8), (0.1, 1.0)])
def test_full_range_moments(spec, u, T):
    kind, N, Q = lb.parse_model(spec + "xH(2;3)")[0]
    m = lb.Model([(kind, N, Q), ("H", 2, 3)])
    g = m.g_axis(0, [u], [T])[0]
    p = m.p[0]
    for a in range(N + 1):
        exact = full_line_moment(a, u, T)
        assert float(np.sum(g * p ** a)) == pytest.approx(exact, rel=1e-12, abs=1e-13)


@pytest.mark.parametrize("spec", ["HH(2;3)", "HH(3;4)", "HH(4;8)", "HH(4;16)"])
@pytest.mark.parametrize("u,T", [(0.0, 1.0), (0.3, 1.2), (-0.45, 0.8), (0.05, 1.0)])
def test_half_range_moments(spec, u, T):
    kind, N, Q = lb.parse_model(spec + "xH(2;3)")[0]
    m = lb.Model([(kind, N, Q), ("H", 2, 3)])
    g = m.g_axis(0, [u], [T])[0]
    p = m.p[0]
    Mp = half_line_moments(N, u, T)
    Mm = half_line_moments(N, -u, T)
    for a in range(N + 1):
        plus, minus = Mp[a], (-1) ** a * Mm[a]
        # the recurrence itself against direct integration
        assert plus == pytest.approx(quad(lambda x: x ** a * gauss(x, u, T), 0, 40, epsabs=1e-13, limit=200)[0], rel=1e-8)
        assert float(np.sum(g[:Q] * p[:Q] ** a)) == pytest.approx(plus, rel=1e-12, abs=1e-14)
        assert float(np.sum(g[Q:] * p[Q:] ** a)) == pytest.approx(minus, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("spec", ["HH(4;8)xH(4;20)", "HH(3;4)xH(3;4)", "H(4;5)xH(4;5)"])
def test_rest_equilibrium_is_the_weights(spec):
    m = lb.Model(spec)
    for a in (0, 1):
        np.testing.assert_allclose(m.g_axis(a, [0.0], [1.0])[0], m.w[a], rtol=1e-13, atol=1e-18)


@pytest.mark.parametrize("spec", ["HH(4;8)xH(4;20)", "HH(3;4)xH(3;4)", "H(4;5)xH(4;5)"])
def test_equilibrium_is_a_collision_fixed_point(spec):
    # moments of f_eq(n, u, T) give back (n, u, T) (N >= 2), so J[f_eq] = 0
    m = lb.Model(spec)
    n = np.array([1.0, 0.7, 1.4]); u0 = np.array([0.0, 0.2, -0.1])
    u1 = np.array([0.0, -0.3, 0.45]); T = np.array([1.0, 1.3, 0.85])
    f1, f2 = m.feq(n, u0, u1, T)
    got = m.moments(np.stack([f1, f2]))
    for x, y in zip(got, (n, u0, u1, T)):
        np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-13)
