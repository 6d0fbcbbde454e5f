"""Pins of the oracle's force kernels K, K~ (Sec. IV.C, App. D).

Two independent checks:
* conservation invariants that hold for the exact derivative operator:
  int d_p f = 0, int p d_p f = -int f, int d_p(p f) = 0, int p d_p(p f) = -int p f;
* a second construction of each kernel, written here from the definition
  (expand f in the orthogonal basis by quadrature, differentiate the expansion
  with numpy polynomial algebra and scipy integration, add the half-range
  jump term delta(p)[f+(0) - f-(0)] split half to each semi-axis), compared
  entry by entry with the printed formulas the oracle implements.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import lbmodel as lb
from oracle import quadrature as qd

OM0 = 1.0 / math.sqrt(2.0 * math.pi)
pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def omega(x):
    return np.exp(-x * x / 2.0) * OM0


def kernels(kind, Q):
    if kind == "H":
        return lb.kernel_K_full(Q), lb.kernel_Kt_full(Q)
    return lb.kernel_K_half(Q), lb.kernel_Kt_half(Q)


@pytest.mark.parametrize("kind,Q", [("H", 3), ("H", 4), ("H", 5), ("H", 12), ("H", 20),
                                    ("HH", 2), ("HH", 3), ("HH", 4), ("HH", 8)])
def test_conservation_invariants(kind, Q):
    K, Kt = kernels(kind, Q)
    p, w = qd.rule(kind, Q)
    for M, first in ((K, None), (Kt, p)):
        scale0 = np.abs(M).sum(axis=0)
        scale1 = np.abs(p[:, None] * M).sum(axis=0)
        assert np.all(np.abs(M.sum(axis=0)) <= 1e-13 * scale0 + 1e-15)
        target = -np.ones_like(p) if first is None else -p
        assert np.all(np.abs((p[:, None] * M).sum(axis=0) - target) <= 1e-13 * scale1 + 1e-15)


@pytest.mark.parametrize("Q", [3, 4, 6, 9])
def test_full_range_exact_on_gaussian_times_polynomial(Q):
    K, Kt = kernels("H", Q)
    p, w = qd.rule("H", Q)
    rng = np.random.default_rng(Q)
    for deg, M, which in ((Q - 1, K, "f"), (Q - 2, Kt, "pf")):
        P = np.polynomial.Polynomial(rng.normal(size=deg + 1))
        f = w * P(p)  # weighted populations of f = omega P
        if which == "f":  # d/dp (omega P) = omega (P' - p P)
            exact = w * (P.deriv()(p) - p * P(p))
        else:  # d/dp (p omega P) = omega ((pP)' - p^2 P)
            X = np.polynomial.Polynomial([0, 1])
            exact = w * ((X * P).deriv()(p) - p * p * P(p))
        np.testing.assert_allclose(M @ f, exact, rtol=1e-10, atol=1e-12 * np.abs(exact).max())


def _half_basis(Q):
    coeffs, _, _, _ = qd.half_range_family(Q)
    return [np.polynomial.Polynomial([float(c) for c in row]) for row in coeffs[:Q]]


def _independent_half_kernels(Q):
    """K and K~ for the half-range rule built from the definition."""
    p, w = qd.rule("HH", Q)
    h = _half_basis(Q)
    X = np.polynomial.Polynomial([0, 1])
    n = 2 * Q
    K = np.zeros((n, n))
    Kt = np.zeros((n, n))
    for kp in range(n):
        f = np.zeros(n)
        f[kp] = 1.0
        # expansion coefficients on each semi-axis
        Fp = np.array([np.sum(f[:Q] * h[l](p[:Q])) for l in range(Q)])
        Fm = np.array([np.sum(f[Q:] * h[l](-p[Q:])) for l in range(Q)])
        Pp = sum(Fp[l] * h[l] for l in range(Q))  # f^+(x) = omega(x) Pp(x),  x = |p| > 0
        Pm = sum(Fm[l] * h[l] for l in range(Q))  # f^-(p) = omega(p) Pm(-p)
        jump = OM0 * (Pp(0.0) - Pm(0.0))
        cp, cm, ctp, ctm = (np.zeros(Q) for _ in range(4))
        for s in range(Q):
            hs = h[s]
            # positive side: d/dx (omega Pp) = omega (Pp' - x Pp)
            dP = Pp.deriv() - X * Pp
            cp[s] = quad(lambda x: omega(x) * dP(x) * hs(x), 0, np.inf, epsabs=1e-14, epsrel=1e-13)[0] + 0.5 * hs(0.0) * jump
            # negative side with x = -p: d/dp = -d/dx
            dM = -(Pm.deriv() - X * Pm)
            cm[s] = quad(lambda x: omega(x) * dM(x) * hs(x), 0, np.inf, epsabs=1e-14, epsrel=1e-13)[0] + 0.5 * hs(0.0) * jump
            # d/dp (p f): positive side omega ((x Pp)' - x^2 Pp); negative side same form in x
            dtP = (X * Pp).deriv() - X * X * Pp
            dtM = (X * Pm).deriv() - X * X * Pm
            ctp[s] = quad(lambda x: omega(x) * dtP(x) * hs(x), 0, np.inf, epsabs=1e-14, epsrel=1e-13)[0]
            ctm[s] = quad(lambda x: omega(x) * dtM(x) * hs(x), 0, np.inf, epsabs=1e-14, epsrel=1e-13)[0]
        for k in range(n):
            x = abs(p[k])
            c, ct = (cp, ctp) if k < Q else (cm, ctm)
            K[k, kp] = w[k] * sum(c[s] * h[s](x) for s in range(Q))
            Kt[k, kp] = w[k] * sum(ct[s] * h[s](x) for s in range(Q))
    return K, Kt


@pytest.mark.parametrize("Q", [2, 3, 4, 5])
def test_half_range_kernels_match_definition(Q):
    K, Kt = kernels("HH", Q)
    Ki, Kti = _independent_half_kernels(Q)
    np.testing.assert_allclose(K, Ki, rtol=0, atol=1e-9 * np.abs(Ki).max())
    np.testing.assert_allclose(Kt, Kti, rtol=0, atol=1e-9 * np.abs(Kti).max())


def test_half_range_K_exact_on_continuous_gaussian_polynomial():
    # a continuous f = omega(p) P(p) with deg P <= Q-2 is differentiated exactly
    Q = 6
    K, _ = kernels("HH", Q)
    p, w = qd.rule("HH", Q)
    P = np.polynomial.Polynomial([0.3, -0.2, 0.5, 0.1, -0.05])
    f = w * P(p)
    exact = w * (P.deriv()(p) - p * P(p))
    np.testing.assert_allclose(K @ f, exact, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("kind,Q", [("H", 4), ("H", 5), ("H", 12), ("H", 20), ("HH", 2), ("HH", 4), ("HH", 8)])
def test_kernels_commute_with_the_reflection(kind, Q):
    """d/dp anticommutes and d/dp (p .) commutes with f(p) -> f(-p); the printed
    kernels keep this exactly on the symmetric node sets (the stage kernels of the
    library split both contractions into even and odd parts on that basis)."""
    m = lb.Model(f"{kind}({min(Q - 1, 4)};{Q})x{kind}({min(Q - 1, 4)};{Q})")
    p, K, Kt = m.p[0], m.K[0], m.Kt[0]
    J = np.array([int(np.argmin(np.abs(p + pk))) for pk in p])
    np.testing.assert_allclose(p[J], -p, rtol=0, atol=1e-14 * np.abs(p).max())
    np.testing.assert_allclose(K[np.ix_(J, J)], -K, rtol=0, atol=1e-13 * np.abs(K).max())
    np.testing.assert_allclose(Kt[np.ix_(J, J)], Kt, rtol=0, atol=1e-13 * np.abs(Kt).max())
