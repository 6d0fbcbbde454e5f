"""Seeding a distribution from macroscopic fields (oracle; test infrastructure only).

The paper has no warm start; this is the reference for the seeding kernel that
turns predicted fields (n, u^0, u^1, T and the heat flux q) into the populations
of a model, and for the heat-flux term of the Shakhov collision.  The continuous distribution is Grad's 13-moment form
with only the heat-flux part kept, in three momentum dimensions (p^z is
integrated out as in Sec. II, which gives the reduced pair f', f''):

    f = f_M(n, u, T) [1 + (q . xi) / (n T^2) (xi^2 / (5 T) - 1)],   xi = p - u,

so that (1/2) int f xi^2 xi = q while n, u and T are those of f_M.  The
reduced functions (f' = int f dp^z, f'' = int (p^z)^2 f dp^z, u^z = 0) are

    f'  = n g_0 g_1 + q^0/T^2 g_0 g_1 xi_0 [(xi_0^2 + xi_1^2)/(5T) - 4/5],
    f'' = T n g_0 g_1 + q^0/T^2 g_0 g_1 xi_0 [(xi_0^2 + xi_1^2)/5 - 2T/5],

with g_a the unit-mass Gaussian of mean u^a and variance T on axis a.  Each
is a sum of products of one-axis functions xi_a^k g_a, so its projection on
the model's tensor-product basis is the sum of the products of the one-axis
projections.

One-axis projection (the definition, Sec. III): on a full-range axis the
function h is expanded on the orthonormal Hermite polynomials He_l/sqrt(l!),
c_l = int h He_l / sqrt(l!) dp for l <= N, and the population at node p_k is
w_k sum_l c_l He_l(p_k) / sqrt(l!).  On a half-range axis each semi-axis is
expanded separately on the orthonormal half-range polynomials h_l (Eq. hh_exp),
c_l^+- = int_0^inf h(+-p) h_l(p) dp, and the population at the node +-p_k is
w_k sum_l c_l^+- h_l(p_k).  The coefficients are computed here by adaptive
numerical integration (scipy.integrate.quad), independently of the closed
forms of Eqs. (eq_gak_H) and (eq_gak_hh).
"""
from __future__ import annotations

import functools
import math
import warnings

import numpy as np
from scipy import integrate

from . import quadrature as qd
from .lbmodel import Model


@functools.lru_cache(maxsize=None)
def _basis(kind: str, N: int, Q: int):
    """Float64 coefficients (ascending powers) of the orthonormal polynomials of degree 0..N."""
    if kind == "H":
        H = qd.hermite_family(N)
        return [np.array([float(c) for c in H[l]]) / math.sqrt(math.factorial(l)) for l in range(N + 1)]
    coeffs, _, _, _ = qd.half_range_family(max(Q, N))
    return [np.array([float(c) for c in coeffs[l]]) for l in range(N + 1)]


def _poly(c, x):
    return np.polynomial.polynomial.polyval(x, c)


def _coeffs(kind, N, Q, h, u, T):
    """Projection coefficients of h (callable) on one axis: full range -> (N+1,);
    half range -> ((N+1,), (N+1,)) for the positive and negative semi-axes.
    quad reports round-off on coefficients that vanish by symmetry; the
    accuracy of the result is what the pins of this module check."""
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        return _coeffs_quad(kind, N, Q, h, u, T)


def _coeffs_quad(kind, N, Q, h, u, T):
    B = _basis(kind, N, Q)
    s = math.sqrt(T)
    opts = dict(epsabs=1e-15, epsrel=1e-13, limit=400)
    if kind == "H":
        lo, hi = u - 40 * s, u + 40 * s
        return np.array([integrate.quad(lambda p, l=l: h(p) * _poly(B[l], p), lo, hi, points=[u], **opts)[0]
                         for l in range(N + 1)])
    out = []
    for sign in (1.0, -1.0):
        c = sign * u  # centre of h(sign p) on the positive semi-axis
        hi = max(c, 0.0) + 40 * s
        pts = [c] if 0.0 < c < hi else None
        out.append(np.array([integrate.quad(lambda p, l=l: h(sign * p) * _poly(B[l], p), 0.0, hi, points=pts,
                                            **opts)[0] for l in range(N + 1)]))
    return tuple(out)


def project_axis(model: Model, a: int, h, u, T):
    """Populations (nq_a,) of the one-axis function h (callable of p) on axis a."""
    kind, N, Q = model.spec[a]
    p, w = model.p[a], model.w[a]
    B = _basis(kind, N, Q)
    if kind == "H":
        c = _coeffs(kind, N, Q, h, u, T)
        return w * sum(c[l] * _poly(B[l], p) for l in range(N + 1))
    cp, cm = _coeffs(kind, N, Q, h, u, T)
    out = np.empty(len(p))
    for k, pk in enumerate(p):
        c = cp if pk > 0 else cm
        out[k] = w[k] * sum(c[l] * _poly(B[l], abs(pk)) for l in range(N + 1))
    return out


def _gauss_power(k, u, T):
    """xi^k g(p): the unit-mass Gaussian of mean u and variance T times (p - u)^k."""
    norm = 1.0 / math.sqrt(2.0 * math.pi * T)
    return lambda p: (p - u) ** k * norm * math.exp(-(p - u) ** 2 / (2.0 * T))


def seed(model: Model, n, u0, u1, T, q0=None, q1=None):
    """(f', f'') of shape (S, nq0, nq1) for fields per cell; q0 / q1 = None mean a zero
    heat flux along that axis.  The axis-1 part is the mirror of the axis-0 part:
    q^1/T^2 g_0 g_1 xi_1 [(xi_0^2 + xi_1^2)/(5T) - 4/5] in f' (and /5, 2T/5 in f'')."""
    n, u0, u1, T = (np.atleast_1d(np.asarray(x, dtype=np.float64)) for x in (n, u0, u1, T))
    q0 = np.zeros_like(n) if q0 is None else np.atleast_1d(np.asarray(q0, dtype=np.float64))
    q1 = np.zeros_like(n) if q1 is None else np.atleast_1d(np.asarray(q1, dtype=np.float64))
    S = len(n)
    f1 = np.empty((S, model.nq[0], model.nq[1]))
    f2 = np.empty_like(f1)
    for c in range(S):
        A = {k: project_axis(model, 0, _gauss_power(k, u0[c], T[c]), u0[c], T[c]) for k in (0, 1, 2, 3)}
        Bv = {k: project_axis(model, 1, _gauss_power(k, u1[c], T[c]), u1[c], T[c]) for k in (0, 1, 2, 3)}
        base = np.outer(A[0], Bv[0])
        t3 = np.outer(A[3], Bv[0]) + np.outer(A[1], Bv[2])  # xi_0 (xi_0^2 + xi_1^2) g_0 g_1
        t1 = np.outer(A[1], Bv[0])                           # xi_0 g_0 g_1
        s3 = np.outer(A[2], Bv[1]) + np.outer(A[0], Bv[3])  # xi_1 (xi_0^2 + xi_1^2) g_0 g_1
        s1 = np.outer(A[0], Bv[1])                           # xi_1 g_0 g_1
        Tc, a0, a1 = T[c], q0[c], q1[c]
        f1[c] = n[c] * base + (a0 * (t3 / (5.0 * Tc) - 0.8 * t1) + a1 * (s3 / (5.0 * Tc) - 0.8 * s1)) / Tc ** 2
        f2[c] = Tc * n[c] * base + (a0 * (t3 / 5.0 - 0.4 * Tc * t1) + a1 * (s3 / 5.0 - 0.4 * Tc * s1)) / Tc ** 2
    return f1, f2


def heat_flux_term(model: Model, n, u0, u1, T, q0, q1):
    """G = seed(n, u, T, q) - seed(n, u, T, 0): the heat-flux part of Grad's form on the model
    basis, (G', G'') of shape (S, nq0, nq1).  The Shakhov collision term, the extension of
    BGK the paper names in Sec. II.C, relaxes towards f_eq + (1 - Pr) G with G built from
    the current q, so that q relaxes at the rate Pr / tau."""
    f1, f2 = seed(model, n, u0, u1, T, q0, q1)
    b1, b2 = seed(model, n, u0, u1, T)
    return f1 - b1, f2 - b2
