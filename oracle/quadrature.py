"""Full-range and half-range Gauss-Hermite quadratures (oracle; test infrastructure only).

Sec. IV.B defines the two rules used on each momentum axis:

* full range: nodes are the roots of the probabilists' Hermite polynomial H_Q
  (orthogonal on the real line under omega(x) = exp(-x^2/2)/sqrt(2 pi)), with
  weights from Eq. (w_H):  w_k = Q! / H_{Q+1}(p_k)^2;
* half range: nodes on the positive semi-axis are the roots of the half-range
  Hermite polynomial h_Q (Eq. hh_roots), mirrored to the negative semi-axis
  (p_{Q+i} = -p_i); weights from Eq. (w_hh)
      w_i = p_i a_{Q-1}^2 / ( h_{Q-1}(p_i)^2 [p_i + h_Q(0)^2 / sqrt(2 pi)] ),
  with a_l = h_{l+1,l+1} / h_{l,l} (Eq. hh_a) and h_{l,s} the coefficient of
  x^s in h_l (Eq. hh_exp).

The paper does not spell out the normalisation of h_l.  Reading used here:
h_l is orthonormal on [0, inf) under omega, with a positive leading
coefficient (so h_0 = sqrt(2)).  With that reading Eq. (w_hh) gives w = 1/2 for
Q = 1, the half-range weights sum to 1/2 on each semi-axis, and the force
kernels of Sec. IV.C conserve mass and momentum.

Everything is computed in ``decimal`` arithmetic at a precision that grows
with Q (Gram-Schmidt on exact half-Gaussian moments loses digits as Q grows),
then rounded to float64.  Roots are found by bisection on the Sturm sign-change
count of the orthogonal family, which is slow but obviously correct.
"""
from __future__ import annotations

import functools
from decimal import Decimal, localcontext

import numpy as np


def _digits(Q: int) -> int:
    return 60 + 4 * Q


def _pi(ctx) -> Decimal:
    """pi by Machin's formula, 16 atan(1/5) - 4 atan(1/239), to the context precision."""
    def atan_inv(n: int) -> Decimal:
        x = Decimal(1) / n
        x2 = x * x
        term, total, k = x, x, 1
        eps = Decimal(10) ** (-(ctx.prec + 5))
        while abs(term) > eps:
            term *= -x2
            total += term / (2 * k + 1)
            k += 1
        return total
    return 16 * atan_inv(5) - 4 * atan_inv(239)


def _poly_eval(c, x):
    """Horner evaluation of sum_s c[s] x^s."""
    acc = c[-1] * 0
    for a in reversed(c):
        acc = acc * x + a
    return acc


def _count_roots_below(x, alpha, beta):
    """Number of zeros of p_n below x for the monic family
    p_{k+1} = (x - alpha_k) p_k - beta_k p_{k-1}: n minus the sign changes of
    (p_0(x), ..., p_n(x)) (Sturm property of orthogonal polynomials)."""
    n = len(alpha)
    p_prev, p = Decimal(0), Decimal(1)
    changes = 0
    last_sign = 1
    for k in range(n):
        p_next = (x - alpha[k]) * p - (beta[k] * p_prev if k > 0 else 0)
        p_prev, p = p, p_next
        if p != 0:
            s = 1 if p > 0 else -1
            if s != last_sign:
                changes += 1
            last_sign = s
        else:
            # an exact zero takes the sign opposite to its predecessor (standard convention)
            last_sign = -last_sign
            changes += 1
    return n - changes


def _bisect_roots(alpha, beta, lo, hi, iters):
    n = len(alpha)
    roots = []
    for k in range(n):
        a, b = Decimal(lo), Decimal(hi)
        for _ in range(iters):
            m = (a + b) / 2
            if _count_roots_below(m, alpha, beta) > k:
                b = m
            else:
                a = m
        roots.append((a + b) / 2)
    return roots


@functools.lru_cache(maxsize=None)
def half_range_family(Q: int):
    """Coefficients h_{l,s} (l = 0..Q, s = 0..l) of the orthonormal half-range
    Hermite polynomials, plus the monic recurrence coefficients, in Decimal.

    Built by Gram-Schmidt (Stieltjes form) on the exact moments of omega on
    [0, inf):  mu_k = int_0^inf x^k omega dx,  mu_0 = 1/2, mu_1 = 1/sqrt(2 pi),
    mu_k = (k - 1) mu_{k-2}.
    """
    with localcontext() as ctx:
        ctx.prec = _digits(Q)
        pi = _pi(ctx)
        s2pi = (2 * pi).sqrt()
        K = 2 * Q + 2
        mu = [Decimal(0)] * (K + 1)
        mu[0] = Decimal(1) / 2
        mu[1] = 1 / s2pi
        for k in range(2, K + 1):
            mu[k] = (k - 1) * mu[k - 2]

        def inner(a, b):
            return sum(a[i] * b[j] * mu[i + j] for i in range(len(a)) for j in range(len(b)))

        monic = [[Decimal(1)]]
        alpha, beta = [], []
        norms = [inner(monic[0], monic[0])]
        for k in range(Q):
            pk = monic[k]
            xpk = [Decimal(0)] + pk
            a_k = inner(xpk, pk) / norms[k]
            alpha.append(a_k)
            nxt = [xpk[i] - (a_k * pk[i] if i < len(pk) else 0) for i in range(len(xpk))]
            if k > 0:
                b_k = norms[k] / norms[k - 1]
                beta.append(b_k)
                pm = monic[k - 1]
                for i in range(len(pm)):
                    nxt[i] -= b_k * pm[i]
            else:
                beta.append(Decimal(0))
            monic.append(nxt)
            norms.append(inner(nxt, nxt))
        coeffs = [[c / norms[l].sqrt() for c in monic[l]] for l in range(Q + 1)]
        return coeffs, alpha, beta, pi


@functools.lru_cache(maxsize=None)
def half_range_rule(Q: int):
    """Nodes p (length 2Q: Q positive roots of h_Q ascending, then their negatives)
    and weights w (Eq. w_hh, same weight for a node and its mirror), float64,
    together with the Decimal positive nodes for table construction."""
    coeffs, alpha, beta, pi = half_range_family(Q)
    with localcontext() as ctx:
        ctx.prec = _digits(Q)
        hi = 4 + 3 * Decimal(Q).sqrt()
        roots = _bisect_roots(alpha, beta, 0, hi, iters=int(3.4 * ctx.prec) + 20)
        s2pi = (2 * pi).sqrt()
        hQ0 = coeffs[Q][0]
        a_Qm1 = coeffs[Q][Q] / coeffs[Q - 1][Q - 1]
        w = []
        for p in roots:
            hqm1 = _poly_eval(coeffs[Q - 1], p)
            w.append(p * a_Qm1 ** 2 / (hqm1 ** 2 * (p + hQ0 ** 2 / s2pi)))
    pos = np.array([float(r) for r in roots])
    wpos = np.array([float(x) for x in w])
    return np.concatenate([pos, -pos]), np.concatenate([wpos, wpos]), roots, w


@functools.lru_cache(maxsize=None)
def hermite_family(L: int):
    """Integer coefficients of the probabilists' Hermite polynomials H_0..H_L,
    H_{l+1} = x H_l - l H_{l-1}."""
    H = [[1], [0, 1]]
    for l in range(1, L):
        nxt = [0] + H[l]
        for i, c in enumerate(H[l - 1]):
            nxt[i] -= l * c
        H.append(nxt)
    return [list(map(Decimal, h)) for h in H[: L + 1]]


@functools.lru_cache(maxsize=None)
def full_range_rule(Q: int):
    """Nodes (roots of H_Q, ascending) and weights of Eq. (w_H), float64, plus Decimal nodes."""
    with localcontext() as ctx:
        ctx.prec = _digits(Q)
        alpha = [Decimal(0)] * Q
        beta = [Decimal(k) for k in range(Q)]
        lim = 3 + 2 * Decimal(Q).sqrt()
        roots = _bisect_roots(alpha, beta, -lim, lim, iters=int(3.4 * ctx.prec) + 20)
        H = hermite_family(Q + 1)
        fact = Decimal(1)
        for k in range(2, Q + 1):
            fact *= k
        w = [fact / _poly_eval(H[Q + 1], p) ** 2 for p in roots]
    return (np.array([float(r) for r in roots]), np.array([float(x) for x in w]), roots, w)


def rule(kind: str, Q: int):
    """(p, w) float64 for an axis: kind 'H' (full range, Q nodes) or 'HH' (half range, 2Q nodes)."""
    if kind == "H":
        p, w, _, _ = full_range_rule(Q)
    elif kind == "HH":
        p, w, _, _ = half_range_rule(Q)
    else:
        raise ValueError(kind)
    return p, w
