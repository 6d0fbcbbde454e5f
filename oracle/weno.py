"""Epsilon-free WENO-5 interface values (oracle; test infrastructure only).

Sec. III.C, Eqs. (weno5_flux), (weno5_omega), (weno_sigma) and Table IV.
For an upwind direction with V_{s+1/2} > 0 the five-point stencil is
(F_{s-2}, F_{s-1}, F_s, F_{s+1}, F_{s+2}); for V_{s+1/2} < 0 the paper gives no
formula, and the reading used here is the mirror stencil
(F_{s+3}, F_{s+2}, F_{s+1}, F_s, F_{s-1}) fed to the same expressions.

Weights: w~_q = delta_q / sigma_q^2 with ideal weights (1/10, 6/10, 3/10),
normalised to sum one.  When one or more sigma_q vanish exactly, Table IV's
limiting values are used: the weight is shared among the vanishing indicators
in proportion to delta_q (all three zero gives the ideal weights).
"""
from __future__ import annotations

import numpy as np

D1, D2, D3 = 0.1, 0.6, 0.3


def weno5(a, b, c, d, e):
    """Interface value from the upwind-ordered stencil (a, b, c, d, e) =
    (F_{s-2}, F_{s-1}, F_s, F_{s+1}, F_{s+2}) for positive advection velocity.
    Works elementwise on numpy arrays of equal shape."""
    a, b, c, d, e = (np.asarray(x, dtype=np.float64) for x in (a, b, c, d, e))
    # candidate interpolants
    F1 = a / 3.0 - 7.0 / 6.0 * b + 11.0 / 6.0 * c
    F2 = -b / 6.0 + 5.0 / 6.0 * c + d / 3.0
    F3 = c / 3.0 + 5.0 / 6.0 * d - e / 6.0
    # smoothness indicators, Eq. (weno_sigma)
    s1 = 13.0 / 12.0 * (a - 2.0 * b + c) ** 2 + 0.25 * (a - 4.0 * b + 3.0 * c) ** 2
    s2 = 13.0 / 12.0 * (b - 2.0 * c + d) ** 2 + 0.25 * (b - d) ** 2
    s3 = 13.0 / 12.0 * (c - 2.0 * d + e) ** 2 + 0.25 * (3.0 * c - 4.0 * d + e) ** 2

    z1, z2, z3 = s1 == 0.0, s2 == 0.0, s3 == 0.0
    anyzero = z1 | z2 | z3
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = np.where(anyzero, 0.0, D1 / np.where(z1, 1.0, s1) ** 2)
        t2 = np.where(anyzero, 0.0, D2 / np.where(z2, 1.0, s2) ** 2)
        t3 = np.where(anyzero, 0.0, D3 / np.where(z3, 1.0, s3) ** 2)
    # Table IV: exact zeros share the weight in proportion to the ideal weights
    t1 = np.where(anyzero, np.where(z1, D1, 0.0), t1)
    t2 = np.where(anyzero, np.where(z2, D2, 0.0), t2)
    t3 = np.where(anyzero, np.where(z3, D3, 0.0), t3)
    tot = t1 + t2 + t3
    return (t1 * F1 + t2 * F2 + t3 * F3) / tot


def weno5_weights(a, b, c, d, e):
    """The normalised weights (w1, w2, w3) for scalars; used by the Table IV pin."""
    s = [13.0 / 12.0 * (a - 2 * b + c) ** 2 + 0.25 * (a - 4 * b + 3 * c) ** 2,
         13.0 / 12.0 * (b - 2 * c + d) ** 2 + 0.25 * (b - d) ** 2,
         13.0 / 12.0 * (c - 2 * d + e) ** 2 + 0.25 * (3 * c - 4 * d + e) ** 2]
    D = [D1, D2, D3]
    if any(x == 0.0 for x in s):
        t = [D[q] if s[q] == 0.0 else 0.0 for q in range(3)]
    else:
        t = [D[q] / s[q] ** 2 for q in range(3)]
    tot = sum(t)
    return [x / tot for x in t]


def upwind_interfaces(G, positive, axis=1):
    """Interface values between G[j] and G[j + 1] along `axis`, j = 2 .. len - 4 (the
    interfaces s + 1/2 of data with three ghost layers on each side): the stencil
    (G[j-2], ..., G[j+2]) where `positive` holds (advection velocity >= 0), the
    mirror stencil (G[j+3], G[j+2], G[j+1], G[j], G[j-1]) elsewhere.  `positive`
    broadcasts against the result."""
    n = G.shape[axis]
    j = np.arange(2, n - 3)
    at = lambda k: np.take(G, j + k, axis=axis)
    up = weno5(at(-2), at(-1), at(0), at(1), at(2))
    dn = weno5(at(3), at(2), at(1), at(0), at(-1))
    return np.where(positive, up, dn)
