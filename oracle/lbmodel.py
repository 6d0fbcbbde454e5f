"""Mixed-quadrature LB model HH(N1;Q1) x H(N2;Q2): force kernels and truncated
equilibrium (oracle; test infrastructure only).

* Model notation: Eq. (model), Sec. IV.B.  Axis 0 is the wall-normal axis.
* Weighted populations f_ij = w_i w_j f(p_i, p_j) / (omega(p_i) omega(p_j))
  (Sec. IV.B), so every moment is a plain sum over (i, j) (Eq. mom_quad).
* Force kernels (Sec. IV.C, App. D):
    K^H     Eq. (df_K_H),   K~^H    Eq. (dfp_K_H)    -- full range, Q x Q;
    K^hh    Eq. (df_K_hh),  K~^hh   Eq. (dfp_K_hh)   -- half range, 2Q x 2Q,
  with Phi^n_s(x) = sum_{l=s}^{n} h_{l,s} h_l(x) (Eq. Phi_def).
  Readings: in App. D's derivation of K^hh the Kronecker delta acts on s = l+1
  with coefficient 1/a_l, as in Eq. (df_K_hh) itself; the half-range expansion
  of f carries no 1/l! (the h_l are orthonormal).
* Truncated equilibrium (Sec. IV.D): f'_eq = n g_1 g_2, f''_eq = T f'_eq
  (Eq. feq_red), with g^H from Eq. (eq_gak_H) and g^hh from Eq. (eq_gak_hh)
  (erf, exp and the polynomials P_s^+, P_s^- and P_s^*).

Units: m = 1, k_B = 1.
"""
from __future__ import annotations

import functools
import math
import re
from decimal import Decimal, localcontext

import numpy as np

from . import quadrature as qd

SQRT2PI = math.sqrt(2.0 * math.pi)


def parse_model(s: str):
    """'HH(4;8)xH(4;20)' -> [('HH', 4, 8), ('H', 4, 20)] (Eq. model)."""
    parts = re.split(r"\s*[x×]\s*", s.strip())
    out = []
    for part in parts:
        m = re.fullmatch(r"(HH|H)\((\d+);(\d+)\)", part.replace(" ", ""))
        if not m:
            raise ValueError(f"bad model component {part!r}")
        kind, N, Q = m.group(1), int(m.group(2)), int(m.group(3))
        if not 0 <= N < Q:  # Eq. (norder_limit)
            raise ValueError("expansion order must satisfy 0 <= N < Q")
        out.append((kind, N, Q))
    if len(out) != 2:
        raise ValueError("two axes expected")
    return out


@functools.lru_cache(maxsize=None)
def _full_tables_dec(Q: int):
    """He_l(p_k) for l = 0..Q+1 and the weights, in Decimal."""
    _, _, roots, w = qd.full_range_rule(Q)
    H = qd.hermite_family(Q + 2)
    with localcontext() as ctx:
        ctx.prec = qd._digits(Q)
        He = [[qd._poly_eval(H[l], r) for r in roots] for l in range(Q + 2)]
    return He, w


@functools.lru_cache(maxsize=None)
def _full_tables(Q: int):
    """Float64 copy: nodes, weights, He_l(p_k)."""
    p, w, _, _ = qd.full_range_rule(Q)
    He, _ = _full_tables_dec(Q)
    return p, w, np.array([[float(v) for v in row] for row in He])


@functools.lru_cache(maxsize=None)
def _half_tables_dec(Q: int):
    """Decimal h_l(|p_k|) (l = 0..Q, k over the Q positive nodes), h_{l,0}, a_l, weights."""
    coeffs, _, _, _ = qd.half_range_family(Q)
    _, _, roots, w = qd.half_range_rule(Q)
    with localcontext() as ctx:
        ctx.prec = qd._digits(Q)
        hv = [[qd._poly_eval(coeffs[l], r) for r in roots] for l in range(Q + 1)]
        h0 = [coeffs[l][0] for l in range(Q + 1)]
        a = [coeffs[l + 1][l + 1] / coeffs[l][l] for l in range(Q)]
        Phi = [[[sum(coeffs[l][s] * hv[l][k] for l in range(s, n + 1)) if s <= n else Decimal(0)
                 for k in range(Q)] for s in range(Q + 1)] for n in range(Q + 1)]
    return hv, h0, a, w, Phi


@functools.lru_cache(maxsize=None)
def _half_tables(Q: int):
    """Float64 copies: nodes, weights, h_l(|p_k|), h_{l,0}, a_l, Phi^n_s(|p_k|) (Eq. Phi_def)."""
    p, w, _, _ = qd.half_range_rule(Q)
    hv, h0, a, _, Phi = _half_tables_dec(Q)
    f = np.vectorize(float)
    return p, w, f(np.array(hv, dtype=object)), f(np.array(h0, dtype=object)), \
        f(np.array(a, dtype=object)), f(np.array(Phi, dtype=object))


def _to_float(M):
    return np.array([[float(v) for v in row] for row in M])


@functools.lru_cache(maxsize=None)
def kernel_K_full(Q: int) -> np.ndarray:
    """Eq. (df_K_H): K_{k,k'} = -w_k sum_{l=0}^{Q-1} (1/l!) H_{l+1}(p_k) H_l(p_k')."""
    He, w = _full_tables_dec(Q)
    with localcontext() as ctx:
        ctx.prec = qd._digits(Q)
        fact = [Decimal(math.factorial(l)) for l in range(Q + 1)]
        K = [[-w[k] * sum(He[l + 1][k] * He[l][kp] / fact[l] for l in range(Q))
              for kp in range(Q)] for k in range(Q)]
    return _to_float(K)


@functools.lru_cache(maxsize=None)
def kernel_Kt_full(Q: int) -> np.ndarray:
    """Eq. (dfp_K_H): K~_{k,k'} = -w_k sum_{l=0}^{Q-2} (1/l!) H_{l+1}(p_k) [H_{l+1}(p_k') + l H_{l-1}(p_k')]."""
    He, w = _full_tables_dec(Q)
    with localcontext() as ctx:
        ctx.prec = qd._digits(Q)
        fact = [Decimal(math.factorial(l)) for l in range(Q + 1)]
        K = [[-w[k] * sum(He[l + 1][k] * (He[l + 1][kp] + (l * He[l - 1][kp] if l >= 1 else 0)) / fact[l]
                          for l in range(Q - 1))
              for kp in range(Q)] for k in range(Q)]
    return _to_float(K)


@functools.lru_cache(maxsize=None)
def kernel_K_half(Q: int) -> np.ndarray:
    """Eq. (df_K_hh), 2Q x 2Q.  Index k < Q is the positive node p_k, k >= Q its mirror -p_k."""
    hv, h0, a, w, Phi = _half_tables_dec(Q)
    n = 2 * Q
    with localcontext() as ctx:
        ctx.prec = qd._digits(Q)
        s2pi = (2 * qd.half_range_family(Q)[3]).sqrt()
        K = [[Decimal(0)] * n for _ in range(n)]
        for k in range(n):
            sk, ik = (1, k) if k < Q else (-1, k - Q)
            for kp in range(n):
                skp, ikp = (1, kp) if kp < Q else (-1, kp - Q)
                acc = Decimal(0)
                if sk == skp:  # (1 + sigma_k sigma_k') / 2
                    for l in range(Q - 1):
                        inner = h0[l] / s2pi * sum(h0[s] * hv[s][ik] for s in range(l + 1, Q))
                        inner -= hv[l + 1][ik] / a[l]  # h_{l,l} / h_{l+1,l+1} = 1 / a_l
                        acc += hv[l][ikp] * inner
                acc -= Phi[Q][0][ik] * Phi[Q][0][ikp] / (2 * s2pi)
                K[k][kp] = w[ik] * sk * acc
    return _to_float(K)


@functools.lru_cache(maxsize=None)
def kernel_Kt_half(Q: int) -> np.ndarray:
    """Eq. (dfp_K_hh), 2Q x 2Q, block diagonal in the sign of p (h_{-1} = h_{-2} = 0)."""
    hv, h0, a, w, Phi = _half_tables_dec(Q)
    n = 2 * Q
    with localcontext() as ctx:
        ctx.prec = qd._digits(Q)
        s2pi = (2 * qd.half_range_family(Q)[3]).sqrt()
        K = [[Decimal(0)] * n for _ in range(n)]
        for k in range(n):
            sk, ik = (1, k) if k < Q else (-1, k - Q)
            for kp in range(n):
                skp, ikp = (1, kp) if kp < Q else (-1, kp - Q)
                if sk != skp:
                    continue
                acc = Decimal(0)
                for l in range(Q):
                    term = l * hv[l][ikp]
                    if l >= 1:
                        term += (h0[l] ** 2 + h0[l - 1] ** 2) / (a[l - 1] * s2pi) * hv[l - 1][ikp]
                    if l >= 2:
                        term += hv[l - 2][ikp] / (a[l - 1] * a[l - 2])
                    acc += hv[l][ik] * term
                K[k][kp] = -w[ik] * acc
    return _to_float(K)


# ---------------------------------------------------------------- equilibrium

@functools.lru_cache(maxsize=None)
def _P_polys(S: int):
    """Integer coefficient lists of P_s^+, P_s^- (P_s^pm(x) = e^{-+x^2} d^s/dx^s e^{+-x^2})
    and P_s^* = sum_{j=0}^{s-1} C(s,j) P_j^+ P_{s-j-1}^- for s = 0..S (Sec. IV.D)."""
    def deriv(c):
        return [i * c[i] for i in range(1, len(c))] or [0]

    def add(a, b):
        n = max(len(a), len(b))
        return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]

    def mul(a, b):
        out = [0] * (len(a) + len(b) - 1)
        for i, x in enumerate(a):
            for j, y in enumerate(b):
                out[i + j] += x * y
        return out

    Pp, Pm = [[1]], [[1]]
    for s in range(S):
        # d/dx [e^{+-x^2} P] = e^{+-x^2} (P' +- 2x P)
        Pp.append(add(deriv(Pp[s]), [0] + [2 * c for c in Pp[s]]))
        Pm.append(add(deriv(Pm[s]), [0] + [-2 * c for c in Pm[s]]))
    Ps = []
    for s in range(S + 1):
        acc = [0]
        for j in range(s):
            acc = add(acc, [math.comb(s, j) * c for c in mul(Pp[j], Pm[s - j - 1])])
        Ps.append(acc)
    return Pp, Pm, Ps


def _peval(c, x):
    acc = np.zeros_like(x)
    for a in reversed(c):
        acc = acc * x + a
    return acc


class Model:
    """Tables of one model HH(N1;Q1) x H(N2;Q2) (either axis may be H or HH)."""

    def __init__(self, spec):
        if isinstance(spec, str):
            spec = parse_model(spec)
        self.spec = spec
        self.p, self.w, self.K, self.Kt = [], [], [], []
        for kind, N, Q in spec:
            p, w = qd.rule(kind, Q)
            self.p.append(p)
            self.w.append(w)
            if kind == "H":
                self.K.append(kernel_K_full(Q))
                self.Kt.append(kernel_Kt_full(Q))
            else:
                self.K.append(kernel_K_half(Q))
                self.Kt.append(kernel_Kt_half(Q))
        self.nq = [len(p) for p in self.p]

    def g_axis(self, a: int, u, T):
        """Equilibrium factor g_{a,k}(u, T) per cell: arrays u, T of shape (S,) -> (S, nq_a)."""
        kind, N, Q = self.spec[a]
        u = np.asarray(u, dtype=np.float64)[:, None]
        T = np.asarray(T, dtype=np.float64)[:, None]
        if kind == "H":  # Eq. (eq_gak_H)
            _, w, He = _full_tables(Q)
            g = np.zeros((u.shape[0], Q))
            for l in range(N + 1):
                c = sum((T - 1.0) ** s * u ** (l - 2 * s) / (2.0 ** s * math.factorial(s) * math.factorial(l - 2 * s))
                        for s in range(l // 2 + 1))
                g += He[l][None, :] * c
            return w[None, :] * g
        # Eq. (eq_gak_hh)
        p, w, h, h0, a_, Phi = _half_tables(Q)
        Pp, Pm, Ps = _P_polys(N)
        sig = np.concatenate([np.ones(Q), -np.ones(Q)])[None, :]
        idx = np.arange(2 * Q) % Q
        zeta = sig * u * np.sqrt(1.0 / (2.0 * T))
        erfz = np.vectorize(math.erf)(zeta)
        g = np.zeros((u.shape[0], 2 * Q))
        for s in range(N + 1):
            bracket = (1.0 + erfz) * _peval(Pp[s], zeta) + 2.0 / math.sqrt(math.pi) * np.exp(-zeta ** 2) * _peval(Ps[s], zeta)
            g += (T / 2.0) ** (s / 2.0) * Phi[N, s, idx][None, :] * bracket
        return 0.5 * w[None, :] * g

    def feq(self, n, u0, u1, T):
        """(f'_eq, f''_eq) of shape (S, nq0, nq1) each (Eq. feq_red)."""
        g0 = self.g_axis(0, u0, T)
        g1 = self.g_axis(1, u1, T)
        n = np.asarray(n, dtype=np.float64)
        f1 = n[:, None, None] * g0[:, :, None] * g1[:, None, :]
        return f1, np.asarray(T)[:, None, None] * f1

    def moments(self, F):
        """n, u^0, u^1, T of F with shape (2, S, nq0, nq1) (Eqs. macro_red, mom_quad; m = 1)."""
        f1, f2 = F[0], F[1]
        p0 = self.p[0][None, :, None]
        p1 = self.p[1][None, None, :]
        n = f1.sum(axis=(1, 2))
        u0 = (f1 * p0).sum(axis=(1, 2)) / n
        u1 = (f1 * p1).sum(axis=(1, 2)) / n
        xi2 = (p0 - u0[:, None, None]) ** 2 + (p1 - u1[:, None, None]) ** 2
        T = ((xi2 * f1).sum(axis=(1, 2)) + f2.sum(axis=(1, 2))) / (3.0 * n)
        return n, u0, u1, T

    def full_moments(self, F):
        """n, u^a, T, T^{ab} (00, 01, 11) and q^a per cell (Eqs. macro_red_Tab, macro_red_q)."""
        n, u0, u1, T = self.moments(F)
        f1, f2 = F[0], F[1]
        x0 = self.p[0][None, :, None] - u0[:, None, None]
        x1 = self.p[1][None, None, :] - u1[:, None, None]
        T00 = (x0 * x0 * f1).sum(axis=(1, 2))
        T01 = (x0 * x1 * f1).sum(axis=(1, 2))
        T11 = (x1 * x1 * f1).sum(axis=(1, 2))
        e = 0.5 * (x0 * x0 + x1 * x1) * f1 + 0.5 * f2
        q0 = (e * x0).sum(axis=(1, 2))
        q1 = (e * x1).sum(axis=(1, 2))
        return dict(n=n, u0=u0, u1=u1, T=T, T00=T00, T01=T01, T11=T11, q0=q0, q1=q1)
