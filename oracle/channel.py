"""Gradually expanding channel stage in the vielbein frame (oracle; test infrastructure only).

Sec. VII.A-B.  Coordinates lambda = x / (1 + phi(xi)), xi = y; the wall is at
lambda = H/2 = 1 and only the upper half 0 < lambda < 1 is simulated.
Momenta (p^lambda-hat, p^xi-hat) in the orthogonal triad of Eq. (canalie_phat):
half-range Gauss-Hermite on the wall-normal axis (index i), full range on the
tangential axis (index j).

Eq. (canalie_boltz) in the chi form, with V^lambda = a p^lambda,
a = sqrt(1 + lambda^2 phi'^2) / (1 + phi), and V^xi = b p^xi - c p^lambda,
b = (1 + phi) / sqrt(1 + lambda^2 phi'^2), c = lambda phi' b (Eq. canalie_V),
d chi^xi = (1 + phi) d xi (Eq. chi_canalie, closed form Eq. chi_canalie_exp):

  L[f] = -[a_{s+1/2} p^l F_{s+1/2} - a_{s-1/2} p^l F_{s-1/2}] / d lambda_s
         -[V^xi_{p+1/2} F_{p+1/2} - V^xi_{p-1/2} F_{p-1/2}] / d chi^xi_p
         + G_lxx [(p^xi)^2 K^l f - p^l K~^xi f] - G_lxl [(p^l)^2 K^xi f - p^xi K~^l f]
         - (f - f_eq) / tau,

with the discrete connection coefficients of Sec. VII.A (Gamma_{l x l} and
Gamma_{l x x} built from interface values so that f = const is an exact
solution) and tau = Kn / (n T) (Eq. canalie_tau).  The sign of the force
term follows from Eq. (boltz_noncons) with Gamma_{x l l} = -Gamma_{l x l}.

Boundaries:
* centreline lambda = 0: specular reflection, ghosts f_{1-k, i} = f_{k, ibar}
  with p_ibar = -p_i (Sec. VII.C.3);
* wall lambda = 1: diffuse reflection at rest and T_0, per-column n_w from the
  zero-mass-flux balance, outgoing ghosts by quadratic extrapolation
  (Sec. VII.C.4, Eqs. extrapol, weno_populate);
* inlet and outlet, two kinds:
  - particle reservoirs (the pressure-ratio workload): per (row, momentum),
    the populations entering the domain (V^xi > 0 at the inlet, V^xi < 0 at
    the outlet) see ghosts f_eq(n_res, (0, u_x), T_0), with u_x the u^xi of
    the adjacent cell; those leaving see ghosts equal to the adjacent cell
    (zeroth-order extrapolation, as the paper does for its inlet);
  - the paper's flow-rate profiles (Sec. VII.C.1-2, Eqs. canalie_inlet,
    canalie_outlet): the leaving populations as above; the entering ones see
    f_eq(n_s, (0, Q_s), T_0) with Q_s = 3 Q_0 (1 - lambda_s^2) / (H (1 + phi))
    at the end's xi (H = 2) and n_s fixed per row by the flux balance of
    Eq. (canalie_inlet_s): the particle flux through the end interface,
    entering part n_s f_eq(1, (0, Q_s), T_0) and leaving part the adjacent
    cell, equals Q_s.  The balance is taken with the chi-form velocity
    V^xi = (1 + phi) p^y of the interface, so the target is (1 + phi) Q_s
    (the same equation times 1 + phi).

Array layout: F has shape (2, N_lambda, N_xi, nq0, nq1).
"""
from __future__ import annotations

import math

import numpy as np

from .lbmodel import Model
from .weno import upwind_interfaces, weno5


def phi(xi, re_c=100.0):
    """Eq. (canalie_phi) with H = 2."""
    return 0.5 * (math.tanh(2.0) - np.tanh(2.0 - 30.0 * np.asarray(xi) / re_c))


def dphi(xi, re_c=100.0):
    return 0.5 * (30.0 / re_c) / np.cosh(2.0 - 30.0 * np.asarray(xi) / re_c) ** 2


def chi_xi(xi, re_c=100.0):
    """Eq. (chi_canalie_exp) with H = 2 (chi = 0 at xi = 0)."""
    xi = np.asarray(xi, dtype=np.float64)
    return (1.0 + math.tanh(2.0) / 2.0) * xi + re_c / 60.0 * np.log(np.cosh(2.0 - 30.0 * xi / re_c) / math.cosh(2.0))


class ChannelGrid:
    """N_lambda x N_xi cells; lambda(eta) = tanh(eta) / A (Eq. canalie_stretch, H/2 = 1),
    eta equidistant on [0, artanh A]; xi equidistant on [xi_in, xi_out]."""

    def __init__(self, n_lambda, n_xi, xi_in=-10.0, xi_out=40.0, re_c=100.0, A=0.95):
        self.nl, self.nx, self.re_c, self.A = n_lambda, n_xi, re_c, A
        ea = math.atanh(A)
        self.lf = np.tanh(np.arange(n_lambda + 1) / n_lambda * ea) / A  # interfaces lambda_{s+1/2}
        self.lf[-1] = 1.0
        self.lc = np.tanh((np.arange(1, n_lambda + 1) - 0.5) / n_lambda * ea) / A
        self.dl = self.lf[1:] - self.lf[:-1]
        self.xf = xi_in + (xi_out - xi_in) * np.arange(n_xi + 1) / n_xi
        self.xc = xi_in + (xi_out - xi_in) * (np.arange(1, n_xi + 1) - 0.5) / n_xi
        self.dchi = chi_xi(self.xf[1:], re_c) - chi_xi(self.xf[:-1], re_c)
        phc, dpc = phi(self.xc, re_c), dphi(self.xc, re_c)
        phf, dpf = phi(self.xf, re_c), dphi(self.xf, re_c)
        # lambda-interfaces (s+1/2, p): a = sqrt(1 + lambda^2 phi'^2) / (1 + phi), shape (nl+1, nx)
        self.a = np.sqrt(1.0 + self.lf[:, None] ** 2 * dpc[None, :] ** 2) / (1.0 + phc[None, :])
        # xi-interfaces (s, p+1/2): b, c, shape (nl, nx+1)
        root = np.sqrt(1.0 + self.lc[:, None] ** 2 * dpf[None, :] ** 2)
        self.b = (1.0 + phf[None, :]) / root
        self.c = self.lc[:, None] * dpf[None, :] * (1.0 + phf[None, :]) / root
        # discrete connection coefficients per cell (Sec. VII.A), shape (nl, nx)
        self.G_lxl = (self.b[:, 1:] - self.b[:, :-1]) / self.dchi[None, :]
        self.G_lxx = -(self.a[1:, :] - self.a[:-1, :]) / self.dl[:, None] + (self.c[:, 1:] - self.c[:, :-1]) / self.dchi[None, :]
        self.vol = self.dl[:, None] * self.dchi[None, :]


class ChannelOracle:
    def __init__(self, model, grid: ChannelGrid, kn, n_in=2.0, n_out=1.0, T0=1.0, q0=None, prandtl=None):
        self.m = model if isinstance(model, Model) else Model(model)
        self.g = grid
        self.kn, self.n_in, self.n_out, self.T0 = kn, n_in, n_out, T0
        self.q0 = q0  # None: reservoirs; else the half-channel flow rate Q_0 of the flow-rate profiles
        self.prandtl = prandtl  # None: BGK; else the Shakhov collision with this Pr
        self.last_inflow_density = None
        Q = self.m.spec[0][2]
        nq0 = self.m.nq[0]
        self.ibar = np.where(np.arange(nq0) < Q, np.arange(nq0) + Q, np.arange(nq0) - Q)
        self.last_nw = None

    def feq_cells(self, n, u0, u1, T):
        """f_eq per cell for arrays of any shape S -> (2,) + S + (nq0, nq1)."""
        shape = np.shape(n)
        f1, f2 = self.m.feq(np.ravel(n), np.ravel(u0), np.ravel(u1), np.ravel(T))
        return np.stack([f1, f2]).reshape((2,) + shape + f1.shape[1:])

    def initial_state(self, n_profile=None, T0=None):
        g = self.g
        T0 = self.T0 if T0 is None else T0
        if n_profile is None:
            x = (g.xc - g.xf[0]) / (g.xf[-1] - g.xf[0])
            n_profile = self.n_in + (self.n_out - self.n_in) * x
        n = np.broadcast_to(n_profile[None, :], (g.nl, g.nx))
        z = np.zeros((g.nl, g.nx))
        return self.feq_cells(n, z, z, np.full((g.nl, g.nx), T0))

    def flow_profile(self, end):
        """(Q_s, (1 + phi) Q_s) per row at the inlet (end 0) or outlet (end 1):
        Q_s = 3 Q_0 (1 - 4 lambda_s^2 / H^2) / (H (1 + phi(xi_end))), H = 2 (Eqs. canalie_inlet,
        canalie_outlet), lambda_s the row's cell centre, xi_end the end interface."""
        g = self.g
        xe = g.xf[0] if end == 0 else g.xf[-1]
        ph = float(phi(xe, g.re_c))
        H = 2.0
        q = 3.0 * self.q0 * (1.0 - 4.0 * g.lc ** 2 / H ** 2) / (H * (1.0 + ph))
        return q, (1.0 + ph) * q

    def moments(self, F):
        nl, nx = F.shape[1], F.shape[2]
        flat = F.reshape((2, nl * nx) + F.shape[3:])
        return tuple(x.reshape(nl, nx) for x in self.m.moments(flat))

    def L(self, F):
        m, g = self.m, self.g
        nl, nx = g.nl, g.nx
        pl, px = m.p[0], m.p[1]  # p^lambda-hat (half range), p^xi-hat (full range)
        PL = pl[:, None]
        PX = px[None, :]

        n, ul, ux, T = self.moments(F)
        Feq = self.feq_cells(n, ul, ux, T)
        tau = self.kn / (n * T)

        # ---- lambda direction: G[:, s+2, p] holds cell s (1-based), s = -2 .. nl+3
        Gl = np.zeros((2, nl + 6, nx) + F.shape[3:])
        Gl[:, 3:nl + 3] = F
        # centreline: specular, ghost 1-k mirrors cell k
        for k in (1, 2, 3):
            Gl[:, 3 - k] = F[:, k - 1][:, :, self.ibar, :]
        # wall: outgoing (p^lambda > 0) quadratic extrapolation, flux, n_w per column, incoming equilibrium
        pos = pl > 0
        FN, FN1, FN2 = F[:, nl - 1], F[:, nl - 2], F[:, nl - 3]
        e1 = 3 * FN - 3 * FN1 + FN2
        e2 = 6 * FN - 8 * FN1 + 3 * FN2
        flux_w = weno5(FN2, FN1, FN, e1, e2)  # (2, nx, nq0, nq1), valid for p^lambda > 0
        weq = self.feq_cells(np.ones(1), np.zeros(1), np.zeros(1), np.full(1, self.T0))[:, 0]
        den = (weq[0][~pos] * PL[~pos]).sum()
        num = (flux_w[0][:, pos] * PL[pos][None]).sum(axis=(1, 2))
        nw = -num / den  # (nx,)
        self.last_nw = nw
        for k, e in ((1, e1), (2, e2), (3, e2)):
            inc = nw[None, :, None, None] * weq[:, None]  # (2, nx, nq0, nq1)
            Gl[:, nl + 2 + k] = np.where(pos[None, None, :, None], e, inc)
        # interfaces s+1/2, s = 0..nl, between Gl[:, s+2] and Gl[:, s+3]
        Fl_ = upwind_interfaces(Gl, (pl >= 0)[None, None, None, :, None], axis=1)  # (2, nl+1, nx, nq0, nq1)
        fluxl = g.a[None, :, :, None, None] * PL[None, None, None] * Fl_
        adv = (fluxl[:, 1:] - fluxl[:, :-1]) / g.dl[None, :, None, None, None]

        # ---- xi direction: H[:, s, p+2] holds cell p (1-based), p = -2 .. nx+3
        Vx = g.b[:, :, None, None] * PX[None, None] - g.c[:, :, None, None] * PL[None, None]  # (nl, nx+1, nq0, nq1)
        Hx = np.zeros((2, nl, nx + 6) + F.shape[3:])
        Hx[:, :, 3:nx + 3] = F
        into_in = Vx[:, 0] > 0  # (nl, nq0, nq1)
        into_out = Vx[:, nx] < 0
        if self.q0 is None:
            f_in = self.feq_cells(np.full(nl, self.n_in), np.zeros(nl), ux[:, 0], np.full(nl, self.T0))  # (2, nl, nq0, nq1)
            f_out = self.feq_cells(np.full(nl, self.n_out), np.zeros(nl), ux[:, -1], np.full(nl, self.T0))
        else:
            ns = []
            fe = []
            for end, into, Fadj, V in ((0, into_in, F[0, :, 0], Vx[:, 0]), (1, into_out, F[0, :, nx - 1], Vx[:, nx])):
                q, target = self.flow_profile(end)
                e1 = self.feq_cells(np.ones(nl), np.zeros(nl), q, np.full(nl, self.T0))  # f_eq(1, (0, Q_s), T0)
                # Eq. (canalie_inlet_s): n_s sum_in V f'_eq(1) + sum_out V f'_adjacent = (1 + phi) Q_s
                leaving = np.where(into, 0.0, V * Fadj).sum(axis=(1, 2))
                entering = np.where(into, V * e1[0], 0.0).sum(axis=(1, 2))
                n_s = (target - leaving) / entering
                ns.append(n_s)
                fe.append(n_s[None, :, None, None] * e1)
            f_in, f_out = fe
            self.last_inflow_density = tuple(ns)
        for k in (0, 1, 2):
            Hx[:, :, k] = np.where(into_in[None], f_in, F[:, :, 0])
            Hx[:, :, nx + 3 + k] = np.where(into_out[None], f_out, F[:, :, nx - 1])
        Fx = upwind_interfaces(Hx, (Vx >= 0)[None], axis=2)  # (2, nl, nx+1, nq0, nq1)
        fluxx = Vx[None] * Fx
        adv = adv + (fluxx[:, :, 1:] - fluxx[:, :, :-1]) / g.dchi[None, None, :, None, None]

        # ---- inertial force with the discrete connection coefficients
        Kl, Ktl = m.K[0], m.Kt[0]
        Kx, Ktx = m.K[1], m.Kt[1]
        dl_f = np.einsum("ik,dspkj->dspij", Kl, F)    # d/dp^l f
        dlp_f = np.einsum("ik,dspkj->dspij", Ktl, F)  # d/dp^l (p^l f)
        dx_f = np.einsum("jk,dspik->dspij", Kx, F)    # d/dp^x f
        dxp_f = np.einsum("jk,dspik->dspij", Ktx, F)  # d/dp^x (p^x f)
        Glxx = g.G_lxx[None, :, :, None, None]
        Glxl = g.G_lxl[None, :, :, None, None]
        PLb, PXb = PL[None, None, None], PX[None, None, None]
        force = Glxx * (PXb ** 2 * dl_f - PLb * dxp_f) - Glxl * (PLb ** 2 * dx_f - PXb * dlp_f)

        coll = -(F - Feq) / tau[None, :, :, None, None]
        if self.prandtl is not None:  # Shakhov: the target gains (1 - Pr) times the heat-flux term
            from .couette import shakhov_term
            flat = F.reshape((2, nl * nx) + F.shape[3:])
            G = shakhov_term(m, flat).reshape(F.shape)
            coll = coll + (1.0 - self.prandtl) * G / tau[None, :, :, None, None]
        self.last_boundary_flux = dict(
            inlet=(g.dl[:, None, None] * fluxx[0, :, 0]).sum(), outlet=(g.dl[:, None, None] * fluxx[0, :, nx]).sum(),
            wall=(g.dchi[:, None, None] * fluxl[0, nl]).sum(), centre=(g.dchi[:, None, None] * fluxl[0, 0]).sum(),
            inlet_rows=fluxx[0, :, 0].sum(axis=(1, 2)), outlet_rows=fluxx[0, :, nx].sum(axis=(1, 2)))
        return -adv + force + coll

    def stage(self, k, dt, F_l, F_prev):
        Lp = self.L(F_prev)
        if k == 1:
            return F_l + dt * Lp
        if k == 2:
            return 0.75 * F_l + 0.25 * F_prev + 0.25 * dt * Lp
        return F_l / 3.0 + 2.0 / 3.0 * F_prev + 2.0 / 3.0 * dt * Lp

    def step(self, F, dt):
        F1 = self.stage(1, dt, F, F)
        F2 = self.stage(2, dt, F, F1)
        return self.stage(3, dt, F, F2)

    def n_tot(self, F):
        return float((self.g.vol * F[0].sum(axis=(2, 3))).sum())


def lambda_derivative(f, lam):
    """d f / d lambda on the non-equidistant row centres lam (axis 0 of f) with the paper's
    three-point formulas of Sec. VII.F: the bulk formula for 1 < s < N_lambda, the one-sided
    forward formula at the first node and the backward one at the last."""
    f = np.asarray(f, dtype=np.float64)
    d = np.empty_like(f)
    L = lam
    for s in range(1, len(L) - 1):
        lm, l0, lp = L[s - 1], L[s], L[s + 1]
        d[s] = ((l0 - lm) * f[s + 1] / ((lp - l0) * (lp - lm))
                + (lp - 2 * l0 + lm) * f[s] / ((lp - l0) * (l0 - lm))
                - (lp - l0) * f[s - 1] / ((lp - lm) * (l0 - lm)))
    l1, l2, l3 = L[0], L[1], L[2]
    d[0] = (-(l2 + l3 - 2 * l1) * f[0] / ((l2 - l1) * (l3 - l1))
            + (l3 - l1) * f[1] / ((l2 - l1) * (l3 - l2))
            - (l2 - l1) * f[2] / ((l3 - l1) * (l3 - l2)))
    lN, lN1, lN2 = L[-1], L[-2], L[-3]
    d[-1] = ((2 * lN - lN1 - lN2) * f[-1] / ((lN - lN1) * (lN - lN2))
             - (lN - lN2) * f[-2] / ((lN - lN1) * (lN1 - lN2))
             + (lN - lN1) * f[-3] / ((lN - lN2) * (lN1 - lN2)))
    return d


def xi_derivative(f, dxi):
    """d f / d xi on the equidistant columns (axis 1 of f): centred differences, the
    second-order forward formula at the inlet column and the backward one at the outlet."""
    f = np.asarray(f, dtype=np.float64)
    d = np.empty_like(f)
    d[:, 1:-1] = (f[:, 2:] - f[:, :-2]) / (2.0 * dxi)
    d[:, 0] = (-3.0 * f[:, 0] + 4.0 * f[:, 1] - f[:, 2]) / (2.0 * dxi)
    d[:, -1] = (3.0 * f[:, -1] - 4.0 * f[:, -2] + f[:, -3]) / (2.0 * dxi)
    return d


def postprocess(oracle: ChannelOracle, F):
    """Macroscopic fields of Sec. VII.D-F from the populations F (2, N_lambda, N_xi, nq0, nq1):
    * u^x, u^y, the Cartesian velocity of Eq. (canalie_u) from the triad components;
    * psi at the row interfaces lambda_{s+1/2} (N_lambda + 1 per column), Eq.
      (canalie_psi_sol): psi = 0 on the centreline, psi_{s+1/2} = psi_{s-1/2} -
      rho u^y (x_{s+1/2} - x_{s-1/2}) along each column, x = lambda (1 + phi(xi_p));
    * omega of Eq. (canalie_vorti) with the derivative formulas above;
    * P_w, the wall pressure per column: P = n T extrapolated linearly in x from the
      last two rows to the wall (Sec. VII.D; the ratio of x differences within a column
      is that of the lambda differences)."""
    g = oracle.g
    n, ul, ux_hat, T = oracle.moments(F)
    ph, dp = phi(g.xc, g.re_c)[None, :], dphi(g.xc, g.re_c)[None, :]
    lam = g.lc[:, None]
    root = np.sqrt(1.0 + lam ** 2 * dp ** 2)
    ux = (ul + lam * dp * ux_hat) / root
    uy = (ux_hat - lam * dp * ul) / root
    psi = np.zeros((g.nl + 1, g.nx))
    for s in range(g.nl):
        psi[s + 1] = psi[s] - n[s] * uy[s] * (g.lf[s + 1] - g.lf[s]) * (1.0 + ph[0])
    dxi = g.xc[1] - g.xc[0]
    omega = -xi_derivative(ux, dxi) + (lambda_derivative(uy, g.lc) + lam * dp * lambda_derivative(ux, g.lc)) / (1.0 + ph)
    P = n * T
    lw, l1, l2 = g.lf[-1], g.lc[-1], g.lc[-2]
    pw = ((lw - l2) * P[-1] - (lw - l1) * P[-2]) / (l1 - l2)
    return dict(ux=ux, uy=uy, psi=psi, omega=omega, pw=pw)


class ClbChannelOracle(ChannelOracle):
    """The Cartesian-split channel of Sec. VII.G (Eq. canalie_coord_beq_cons): momenta are the
    Cartesian (p^x, p^y) on the model's axes 0 and 1 (both usually half range), there is no
    force term, and the advection is

      L[f] = -[V^l_{s+1/2} F_{s+1/2} - V^l_{s-1/2} F_{s-1/2}] / d lambda_s
             -[V^x_{p+1/2} F_{p+1/2} - V^x_{p-1/2} F_{p-1/2}] / d chi^xi_p - (f - f_eq)/tau,

    V^lambda = (p^x - lambda phi' p^y) / (1 + phi) at (lambda_{s+1/2}, xi_p) and
    V^xi = (1 + phi) p^y at xi_{p+1/2}: each lambda interface of a column upwinds by the sign of
    a combination of p^x and p^y, so the wall's incoming half-plane V^lambda < 0 depends on
    the column (Eq. canalie_coord_nw).  Boundaries as in ChannelOracle: the centreline mirrors
    p^x, the wall is diffuse at rest and T_0 (outgoing half extrapolated, n_w per column),
    the reservoirs at the ends fill the populations entering (p^y > 0 at the inlet, < 0 at the
    outlet) with f_eq(n_res, (0, u^y of the adjacent cell), T_0)."""

    def __init__(self, model, grid: ChannelGrid, kn, n_in=2.0, n_out=1.0, T0=1.0, prandtl=None):
        super().__init__(model, grid, kn, n_in=n_in, n_out=n_out, T0=T0, prandtl=prandtl)
        g = grid
        phc, dpc = phi(g.xc, g.re_c), dphi(g.xc, g.re_c)
        self.Vl_a = 1.0 / (1.0 + phc)                     # V^l = a (p^x - lambda_f phi' p^y)
        self.Vl_b = g.lf[:, None] * dpc[None, :]          # lambda_{s+1/2} phi'(xi_p), (nl+1, nx)
        self.Vx = 1.0 + phi(g.xf, g.re_c)                 # V^xi / p^y at xi_{p+1/2}, (nx+1,)

    def L(self, F):
        m, g = self.m, self.g
        nl, nx = g.nl, g.nx
        px, py = m.p[0], m.p[1]
        PX, PY = px[:, None], py[None, :]
        n, ux, uy, T = self.moments(F)
        Feq = self.feq_cells(n, ux, uy, T)
        tau = self.kn / (n * T)

        # ---- lambda: V^l (nl+1, nx, nq0, nq1) at the row interfaces of each column
        Vl = self.Vl_a[None, :, None, None] * (PX[None, None] - self.Vl_b[:, :, None, None] * PY[None, None])
        Gl = np.zeros((2, nl + 6, nx) + F.shape[3:])
        Gl[:, 3:nl + 3] = F
        for k in (1, 2, 3):  # centreline: specular in p^x
            Gl[:, 3 - k] = F[:, k - 1][:, :, self.ibar, :]
        out = Vl[nl] > 0  # (nx, nq0, nq1): leaving through the wall
        FN, FN1, FN2 = F[:, nl - 1], F[:, nl - 2], F[:, nl - 3]
        e1 = 3 * FN - 3 * FN1 + FN2
        e2 = 6 * FN - 8 * FN1 + 3 * FN2
        flux_w = np.where(out[None], weno5(FN2, FN1, FN, e1, e2), 0.0)  # the WENO value of the leaving half
        weq = self.feq_cells(np.ones(1), np.zeros(1), np.zeros(1), np.full(1, self.T0))[:, 0]  # (2, nq0, nq1)
        num = (flux_w[0] * Vl[nl]).sum(axis=(1, 2))
        den = np.where(~out, weq[0][None] * Vl[nl], 0.0).sum(axis=(1, 2))
        nw = -num / den  # Eq. (canalie_coord_nw), per column
        self.last_nw = nw
        for k, e in ((1, e1), (2, e2), (3, e2)):
            inc = nw[None, :, None, None] * weq[:, None]
            Gl[:, nl + 2 + k] = np.where(out[None], e, inc)
        Fl_ = upwind_interfaces(Gl, (Vl >= 0)[None], axis=1)
        fluxl = Vl[None] * Fl_
        adv = (fluxl[:, 1:] - fluxl[:, :-1]) / g.dl[None, :, None, None, None]

        # ---- xi: V^xi = (1 + phi) p^y at the column interfaces
        Vx = self.Vx[None, :, None, None] * PY[None, None] * np.ones((nl, 1, len(px), 1))  # (nl, nx+1, nq0, nq1)
        Hx = np.zeros((2, nl, nx + 6) + F.shape[3:])
        Hx[:, :, 3:nx + 3] = F
        f_in = self.feq_cells(np.full(nl, self.n_in), np.zeros(nl), uy[:, 0], np.full(nl, self.T0))
        f_out = self.feq_cells(np.full(nl, self.n_out), np.zeros(nl), uy[:, -1], np.full(nl, self.T0))
        into_in, into_out = Vx[:, 0] > 0, Vx[:, nx] < 0
        for k in (0, 1, 2):
            Hx[:, :, k] = np.where(into_in[None], f_in, F[:, :, 0])
            Hx[:, :, nx + 3 + k] = np.where(into_out[None], f_out, F[:, :, nx - 1])
        Fx = upwind_interfaces(Hx, (Vx >= 0)[None], axis=2)
        fluxx = Vx[None] * Fx
        adv = adv + (fluxx[:, :, 1:] - fluxx[:, :, :-1]) / g.dchi[None, None, :, None, None]
        self.last_boundary_flux = dict(
            inlet=(g.dl[:, None, None] * fluxx[0, :, 0]).sum(), outlet=(g.dl[:, None, None] * fluxx[0, :, nx]).sum(),
            wall=(g.dchi[:, None, None] * fluxl[0, nl]).sum(), centre=(g.dchi[:, None, None] * fluxl[0, 0]).sum())
        coll = -(F - Feq) / tau[None, :, :, None, None]
        if self.prandtl is not None:  # Shakhov, as in the vielbein channel: (1 - Pr) G of the cell's own q
            from .couette import shakhov_term
            flat = F.reshape((2, nl * nx) + F.shape[3:])
            coll = coll + (1.0 - self.prandtl) * shakhov_term(m, flat).reshape(F.shape) / tau[None, :, :, None, None]
        return -adv + coll
