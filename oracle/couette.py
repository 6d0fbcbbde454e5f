"""Chi-formulation circular Couette stage (oracle; test infrastructure only).

The stage operator L[F] of Eq. (L_def) for Eq. (boltz_couette_kom) (and its
stretched form, Eq. boltz_couette_str_kom), followed step by step:

1. moments n, u^R, u^phi, T of f', f'' (Eqs. macro_red, mom_quad);
2. truncated equilibrium f'_eq = n g_R g_phi, f''_eq = T f'_eq (Eq. feq_red)
   and the relaxation time (Eq. hydro_tau, Eq. tau_aoki, or Kn/n);
3. diffuse-reflection walls (Sec. III.E): outgoing ghosts by quadratic
   extrapolation (Eq. extrapol), the WENO-5 wall flux for the outgoing half,
   n_w from the zero-mass-flux balance (Eq. nw), then incoming ghosts
   F_{-2} = F_{-1} = F_0 = f_eq(n_w, u_w, T_w) (Eq. weno_populate), with
   f''-ghosts T_w times the f'-ghosts;
4. WENO-5 interface values on every interface (Sec. III.C) and the chi flux
   difference 2 p^R (R_{s+1/2} F_{s+1/2} - R_{s-1/2} F_{s-1/2}) /
   (R_{s+1/2}^2 - R_{s-1/2}^2) (Eqs. flux_kom_R, flux_kom_eta);
5. the inertial force (1/R)[(p^phi)^2 d_{p^R} f - p^R d_{p^phi}(p^phi f)],
   with the momentum derivatives as K and K~ contractions (Sec. IV.C);
6. BGK relaxation -(F - F_eq)/tau (Eq. BGK), or, with a Prandtl number given, the
   Shakhov collision the paper names as the extension of BGK (Sec. II.C):
   -(F - F_eq - (1 - Pr) G)/tau, G the heat-flux part of Grad's form for the
   cell's own q, projected on the model basis (oracle.seeding).

L = -(advection) - (force) - (F - F_eq)/tau; TVD-RK3 per Eq. (rk3).

Readings where the paper is silent: the outer wall mirrors the inner one;
within a stage n_w is computed from the same F as the fluxes; on a stretched
grid the 1/R of the force term is 2/(R_{s+1/2} + R_{s-1/2}), which equals the
factor the chi flux difference produces for a constant F, so that the rest
state of Sec. VI.C.2 stays exact (on the equidistant grid it is R_s itself).

Array layout: F has shape (2, N_R, nq0, nq1): field (f', f''), cell, radial
momentum index i, azimuthal momentum index j.

Radial slabs (domain decomposition): a grid made by CouetteGrid.slab holds a
contiguous range of the cells; at an end that is not a wall, step 3 takes the
three ghost cells from the neighbouring slab (set_halo) and the rest of the
stage is unchanged, so every cell gets what the whole grid gives it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .lbmodel import Model
from .weno import upwind_interfaces, weno5

TAU_KN_OVER_NT, TAU_AOKI, TAU_KN_OVER_N = 0, 1, 2


@dataclass
class Wall:
    u_tangential: float = 0.0  # u^phi of the wall (Omega R)
    T: float = 1.0


class CouetteGrid:
    """Radial grid between R_in and R_out, equidistant (A = 0) or tanh-stretched
    (Eq. eta_def with parameters A, delta; cell centres equidistant in eta)."""

    def __init__(self, n: int, r_in: float = 1.0, r_out: float = 2.0, A: float = 0.0, delta: float = 0.5):
        if n < 3:
            raise ValueError("at least three cells are needed for the wall extrapolation")
        self.n, self.r_in, self.r_out, self.A, self.delta = n, r_in, r_out, A, delta
        s = np.arange(n + 1)
        if A == 0.0:
            self.Rf = r_in + (r_out - r_in) * s / n
            self.Rc = r_in + (np.arange(1, n + 1) - 0.5) / n * (r_out - r_in)
            self.wres = self.Rc * (r_out - r_in) / n
        else:
            A0 = max(delta, 1.0 - delta)
            eta_in = -math.atanh(A * delta / A0)
            eta_out = math.atanh(A * (1.0 - delta) / A0)
            deta = (eta_out - eta_in) / n
            R = lambda eta: r_in + (r_out - r_in) * (delta + A0 / A * np.tanh(eta))
            eta_f = eta_in + s * deta
            eta_c = eta_in + (np.arange(1, n + 1) - 0.5) * deta
            self.Rf = R(eta_f)
            self.Rf[0], self.Rf[-1] = r_in, r_out
            self.Rc = R(eta_c)
            # rectangle rule in eta for int dR R (.) (steady-state norms, Sec. VI.G)
            self.wres = A0 / A * (r_out - r_in) * self.Rc * deta / np.cosh(eta_c) ** 2
        self.dchi = 0.5 * (self.Rf[1:] ** 2 - self.Rf[:-1] ** 2)
        self.Rbar = 0.5 * (self.Rf[1:] + self.Rf[:-1])
        self.n_total, self.cell_begin = n, 0  # a whole grid: both ends are walls
        # the f~ formulation (Eqs. boltz_couette_cons, boltz_couette_str_cons): the advected
        # F~ = sqrt(g) f, its flux p e F~ differenced over d eta (equidistant: e = 1, d eta = dR)
        if A == 0.0:
            self.sqrtg = self.Rc.copy()
            self.e_f = np.ones(n + 1)
            self.deta = (r_out - r_in) / n
        else:
            self.sqrtg = A0 * (r_out - r_in) * self.Rc / (A * np.cosh(eta_c) ** 2)
            self.e_f = A * np.cosh(eta_f) ** 2 / (A0 * (r_out - r_in))
            self.deta = deta

    def slab(self, begin: int, end: int) -> "CouetteGrid":
        """Cells [begin, end) of this grid with their own geometry: a radial slab of a
        domain decomposition.  An end inside the grid has no wall; the oracle takes its
        three ghost cells from the neighbouring slab (CouetteOracle.set_halo)."""
        if not (0 <= begin and end <= self.n and end - begin >= 3):
            raise ValueError("a slab needs at least three cells of the grid")
        g = object.__new__(CouetteGrid)
        g.n, g.r_in, g.r_out, g.A, g.delta = end - begin, self.r_in, self.r_out, self.A, self.delta
        g.Rf = self.Rf[begin:end + 1].copy()
        for name in ("Rc", "wres", "dchi", "Rbar", "sqrtg"):
            setattr(g, name, getattr(self, name)[begin:end].copy())
        g.e_f, g.deta = self.e_f[begin:end + 1].copy(), self.deta
        g.n_total, g.cell_begin = self.n, begin
        return g

    @property
    def inner_is_wall(self) -> bool:
        return self.cell_begin == 0

    @property
    def outer_is_wall(self) -> bool:
        return self.cell_begin + self.n == self.n_total


def shakhov_term(model: Model, F):
    """The heat-flux term G[F] of the Shakhov target f_eq + (1 - Pr) G (oracle.seeding.heat_flux_term)
    for the moments n, u, T, q of F, shape (2, S, nq0, nq1) like F."""
    from .seeding import heat_flux_term
    mom = model.full_moments(F)
    g1, g2 = heat_flux_term(model, mom["n"], mom["u0"], mom["u1"], mom["T"], mom["q0"], mom["q1"])
    return np.stack([g1, g2])


def relaxation_time(kn, n, T, mode):
    if mode == TAU_KN_OVER_NT:
        return kn / (n * T)
    if mode == TAU_AOKI:
        return math.sqrt(math.pi / 8.0) * kn / n
    if mode == TAU_KN_OVER_N:
        return kn / n
    raise ValueError(mode)


class CouetteOracle:
    def __init__(self, model, grid: CouetteGrid, inner: Wall, outer: Wall, kn: float, tau_mode: int = TAU_AOKI,
                 prandtl=None, formulation: str = "chi"):
        self.m = model if isinstance(model, Model) else Model(model)
        self.g = grid
        self.inner, self.outer = inner, outer
        self.kn, self.tau_mode = kn, tau_mode
        self.prandtl = prandtl  # None: BGK (Eq. BGK); else the Shakhov collision with this Pr
        if formulation not in ("chi", "ftilde"):
            raise ValueError(formulation)
        self.formulation = formulation  # "chi" (Eq. boltz_couette_kom) or "ftilde" (Eq. boltz_couette_cons)
        self.last_nw = (float("nan"), float("nan"))
        self.halo = [None, None]  # ghost cells of slab ends (set_halo)

    def set_halo(self, lo=None, hi=None):
        """Ghost cells of the ends of a slab grid that are not walls, shape (2, 3, nq0, nq1)
        each, in increasing radius: the three cells below the slab (lo) and above it (hi),
        taken from the neighbouring slabs' current stage input."""
        self.halo = [None if lo is None else np.asarray(lo, dtype=np.float64),
                     None if hi is None else np.asarray(hi, dtype=np.float64)]

    # -- equilibrium of a wall, shape (2, nq0, nq1)
    def _wall_feq(self, n, wall: Wall):
        f1, f2 = self.m.feq(np.array([n]), np.array([0.0]), np.array([wall.u_tangential]), np.array([wall.T]))
        return np.stack([f1[0], f2[0]])

    def initial_equilibrium(self, n0=1.0, u0=0.0, u1=0.0, T0=1.0):
        N = self.g.n
        f1, f2 = self.m.feq(np.full(N, n0), np.full(N, u0), np.full(N, u1), np.full(N, T0))
        return np.stack([f1, f2])

    def L(self, F):
        m, g = self.m, self.g
        N = g.n
        p0 = m.p[0]
        p1 = m.p[1]

        # 1-2: moments, equilibrium, relaxation time
        n, u0, u1, T = m.moments(F)
        f1eq, f2eq = m.feq(n, u0, u1, T)
        Feq = np.stack([f1eq, f2eq])
        tau = relaxation_time(self.kn, n, T, self.tau_mode)

        # 3: ghosts; G[:, s + 2] holds cell s (s = -2 .. N + 3).  In the f~ formulation the
        # advected quantity is F~ = sqrt(g) f and the walls act on it (Sec. III.E: the sqrt(g)
        # of the incoming half is absorbed into n_w, the outgoing half is extrapolated in F~)
        ft = self.formulation == "ftilde"
        A = g.sqrtg[None, :, None, None] * F if ft else F
        G = np.zeros((2, N + 6) + F.shape[2:])
        G[:, 3:N + 3] = A
        nw_in = nw_out = 0.0
        if g.inner_is_wall:
            nw_in = self._inner_wall(A, G)
        else:  # a slab end inside the grid: the neighbour's cells
            G[:, 0:3] = self.halo[0]
        if g.outer_is_wall:
            nw_out = self._outer_wall(A, G)
        else:
            G[:, N + 3:N + 6] = self.halo[1]
        self.last_nw = (nw_in, nw_out)

        # 4: advection; f~: p (e_{s+1/2} F~_{s+1/2} - e_{s-1/2} F~_{s-1/2}) / d eta (Eqs. flux_cons_R,
        # flux_cons_eta), divided by sqrt(g_s) to act on f
        adv = self.advection_tilde(G) if ft else self.advection(G)

        # 5: inertial force, (1/R)[(p^phi)^2 K^R f - p^R K~^phi f]: R = 2 / (R_{s+1/2} + R_{s-1/2})
        # in the chi formulation (reading that keeps the rest state exact), the cell centre R_s in
        # the f~ formulation (as printed)
        dfdpR = np.einsum("ik,dskj->dsij", m.K[0], F)
        dpfdpphi = np.einsum("jk,dsik->dsij", m.Kt[1], F)
        Rf = g.Rc if ft else g.Rbar
        force = (p1[None, None, None, :] ** 2 * dfdpR - p0[None, None, :, None] * dpfdpphi) / Rf[None, :, None, None]

        # 6: BGK, or Shakhov: the target gains (1 - Pr) times the heat-flux term of the cell's q
        coll = -(F - Feq) / tau[None, :, None, None]
        if self.prandtl is not None:
            coll = coll + (1.0 - self.prandtl) * shakhov_term(m, F) / tau[None, :, None, None]
        return -adv - force + coll

    def _inner_wall(self, F, G):
        """Ghost cells -3 .. -1 of the inner wall (step 3) written into G; returns n_w."""
        p0 = self.m.p[0]
        pos, neg = p0 > 0, p0 < 0
        # inner wall: outgoing (p^R < 0) ghosts by quadratic extrapolation
        F1, F2, F3 = F[:, 0], F[:, 1], F[:, 2]
        G[:, 2][:, neg] = (3 * F1 - 3 * F2 + F3)[:, neg]
        G[:, 1][:, neg] = (6 * F1 - 8 * F2 + 3 * F3)[:, neg]
        flux_in = weno5(G[:, 5], G[:, 4], G[:, 3], G[:, 2], G[:, 1])  # mirror stencil at s = 1/2
        feq1 = self._wall_feq(1.0, self.inner)
        num = -(flux_in[0][neg] * p0[neg, None]).sum()
        den = (feq1[0][pos] * p0[pos, None]).sum()
        nw_in = num / den
        ghost = nw_in * feq1
        for k in (0, 1, 2):
            G[:, k][:, pos] = ghost[:, pos]
        return nw_in

    def _outer_wall(self, F, G):
        """Ghost cells N .. N+2 of the outer wall (step 3) written into G; returns n_w."""
        p0 = self.m.p[0]
        pos, neg = p0 > 0, p0 < 0
        N = F.shape[1]
        # outer wall: outgoing (p^R > 0) ghosts, mirrored
        FN, FN1, FN2 = F[:, N - 1], F[:, N - 2], F[:, N - 3]
        G[:, N + 3][:, pos] = (3 * FN - 3 * FN1 + FN2)[:, pos]
        G[:, N + 4][:, pos] = (6 * FN - 8 * FN1 + 3 * FN2)[:, pos]
        flux_out = weno5(G[:, N], G[:, N + 1], G[:, N + 2], G[:, N + 3], G[:, N + 4])
        feq1o = self._wall_feq(1.0, self.outer)
        num = -(flux_out[0][pos] * p0[pos, None]).sum()
        den = (feq1o[0][neg] * p0[neg, None]).sum()
        nw_out = num / den
        ghost = nw_out * feq1o
        for k in (N + 3, N + 4, N + 5):
            G[:, k][:, neg] = ghost[:, neg]
        return nw_out

    def advection(self, G):
        """chi-form flux difference p^R (R_{s+1/2} F_{s+1/2} - R_{s-1/2} F_{s-1/2}) / d chi_s
        (Eqs. flux_kom_R, flux_kom_eta; d chi = R dR) of the ghosted populations G, shape
        (2, N + 6, nq0, nq1) with G[:, s + 2] holding cell s (s = -2 .. N + 3), from the
        WENO-5 interface values of the upwind side of each velocity."""
        p0 = self.m.p[0]
        Fl = upwind_interfaces(G, (p0 >= 0)[None, None, :, None], axis=1)  # (2, N+1, nq0, nq1)
        RF = self.g.Rf[None, :, None, None] * Fl
        return p0[None, None, :, None] * (RF[:, 1:] - RF[:, :-1]) / self.g.dchi[None, :, None, None]

    def advection_tilde(self, G):
        """f~ formulation: p (e_{s+1/2} F~_{s+1/2} - e_{s-1/2} F~_{s-1/2}) / (d eta sqrt(g_s)) of the
        ghosted G = F~ (Eqs. flux_cons_R, flux_cons_eta), the WENO-5 interface values of F~ on
        the upwind side; divided by sqrt(g_s) it is the advection of f."""
        p0 = self.m.p[0]
        Fl = upwind_interfaces(G, (p0 >= 0)[None, None, :, None], axis=1)
        flux = self.g.e_f[None, :, None, None] * Fl
        return p0[None, None, :, None] * (flux[:, 1:] - flux[:, :-1]) / (self.g.deta * self.g.sqrtg[None, :, None, None])

    def stage(self, k: int, dt: float, F_l, F_prev):
        """One TVD-RK3 stage, Eq. (rk3): k = 1, 2, 3 with F_prev = F_l, F^(1), F^(2)."""
        Lp = self.L(F_prev)
        if k == 1:
            return F_l + dt * Lp
        if k == 2:
            return 0.75 * F_l + 0.25 * F_prev + 0.25 * dt * Lp
        if k == 3:
            return F_l / 3.0 + 2.0 / 3.0 * F_prev + 2.0 / 3.0 * dt * Lp
        raise ValueError(k)

    def step(self, F, dt: float):
        F1 = self.stage(1, dt, F, F)
        F2 = self.stage(2, dt, F, F1)
        return self.stage(3, dt, F, F2)

    def n_tot(self, F):
        """Particle number per unit height divided by 2 pi: sum_s dchi_s sum_ij f'_{s,ij} (Eq. Ntot_def)."""
        return float((self.g.dchi * F[0].sum(axis=(1, 2))).sum())

    def n_tot_ftilde(self, F):
        """The particle number the f~ scheme conserves: sum_s d eta sqrt(g_s) sum_ij f'_{s,ij}
        (its flux difference telescopes over d eta)."""
        return float((self.g.deta * self.g.sqrtg * F[0].sum(axis=(1, 2))).sum())

    def residual(self, mom_now, mom_prev, u_w):
        """L2 norms of Eq. (msites_steady) between two successive checks."""
        n1, _, ph1, T1 = mom_now
        n0, _, ph0, T0 = mom_prev
        w = self.g.wres
        l2u = math.sqrt((w * ((ph1 - ph0) / u_w) ** 2).sum())
        l2n = math.sqrt((w * (n1 / n0 - 1.0) ** 2).sum())
        l2T = math.sqrt((w * (T1 / T0 - 1.0) ** 2).sum())
        return l2u, l2n, l2T
