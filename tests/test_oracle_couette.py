"""Pins of the oracle's chi-formulation Couette stage (Secs. III, VI)."""
import math

import numpy as np
import pytest

from oracle import analytic as an
from oracle.couette import TAU_AOKI, TAU_KN_OVER_N, TAU_KN_OVER_NT, CouetteGrid, CouetteOracle, Wall
from paper_1708_05944_gb300.inputs import perturbation


@pytest.mark.parametrize("spec", ["HH(3;4)xH(3;4)", "HH(4;8)xH(4;20)", "H(4;5)xH(4;5)", "HH(2;3)xH(2;3)"])
@pytest.mark.parametrize("A", [0.0, 0.95])
def test_rest_state_is_exact(spec, A):
    # cylinders at rest, f = f_eq(1, 0, T_w): L[f] = 0 (Sec. VI.C.2)
    o = CouetteOracle(spec, CouetteGrid(16, A=A), Wall(0.0), Wall(0.0), 0.05, TAU_KN_OVER_N)
    F = o.initial_equilibrium()
    assert np.abs(o.L(F)).max() < 1e-13
    assert o.last_nw[0] == pytest.approx(1.0, abs=1e-14) and o.last_nw[1] == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("A", [0.0, 0.95])
def test_mass_is_conserved_with_diffuse_walls(A):
    # only wall fluxes change N_tot, and n_w cancels them (Sec. III.D, Eq. nw)
    o = CouetteOracle("HH(3;4)xH(3;4)", CouetteGrid(24, A=A), Wall(0.2), Wall(-0.1), 0.1, TAU_AOKI)
    F = o.initial_equilibrium() * perturbation((2, 24, 8, 4), seed=3, amplitude=0.02)
    N0 = o.n_tot(F)
    for _ in range(60):
        F = o.step(F, 2e-3)
    assert abs(o.n_tot(F) / N0 - 1.0) < 1e-13


def test_wall_flux_vanishes():
    # with n_w from Eq. (nw) the wall mass flux is zero: check through dN/dt of one L
    o = CouetteOracle("HH(4;8)xH(4;20)", CouetteGrid(12), Wall(0.3), Wall(0.0), 0.3, TAU_KN_OVER_NT)
    F = o.initial_equilibrium() * perturbation((2, 12, 16, 20), seed=5)
    L = o.L(F)
    assert abs((o.g.dchi * L[0].sum(axis=(1, 2))).sum()) < 1e-13


@pytest.mark.slow
def test_rigid_rotation_is_held():
    # f = f_eq(n(R), Omega R, T_w) with Eq. (rigid_density) solves the kinetic equation for all tau
    # (Sec. VI.C.3); the scheme keeps it up to velocity truncation and O(dR^2)
    Om, N = 0.3, 32
    g = CouetteGrid(N)
    o = CouetteOracle("H(4;5)xH(4;5)", g, Wall(Om * 1.0), Wall(Om * 2.0), 0.1, TAU_KN_OVER_N)
    n = an.rigid_density(g.Rc, Om, 1.0, 1.0, 2.0)
    f1, f2 = o.m.feq(n, np.zeros(N), Om * g.Rc, np.ones(N))
    F = np.stack([f1, f2])
    dt = 0.4 / N / 4
    for _ in range(int(2.0 / dt)):
        F = o.step(F, dt)
    nn, u0, u1, T = o.m.moments(F)
    assert np.abs(nn / n - 1).max() < 2e-3
    assert np.abs(u1 / (Om * g.Rc) - 1).max() < 3e-3
    assert np.abs(T - 1).max() < 2e-3


def test_navier_stokes_closed_forms_are_consistent():
    # the printed NS profiles satisfy their defining relations (Sec. VI.D.1)
    ri, ro, Om, mu, Tw = 1.0, 2.0, 0.5, 1e-3, 1.0
    kappa = 2.5 * mu  # Eq. (CE_tcoeff), m = 1
    R = np.linspace(ri, ro, 2001)
    u = an.ns_u_phi(R, Om, ri, ro)
    assert u[0] == pytest.approx(Om * ri, abs=1e-14) and u[-1] == pytest.approx(0.0, abs=1e-14)
    # T^{R phi} = -mu R d/dR (u/R) (Eq. NS_TRph_aux)
    Trp = -mu * R * np.gradient(u / R, R, edge_order=2)
    np.testing.assert_allclose(Trp, an.ns_T_Rphi(R, mu, Om, ri, ro), rtol=1e-5)
    T = an.ns_T(R, mu / kappa, Om, Tw, ri, ro)
    assert T[0] == pytest.approx(Tw, abs=1e-14) and T[-1] == pytest.approx(Tw, abs=1e-14)
    qR = an.ns_qR(R, mu, Om, ri, ro)
    np.testing.assert_allclose(qR, -kappa * np.gradient(T, R, edge_order=2), rtol=0, atol=1e-5 * np.abs(qR).max())
    # q^R + u^phi T^{R phi} = Q / R (Eq. Q_def)
    np.testing.assert_allclose(R * (qR + u * an.ns_T_Rphi(R, mu, Om, ri, ro)), an.ns_Q(mu, Om, ri, ro), rtol=1e-12)
    # temperature maximum (Eq. NS_Rmax)
    assert R[np.argmax(T)] == pytest.approx(an.ns_R_Tmax(ri, ro), abs=1e-3)


def test_rigid_density_normalisation():
    ri, ro, Om = 1.0, 2.0, 0.7
    R = np.linspace(ri, ro, 20001)
    n = an.rigid_density(R, Om, 1.0, ri, ro)
    total = 2 * math.pi * np.trapezoid(n * R, R)
    assert total == pytest.approx(math.pi * (ro ** 2 - ri ** 2), rel=1e-8)


def test_steady_state_near_the_navier_stokes_limit():
    """Sec. VI.D.1 at Kn = 0.02 (tau = Kn / (n T), so mu = Kn), 32 cells, steady
    after about 30 time units (viscous time 1 / (pi^2 Kn)):
    * the azimuthal velocity is the no-slip Navier-Stokes profile A R + B / R
      (Eq. NS_U) up to the velocity slip at the walls, first order in Kn
      (6 % of u_w here; 3 % at Kn = 0.01);
    * the angular-momentum flux R^2 T^{R phi} is the same at every radius (Eq.
      TRph), and equals the Navier-Stokes torque (Eq. NS_TRph) reduced by the slip
      (0.92 of it here);
    * the energy flux R (q^R + u^phi T^{R phi}) is the same at every radius (Eq.
      Q_def) and 0.92 of its Navier-Stokes value (Eq. NS_Q); the viscous heating
      raises T as Eq. (NS_T) with mu / kappa = 2/5 (peak within 2 %), with the
      maximum one cell from Eq. (NS_Rmax).
    The fluxes pin the force term: with its sign flipped their spreads are 130 % and
    3400 % and the peak temperature rise a fifth of the NS one, while the velocity
    profile alone hardly changes."""
    o = CouetteOracle("HH(3;4)xH(3;4)", CouetteGrid(32), Wall(0.1), Wall(0.0), 0.02, TAU_KN_OVER_NT)
    F = o.initial_equilibrium()
    for _ in range(7500):
        F = o.step(F, 4e-3)
    R = o.g.Rc
    mom = o.m.full_moments(F)
    assert np.abs(mom["u1"] - an.ns_u_phi(R, 0.1, 1.0, 2.0)).max() / 0.1 < 0.08
    flux = R ** 2 * mom["T01"]
    assert (flux.max() - flux.min()) / abs(flux.mean()) < 0.10
    torque = float((R ** 2 * an.ns_T_Rphi(R, 0.02, 0.1, 1.0, 2.0)).mean())
    assert abs(flux.mean() / torque - 1.0) < 0.15
    energy = R * (mom["q0"] + mom["u1"] * mom["T01"])
    assert (energy.max() - energy.min()) / abs(energy.mean()) < 0.10
    assert abs(energy.mean() / an.ns_Q(0.02, 0.1, 1.0, 2.0) - 1.0) < 0.15
    rise, rise_ns = mom["T"] - 1.0, an.ns_T(R, 0.4, 0.1, 1.0, 1.0, 2.0) - 1.0
    assert abs(rise.max() / rise_ns.max() - 1.0) < 0.10
    assert abs(R[np.argmax(rise)] - an.ns_R_Tmax(1.0, 2.0)) < 2.0 / 32


def test_steady_state_in_the_free_molecular_limit():
    """Sec. VI.D.2 (no collisions: Kn = 1000), 32 cells, HH(3;4) x H(3;4), steady
    after about 12 time units.  Exactly, the angular-momentum and energy fluxes
    are the same at every radius, R^2 T^{R phi} = n_w T_w Om R_in^2 / sqrt(pi)
    (Eq. bal_TRp) and Q = n_w R_in T_w^{3/2} Om^2 / sqrt(2 pi) (Eq. bal_Q) with
    Om = Omega_in R_in sqrt(1 / (2 T_w)) and n_w = 1 to O(Omega^2), and u^phi
    follows Eq. (bal_u_willis) to O(Omega^3).  The fluxes come out constant to
    about 1 %; their values are 14 % and 16 % above the closed forms with this
    small velocity set (9 % and 6 % with HH(4;8) x H(4;12); the paper needs 200
    nodes per half-axis to remove the discrete-velocity error).  With the force
    term's sign flipped the spreads exceed 100 %."""
    o = CouetteOracle("HH(3;4)xH(3;4)", CouetteGrid(32), Wall(0.1), Wall(0.0), 1000.0, TAU_KN_OVER_NT)
    F = o.initial_equilibrium()
    for _ in range(3000):
        F = o.step(F, 4e-3)
    R = o.g.Rc
    mom = o.m.full_moments(F)
    om = 0.1 / math.sqrt(2.0)
    flux = R ** 2 * mom["T01"]
    energy = R * (mom["q0"] + mom["u1"] * mom["T01"])
    for x, exact in ((flux, om / math.sqrt(math.pi)), (energy, om ** 2 / math.sqrt(2.0 * math.pi))):
        assert (x.max() - x.min()) / abs(x.mean()) < 0.03
        assert 1.0 < x.mean() / exact < 1.25
    willis = 0.1 * R / math.pi * (np.arcsin(1.0 / R) - np.sqrt(1.0 - R ** -2) / R)
    assert np.abs(mom["u1"] - willis).max() / 0.1 < 0.10


def _ghosted_centres(N, A, delta=0.5, r_in=1.0, r_out=2.0):
    """Cell centres s = -3 .. N+2 of the grid continued past both walls (equidistant in R,
    or in eta on the tanh-stretched grid), for exact ghost values of a smooth profile."""
    s = np.arange(-3, N + 3) + 0.5
    if A == 0.0:
        return r_in + (r_out - r_in) * s / N
    A0 = max(delta, 1.0 - delta)
    e_in, e_out = -math.atanh(A * delta / A0), math.atanh(A * (1.0 - delta) / A0)
    return r_in + (r_out - r_in) * (delta + A0 / A * np.tanh(e_in + s * (e_out - e_in) / N))


@pytest.mark.parametrize("A", [0.0, 0.9])
def test_chi_advection_is_second_order(A):
    """The chi-form flux difference p^R (R F)|_{s-1/2}^{s+1/2} / d chi of WENO-5 interface
    values approximates (p^R / R) d(R f)/dR at second order when V = p^R R varies across
    the cell (Sec. III.D), on the equidistant and on the tanh-stretched grid, for both
    signs of p^R (the mirror stencil on the negative side).  Exact ghosts, smooth profile."""
    f = lambda R: np.exp(-(R - 1.4) ** 2) * (1.0 + 0.2 * R)
    df = lambda R: np.exp(-(R - 1.4) ** 2) * (0.2 - 2.0 * (R - 1.4) * (1.0 + 0.2 * R))
    errs = []
    for N in (32, 64, 128):
        g = CouetteGrid(N, A=A)
        o = CouetteOracle("HH(2;3)xH(2;3)", g, Wall(0.0), Wall(0.0), 1.0, TAU_KN_OVER_N)
        p0 = o.m.p[0]
        Rg = _ghosted_centres(N, A)
        G = np.broadcast_to(f(Rg)[None, :, None, None], (2, N + 6) + tuple(o.m.nq)).copy()
        adv = o.advection(G)
        R = g.Rc
        exact = p0[None, None, :, None] * (f(R) / R + df(R))[None, :, None, None]
        errs.append(np.abs(adv - exact).max())
    order = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 1.9 < min(order) and max(order) < 2.2, (errs, order)


def test_residual_norms_on_the_equidistant_grid():
    """Eq. (msites_steady) with the rectangle rule of Sec. VI.E: on the equidistant grid the
    weights R_s dR are the midpoint rule of int R dR, exact for a constant integrand, so
    constant relative changes a of n and b of T and a uniform change c u_w of u^phi give the
    norms |a|, |b|, |c| times sqrt((R_out^2 - R_in^2) / 2).  The density and temperature
    enter as ratios (n varies across the gap here), the velocity scaled by u_w."""
    r_in, r_out, u_w = 1.0, 2.5, 0.37
    g = CouetteGrid(40, r_in, r_out)
    o = CouetteOracle("HH(2;3)xH(2;3)", g, Wall(u_w), Wall(0.0), 1.0, TAU_KN_OVER_N)
    R = g.Rc
    n0, T0, u0 = 2.0 + 0.3 * np.sin(3 * R), 1.0 + 0.1 * R, 0.2 / R
    a, b, c = 3e-3, -7e-4, 2e-3
    l2u, l2n, l2T = o.residual((n0 * (1 + a), 0 * R, u0 + c * u_w, T0 * (1 + b)), (n0, 0 * R, u0, T0), u_w)
    S = math.sqrt((r_out ** 2 - r_in ** 2) / 2.0)
    assert l2n == pytest.approx(abs(a) * S, rel=1e-12)
    assert l2T == pytest.approx(abs(b) * S, rel=1e-12)
    assert l2u == pytest.approx(abs(c) * S, rel=1e-12)


@pytest.mark.parametrize("A", [0.5, 0.95])
def test_residual_norms_on_the_stretched_grid(A):
    """On the stretched grid the rule is the rectangle rule in eta with the Jacobian
    (A0/A)(R_out - R_in) / cosh^2(eta) (Sec. VI.E): for the relative change a(R) = (R - R_in)^2
    the squared norm tends to int R (R - R_in)^4 dR = L^6/6 + R_in L^5/5 (L = R_out - R_in) at
    second order in the cell size."""
    r_in, r_out = 1.0, 2.0
    L = r_out - r_in
    exact = L ** 6 / 6.0 + r_in * L ** 5 / 5.0
    errs = []
    for N in (50, 100, 200):
        g = CouetteGrid(N, r_in, r_out, A=A)
        o = CouetteOracle("HH(2;3)xH(2;3)", g, Wall(0.1), Wall(0.0), 1.0, TAU_KN_OVER_N)
        R = g.Rc
        one = np.ones(N)
        _, l2n, _ = o.residual((one * (1 + (R - r_in) ** 2), 0 * R, 0 * R, one), (one, 0 * R, 0 * R, one), 0.1)
        errs.append(abs(l2n ** 2 - exact) / exact)
    order = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 1.8 < min(order) and max(order) < 2.2, (errs, order)
    assert errs[-1] < 2e-3


def _ghosted_sqrtg(N, A, delta=0.5, r_in=1.0, r_out=2.0):
    """sqrt(g) at the ghosted cell centres s = -3 .. N+2 (R on the equidistant grid; on the
    stretched grid A0 (R_out - R_in) R(eta) / (A cosh^2 eta), eta continued past the walls)."""
    R = _ghosted_centres(N, A, delta, r_in, r_out)
    if A == 0.0:
        return R
    A0 = max(delta, 1.0 - delta)
    e_in, e_out = -math.atanh(A * delta / A0), math.atanh(A * (1.0 - delta) / A0)
    eta = e_in + (np.arange(-3, N + 3) + 0.5) * (e_out - e_in) / N
    return A0 * (r_out - r_in) * R / (A * np.cosh(eta) ** 2)


@pytest.mark.parametrize("A", [0.0, 0.9])
def test_ftilde_advection_order(A):
    """The f~ flux difference of WENO-5 values of F~ = sqrt(g) f approximates the same
    operator as the chi form, (p^R / R) d(R f)/dR (e sqrt(g) = R), with exact ghosts: at high
    order on the equidistant grid (e = 1: the finite-difference WENO-5 difference quotient of
    F~), at second order on the stretched grid, where e_{s+1/2} multiplies the reconstructed
    flux (Eq. flux_cons_eta), as the interface factors of the chi form do."""
    f = lambda R: np.exp(-(R - 1.4) ** 2) * (1.0 + 0.2 * R)
    df = lambda R: np.exp(-(R - 1.4) ** 2) * (0.2 - 2.0 * (R - 1.4) * (1.0 + 0.2 * R))
    errs = []
    for N in (32, 64, 128):
        g = CouetteGrid(N, A=A)
        o = CouetteOracle("HH(2;3)xH(2;3)", g, Wall(0.0), Wall(0.0), 1.0, TAU_KN_OVER_N, formulation="ftilde")
        p0 = o.m.p[0]
        G = (_ghosted_sqrtg(N, A) * f(_ghosted_centres(N, A)))[None, :, None, None]
        G = np.broadcast_to(G, (2, N + 6) + tuple(o.m.nq)).copy()
        adv = o.advection_tilde(G)
        exact = p0[None, None, :, None] * (f(g.Rc) / g.Rc + df(g.Rc))[None, :, None, None]
        errs.append(np.abs(adv - exact).max())
    order = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    if A == 0.0:
        assert min(order) > 3.5, (errs, order)
    else:
        assert 1.8 < min(order) and max(order) < 2.3, (errs, order)


@pytest.mark.parametrize("A", [0.0, 0.95])
def test_ftilde_conserves_particles(A):
    """The f~ scheme conserves sum d eta sqrt(g) sum f' exactly: its flux difference telescopes
    and the diffuse walls carry no particles (Sec. III.F)."""
    o = CouetteOracle("HH(3;4)xH(3;4)", CouetteGrid(16, A=A), Wall(0.2), Wall(-0.1), 0.3, TAU_AOKI,
                      formulation="ftilde")
    F = o.initial_equilibrium()
    F = F * perturbation(F.shape, seed=11, amplitude=0.03)
    n0 = o.n_tot_ftilde(F)
    for _ in range(60):
        F = o.step(F, 1e-3)
    assert abs(o.n_tot_ftilde(F) / n0 - 1) < 1e-13


def test_ftilde_rest_state_is_not_held_at_the_walls():
    """The drawback of the f~ formulation (Sec. VI.B): f = const is not a steady state of the
    discrete scheme.  In the interior the residual of the rest state vanishes on the
    equidistant grid and falls at second order on the stretched grid, but in the cells next
    to the walls (ghosts of F~ that do not follow sqrt(g)) it stays of order 1e-2 and does
    not fall under refinement, where the chi formulation holds the rest state exactly."""
    for A in (0.0, 0.95):
        interior, wall = [], []
        for N in (16, 32, 64):
            o = CouetteOracle("HH(3;4)xH(3;4)", CouetteGrid(N, A=A), Wall(0.0), Wall(0.0), 0.1, TAU_AOKI,
                              formulation="ftilde")
            F = o.initial_equilibrium()
            per = np.abs(o.L(F)).max(axis=(0, 2, 3)) / np.abs(F).max()
            interior.append(per[4:-4].max())
            wall.append(per[[0, -1]].min())
            chi = CouetteOracle("HH(3;4)xH(3;4)", CouetteGrid(N, A=A), Wall(0.0), Wall(0.0), 0.1, TAU_AOKI)
            assert np.abs(chi.L(F)).max() / np.abs(F).max() < 1e-13
        if A == 0.0:
            assert max(interior) < 1e-13
        else:
            assert 3.0 < interior[0] / interior[1] and 3.0 < interior[1] / interior[2], interior
        assert min(wall) > 1e-2, wall
