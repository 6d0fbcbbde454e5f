"""Pins of the oracle's gradually-expanding-channel stage (Sec. VII.A-C)."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle.channel import ChannelGrid, ChannelOracle, chi_xi, dphi, phi
from paper_1708_05944_gb300.inputs import perturbation

MODEL = "HH(4;8)xH(4;12)"


def test_wall_shape_limits_and_chi_closed_form():
    # phi(-inf) = (tanh 2 - 1)/2 ~ -0.018, phi(+inf) = (tanh 2 + 1)/2 ~ 0.982, phi(0) = 0 (Sec. VII.B)
    assert phi(-1e4) == pytest.approx((math.tanh(2) - 1) / 2, abs=1e-15)
    assert phi(1e4) == pytest.approx((math.tanh(2) + 1) / 2, abs=1e-15)
    assert phi(0.0) == pytest.approx(0.0, abs=1e-16)
    # Eq. (chi_canalie_exp) against a numerical integral of d chi = (1 + phi) d xi
    for x in (-10.0, -3.0, 5.0, 17.0, 40.0):
        num = quad(lambda t: 1.0 + phi(t), 0.0, x, epsabs=1e-13, epsrel=1e-13)[0]
        assert chi_xi(x) == pytest.approx(num, rel=1e-11, abs=1e-12)
    # phi' by central differences
    h = 1e-5
    for x in (-2.0, 3.0, 10.0):
        assert dphi(x) == pytest.approx((phi(x + h) - phi(x - h)) / (2 * h), rel=1e-7)


def test_stretched_lambda_grid():
    g = ChannelGrid(16, 8)
    assert g.lf[0] == 0.0 and g.lf[-1] == 1.0 and np.all(np.diff(g.lf) > 0)
    # finer near the wall (A = 0.95 pushes points to lambda = 1)
    assert g.dl[-1] < g.dl[0]


@pytest.mark.parametrize("nl,nx", [(8, 16), (6, 10)])
def test_uniform_rest_state_is_exact(nl, nx):
    # f = f_eq(1, 0, 1) everywhere with both reservoirs at n = 1: the discrete connection
    # coefficients of Sec. VII.A make the constant state an exact solution
    o = ChannelOracle(MODEL, ChannelGrid(nl, nx), 0.05, n_in=1.0, n_out=1.0)
    F = o.initial_state()
    assert np.abs(o.L(F)).max() < 1e-13
    np.testing.assert_allclose(o.last_nw, 1.0, rtol=0, atol=1e-14)


def test_particle_balance_is_telescoping():
    # sum over cells of vol * L[f'] equals inlet minus outlet flux: the wall flux vanishes
    # by n_w, the centreline flux by specular symmetry, force and collision carry no mass
    o = ChannelOracle(MODEL, ChannelGrid(8, 12), 0.05)
    F = o.initial_state()
    F = F * perturbation(F.shape, seed=4, amplitude=0.02)
    L = o.L(F)
    b = o.last_boundary_flux
    dN = float((o.g.vol * L[0].sum(axis=(2, 3))).sum())
    assert abs(b["wall"]) < 1e-14 and abs(b["centre"]) < 1e-14
    assert dN == pytest.approx(b["inlet"] - b["outlet"], rel=1e-9, abs=1e-14)


def test_specular_centreline_keeps_mirror_symmetry_of_rest():
    # a state even in p^lambda stays even-balanced: the centreline flux of f' vanishes
    o = ChannelOracle(MODEL, ChannelGrid(6, 8), 0.1)
    F = o.initial_state()
    o.L(F)
    assert abs(o.last_boundary_flux["centre"]) < 1e-15


def test_flow_rate_ends_impose_the_profile():
    """Eq. (canalie_inlet_s) is the definition of the flow-rate boundary: after the ghosts
    are set, the particle flux through each end interface of row s equals (1 + phi) Q_s,
    Q_s the parabolic profile of Eqs. (canalie_inlet, canalie_outlet), on a perturbed
    state (the interface values of the entering and leaving halves come from three equal
    ghost or stencil cells, where WENO-5 returns that value: Table IV)."""
    g = ChannelGrid(10, 12)
    o = ChannelOracle(MODEL, g, 0.05, q0=0.1)
    F = o.initial_state(n_profile=np.ones(12)) * perturbation((2, 10, 12) + tuple(o.m.nq), seed=17)
    o.L(F)
    for end, key in ((0, "inlet_rows"), (1, "outlet_rows")):
        q, target = o.flow_profile(end)
        assert np.abs(o.last_boundary_flux[key] / target - 1).max() < 1e-12
        # the profile: 3 Q_0 / (H (1 + phi)) (1 - lambda^2) (H = 2), zero flux at the wall
        assert np.allclose(target, 1.5 * 0.1 * (1.0 - g.lc ** 2), rtol=1e-14)
        assert np.all(o.last_inflow_density[end] > 0)
    # the inflow densities are near 1 for a state near f_eq(1, 0, 1) with small Q_0
    assert np.abs(o.last_inflow_density[0] - 1).max() < 0.2


def test_flow_rate_rest_state_is_exact():
    """With Q_0 = 0 the rest state f_eq(1, 0, T0) has zero flux through each end on its own
    (sum of V^xi w_i w_j = 0), so n_s = 1 and L vanishes."""
    o = ChannelOracle(MODEL, ChannelGrid(8, 8), 0.05, q0=0.0)
    F = o.initial_state(n_profile=np.ones(8))
    L = o.L(F)
    assert np.abs(L).max() / np.abs(F).max() < 1e-13
    for ns in o.last_inflow_density:
        assert np.abs(ns - 1).max() < 1e-13


def test_flow_rate_ends_conserve_particles():
    """In = out row by row ((1 + phi) Q_s is the same at both ends), the wall and the
    centreline carry no flux: the particle number is constant while the flow develops."""
    o = ChannelOracle(MODEL, ChannelGrid(8, 12), 0.05, q0=0.1)
    F = o.initial_state(n_profile=np.ones(12))
    n0 = o.n_tot(F)
    for _ in range(5):
        F = o.step(F, 1e-3)
    assert abs(o.n_tot(F) / n0 - 1) < 1e-13
    # and the flow is established at the inlet: u^xi of the first column follows the profile's shape
    n, ul, ux, T = o.moments(F)
    assert ux[0, 0] > ux[-1, 0] > 0


def test_post_derivative_formulas_are_exact_on_quadratics():
    """The three-point lambda formulas (bulk, first and last node) on the stretched rows and
    the xi formulas (centred, one-sided second order) differentiate quadratics exactly."""
    from oracle.channel import lambda_derivative, xi_derivative
    g = ChannelGrid(11, 9)
    f = (0.3 - 1.7 * g.lc + 2.2 * g.lc ** 2)[:, None] * np.ones((1, 4))
    np.testing.assert_allclose(lambda_derivative(f, g.lc)[:, 0], -1.7 + 4.4 * g.lc, rtol=1e-11, atol=1e-11)
    x = np.linspace(-3.0, 5.0, 9)
    h = np.ones((3, 1)) * (1.0 + 0.5 * x - 0.25 * x ** 2)[None, :]
    np.testing.assert_allclose(xi_derivative(h, x[1] - x[0])[0], 0.5 - 0.5 * x, rtol=1e-12, atol=1e-12)
    # a wrong sign in the last-node formula would not pass
    assert abs(lambda_derivative(g.lc[:, None] ** 2, g.lc)[-1, 0] - 2 * g.lc[-1]) < 1e-11


def test_post_fields_of_a_poiseuille_state():
    """A state with u^xi-hat = U (1 - lambda^2), u^lambda-hat = 0, n = 1 + 0.1 lambda, T = 1:
    the rotation to (u^x, u^y) keeps |u|; where phi' vanishes (far downstream) the vorticity
    is that of the parabola, -2 U lambda / (1 + phi) (the Poiseuille form -3 u_0 x / x_top^2);
    P = n T is linear in lambda, so its extrapolation to the wall is exact; psi telescopes."""
    from oracle.channel import postprocess
    g = ChannelGrid(12, 16, xi_in=20.0, xi_out=40.0)
    o = ChannelOracle(MODEL, g, 0.05)
    U = 0.15
    lam = g.lc[:, None] * np.ones((1, g.nx))
    n = 1.0 + 0.1 * lam
    F = o.feq_cells(n, 0.0 * lam, U * (1.0 - lam ** 2), np.ones_like(lam))
    p = postprocess(o, F)
    nn, ul, uxh, T = o.moments(F)
    np.testing.assert_allclose(p["ux"] ** 2 + p["uy"] ** 2, ul ** 2 + uxh ** 2, rtol=1e-12, atol=1e-15)
    ph = phi(g.xc)[None, :]
    far = g.xc > 30.0  # phi' < 1e-6 there
    np.testing.assert_allclose(p["omega"][:, far], (-2.0 * U * lam / (1.0 + ph))[:, far], rtol=1e-5)
    np.testing.assert_allclose(p["pw"], 1.1, rtol=1e-12)
    # psi at the wall: minus the row sum of rho u^y times the x width of each row
    wall = -(nn * p["uy"] * g.dl[:, None]).sum(axis=0) * (1.0 + phi(g.xc))
    np.testing.assert_allclose(p["psi"][-1], wall, rtol=1e-12)
    assert np.all(p["psi"][0] == 0.0) and np.all(np.diff(p["psi"], axis=0) < 0)


def test_post_rotation_and_vorticity_in_the_expansion():
    """Where phi' is large (the expanding part, xi in [0, 12]): a Cartesian field given as
    triad components through the inverse rotation comes back unchanged (a sign slip in
    Eq. canalie_u would not), and the two geometric terms of Eq. (canalie_vorti) are exact
    for u^x = W lambda^2, u^y = 0 (omega = 2 W lambda^2 phi' / (1 + phi)) and for
    u^x = W (xi - 5)^2, u^y = 0 (omega = -2 W (xi - 5))."""
    from oracle.channel import postprocess
    g = ChannelGrid(10, 24, xi_in=0.0, xi_out=12.0)
    o = ChannelOracle(MODEL, g, 0.05)
    lam = g.lc[:, None] * np.ones((1, g.nx))
    xi = np.ones((g.nl, 1)) * g.xc[None, :]
    a = lam * dphi(g.xc)[None, :]
    root = np.sqrt(1.0 + a ** 2)
    ph = phi(g.xc)[None, :]
    W = 0.05
    for ux_c, om in ((W * lam ** 2, 2.0 * W * lam ** 2 * dphi(g.xc)[None, :] / (1.0 + ph)),
                     (W * (xi - 5.0) ** 2, -2.0 * W * (xi - 5.0))):
        uy_c = 0.02 + 0.0 * lam
        F = o.feq_cells(np.ones_like(lam), (ux_c - a * uy_c) / root, (a * ux_c + uy_c) / root, np.ones_like(lam))
        p = postprocess(o, F)
        np.testing.assert_allclose(p["ux"], ux_c, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(p["uy"], uy_c, rtol=1e-12)
        np.testing.assert_allclose(p["omega"], om, rtol=1e-9, atol=1e-13)


def test_clb_particle_balance_and_rest_state():
    """The Cartesian-split channel (Sec. VII.G): the particle balance telescopes (wall flux zero
    by n_w, centreline flux zero by the p^x mirror); at rest (n_in = n_out = 1) n_w = 1, and the
    rest state is not exact (no force term balances the geometric part of the advection
    discretely) but its residual falls under refinement."""
    from oracle.channel import ClbChannelOracle
    o = ClbChannelOracle("HH(3;4)xHH(3;4)", ChannelGrid(8, 12), 0.05)
    F = o.initial_state()
    F = F * perturbation(F.shape, seed=4, amplitude=0.02)
    L = o.L(F)
    b = o.last_boundary_flux
    dN = float((o.g.vol * L[0].sum(axis=(2, 3))).sum())
    assert abs(b["wall"]) < 1e-13 and abs(b["centre"]) < 1e-13
    assert dN == pytest.approx(b["inlet"] - b["outlet"], rel=1e-9, abs=1e-14)
    res = []
    for nl, nx in ((8, 12), (16, 24), (32, 48)):
        o = ClbChannelOracle("HH(3;4)xHH(3;4)", ChannelGrid(nl, nx), 0.05, n_in=1.0, n_out=1.0)
        F = o.initial_state()
        res.append(np.abs(o.L(F)).max() / np.abs(F).max())
        np.testing.assert_allclose(o.last_nw, 1.0, rtol=0, atol=1e-13)
    assert res[-1] > 1e-5 and res[-1] < res[0] and res[1] / res[2] > 2.5, res


def test_clb_shakhov_term_relaxes_each_cell_s_heat_flux():
    """The Shakhov collision on the Cartesian split: what it adds to L at each cell carries no
    particles, momentum or energy, and its heat-flux moment is (1 - Pr) q / tau with the cell's
    own q and the channel's tau = Kn / (n T)."""
    from oracle.channel import ClbChannelOracle
    spec, g = "HH(3;4)xHH(3;4)", ChannelGrid(6, 8)
    a = ClbChannelOracle(spec, g, 0.05)
    b = ClbChannelOracle(spec, g, 0.05, prandtl=2.0 / 3.0)
    F = a.initial_state()
    F = F * perturbation(F.shape, seed=8, amplitude=0.05)
    dL = b.L(F) - a.L(F)
    m = a.m
    flat = F.reshape((2, -1) + F.shape[3:])
    dflat = dL.reshape((2, -1) + F.shape[3:])
    mom = m.full_moments(flat)
    tau = 0.05 / (mom["n"] * mom["T"])
    x0 = m.p[0][None, :, None] - mom["u0"][:, None, None]
    x1 = m.p[1][None, None, :] - mom["u1"][:, None, None]
    scale = np.abs(dflat).max()
    assert scale > 1e-4
    assert np.abs(dflat[0].sum(axis=(1, 2))).max() < 1e-12 * scale
    assert np.abs((x0 * dflat[0]).sum(axis=(1, 2))).max() < 1e-12 * scale
    assert np.abs((x1 * dflat[0]).sum(axis=(1, 2))).max() < 1e-12 * scale
    e = 0.5 * (x0 ** 2 + x1 ** 2) * dflat[0] + 0.5 * dflat[1]
    assert np.abs(e.sum(axis=(1, 2))).max() < 1e-11 * scale
    dq = np.stack([(e * x0).sum(axis=(1, 2)), (e * x1).sum(axis=(1, 2))])
    np.testing.assert_allclose(dq, (1.0 / 3.0) * np.stack([mom["q0"], mom["q1"]]) / tau, rtol=1e-9, atol=1e-12)


def test_clb_equals_the_vielbein_channel_where_the_wall_is_straight():
    """Far downstream (xi in [30, 40], phi' < 1e-6) the triad of Eq. (canalie_phat) is the
    Cartesian one and the connection coefficients vanish, so the Cartesian-split and the
    vielbein stage operators agree on the same populations."""
    from oracle.channel import ClbChannelOracle
    g = ChannelGrid(8, 12, xi_in=30.0, xi_out=40.0)
    v = ChannelOracle("HH(3;4)xHH(3;4)", g, 0.05)
    c = ClbChannelOracle("HH(3;4)xHH(3;4)", g, 0.05)
    F = v.initial_state()
    F = F * perturbation(F.shape, seed=6, amplitude=0.02)
    Lv, Lc = v.L(F), c.L(F)
    assert np.abs(Lv - Lc).max() / np.abs(Lv).max() < 1e-5
    # and they differ where the channel expands
    g2 = ChannelGrid(8, 12, xi_in=0.0, xi_out=12.0)
    F2 = ChannelOracle("HH(3;4)xHH(3;4)", g2, 0.05).initial_state() * perturbation(F.shape, seed=6, amplitude=0.02)
    assert np.abs(ChannelOracle("HH(3;4)xHH(3;4)", g2, 0.05).L(F2) - ClbChannelOracle("HH(3;4)xHH(3;4)", g2, 0.05).L(F2)).max() > 1e-3
