"""Pins of the Shakhov collision in the oracle: the heat-flux term G of the target
f_eq + (1 - Pr) G (oracle.seeding.heat_flux_term) carries no particles, momentum or
energy, has exactly the heat flux it is built from, and so relaxes q at Pr / tau;
Pr = 1 is BGK."""
import numpy as np
import pytest

from oracle.couette import TAU_AOKI, CouetteGrid, CouetteOracle, Wall, relaxation_time, shakhov_term
from oracle.lbmodel import Model
from oracle.seeding import heat_flux_term, seed
from paper_1708_05944_gb300.inputs import perturbation

MODELS = ["HH(3;4)xH(3;4)", "HH(4;8)xH(4;20)"]


def fields(S, seed_=3):
    rng = np.random.default_rng(seed_)
    return (1.0 + 0.2 * rng.random(S), 0.2 * rng.standard_normal(S), 0.2 * rng.standard_normal(S),
            0.8 + 0.4 * rng.random(S), 0.05 * rng.standard_normal(S), 0.05 * rng.standard_normal(S))


@pytest.mark.parametrize("spec", MODELS)
def test_seed_moments_with_both_heat_flux_components(spec):
    """Grad's heat-flux form projected on the model (expansion orders >= 3) returns n, u, T and
    both q^0 and q^1 exactly in its discrete moments."""
    m = Model(spec)
    n, u0, u1, T, q0, q1 = fields(3)
    f1, f2 = seed(m, n, u0, u1, T, q0, q1)
    mom = m.full_moments(np.stack([f1, f2]))
    for k, ref in (("n", n), ("u0", u0), ("u1", u1), ("T", T), ("q0", q0), ("q1", q1)):
        np.testing.assert_allclose(mom[k], ref, rtol=1e-10, atol=1e-12, err_msg=k)


@pytest.mark.parametrize("spec", MODELS)
def test_heat_flux_term_is_collision_invariant_free(spec):
    m = Model(spec)
    n, u0, u1, T, q0, q1 = fields(3, 5)
    g1, g2 = heat_flux_term(m, n, u0, u1, T, q0, q1)
    p0, p1 = m.p[0][None, :, None], m.p[1][None, None, :]
    scale = np.abs(g1).max()
    assert np.abs(g1.sum(axis=(1, 2))).max() < 1e-12 * scale          # particles
    assert np.abs((p0 * g1).sum(axis=(1, 2))).max() < 1e-12 * scale   # momentum
    assert np.abs((p1 * g1).sum(axis=(1, 2))).max() < 1e-12 * scale
    energy = ((p0 ** 2 + p1 ** 2) * g1).sum(axis=(1, 2)) + g2.sum(axis=(1, 2))
    assert np.abs(energy).max() < 1e-11 * scale


def test_shakhov_relaxes_the_heat_flux_at_pr_over_tau():
    """A uniform state (no advection, no force): the collision term's heat-flux moment is
    -Pr q / tau, while the BGK one is -q / tau (q of f_eq vanishes for orders >= 3)."""
    m = Model("HH(4;8)xH(4;20)")
    n, u0, u1, T, q0, q1 = fields(2, 9)
    F = np.stack(seed(m, n, u0, u1, T, q0, q1))
    F = F + 0.002 * np.stack(seed(m, n, u0, u1, T)) * (perturbation(F.shape[1:], seed=2) - 1.0)  # other moments too
    mom = m.full_moments(F)
    feq = np.stack(m.feq(mom["n"], mom["u0"], mom["u1"], mom["T"]))
    tau = relaxation_time(0.1, mom["n"], mom["T"], TAU_AOKI)
    for pr in (1.0, 2.0 / 3.0):
        J = (-(F - feq) + (1.0 - pr) * shakhov_term(m, F)) / tau[:, None, None]
        x0 = m.p[0][None, :, None] - mom["u0"][:, None, None]
        x1 = m.p[1][None, None, :] - mom["u1"][:, None, None]
        e = 0.5 * (x0 ** 2 + x1 ** 2) * J[0] + 0.5 * J[1]
        dq = np.stack([(e * x0).sum(axis=(1, 2)), (e * x1).sum(axis=(1, 2))])
        ref = -pr * np.stack([mom["q0"], mom["q1"]]) / tau
        np.testing.assert_allclose(dq, ref, rtol=1e-9, atol=1e-12)


def test_prandtl_one_is_bgk():
    g = CouetteGrid(8)
    a = CouetteOracle("HH(3;4)xH(3;4)", g, Wall(0.1), Wall(0.0), 0.2, TAU_AOKI)
    b = CouetteOracle("HH(3;4)xH(3;4)", g, Wall(0.1), Wall(0.0), 0.2, TAU_AOKI, prandtl=1.0)
    F = a.initial_equilibrium()
    F = F * perturbation(F.shape, seed=6)
    np.testing.assert_array_equal(a.L(F), b.L(F))
