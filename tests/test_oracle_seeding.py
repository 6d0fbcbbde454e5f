"""Pins of the seeding oracle (Grad heat-flux form projected on the model basis).

* with q = 0 the projection, computed by numerical integration of the
  continuous Gaussian, equals the closed-form truncated equilibrium of
  Eqs. (eq_gak_H) and (eq_gak_hh) evaluated by an independent route;
* with q != 0 the model's discrete moments of the seeded populations
  (Eqs. macro_red, macro_red_Tab, macro_red_q) return exactly the n, u, T and
  q^0 the seed was given, q^1 = 0, T^{01} = 0 and T^{00} = T^{11} = n T, which
  fixes every factor and sign of the Grad term;
* below the order the heat flux needs (N = 2 on axis 0) the flux is not
  reproduced, so the moment check above has the power to fail.
"""
import numpy as np
import pytest

from oracle import seeding
from oracle.lbmodel import Model

MODELS = ["HH(4;8)xH(4;20)", "HH(3;4)xH(4;8)", "H(4;6)xHH(3;5)"]


def fields(S, seed):
    rng = np.random.default_rng(seed)
    return (1 + 0.1 * rng.uniform(-1, 1, S), 0.1 * rng.uniform(-1, 1, S), 0.3 * rng.uniform(-1, 1, S),
            1 + 0.2 * rng.uniform(-1, 1, S), 0.05 * rng.uniform(-1, 1, S))


@pytest.mark.parametrize("spec", MODELS)
def test_zero_heat_flux_is_the_closed_form_equilibrium(spec):
    m = Model(spec)
    n, u0, u1, T, _ = fields(4, 1)
    f1, f2 = seeding.seed(m, n, u0, u1, T)
    e1, e2 = m.feq(n, u0, u1, T)
    assert np.abs(f1 - e1).max() < 1e-14
    assert np.abs(f2 - e2).max() < 1e-14


@pytest.mark.parametrize("spec", MODELS)
def test_seed_reproduces_its_moments(spec):
    m = Model(spec)
    n, u0, u1, T, q0 = fields(4, 2)
    f1, f2 = seeding.seed(m, n, u0, u1, T, q0)
    mom = m.full_moments(np.stack([f1, f2]))
    for k, v in (("n", n), ("u0", u0), ("u1", u1), ("T", T), ("q0", q0), ("T00", n * T), ("T11", n * T)):
        assert np.abs(mom[k] - v).max() < 1e-14, k
    assert np.abs(mom["q1"]).max() < 1e-14
    assert np.abs(mom["T01"]).max() < 1e-14


def test_insufficient_order_misses_the_heat_flux():
    m = Model("HH(2;4)xH(4;8)")
    n, u0, u1, T, q0 = fields(3, 3)
    q0 = np.full(3, 0.05)
    f1, f2 = seeding.seed(m, n, u0, u1, T, q0)
    mom = m.full_moments(np.stack([f1, f2]))
    assert np.abs(mom["q0"] - q0).max() > 1e-3
