"""Pins of the oracle's epsilon-free WENO-5 (Sec. III.C, Table IV)."""
import numpy as np
import pytest

from oracle.weno import upwind_interfaces, weno5, weno5_weights


def test_table_iv_limits():
    # stencils built so that exactly the named indicators vanish (the row
    # sigma_3 = sigma_1 = 0 with sigma_2 != 0 has no five-point stencil: sigma_1 = 0
    # forces F_{s-2} = F_{s-1} = F_s and sigma_3 = 0 forces F_s = F_{s+1} = F_{s+2})
    cases = {
        "all": ((1, 1, 1, 1, 1), (0.1, 0.6, 0.3)),
        "s2=s3=0": ((0.3, 1, 1, 1, 1), (0, 2 / 3, 1 / 3)),
        "s1=s2=0": ((1, 1, 1, 1, 5), (1 / 7, 6 / 7, 0)),
        "s1=0": ((2, 2, 2, 3, 7), (1, 0, 0)),
        "s2=0": ((4, 1, 1, 1, 7), (0, 1, 0)),
        "s3=0": ((0, 5, 1, 1, 1), (0, 0, 1)),
    }
    for name, (st, expect) in cases.items():
        np.testing.assert_allclose(weno5_weights(*map(float, st)), expect, rtol=0, atol=1e-15, err_msg=name)


def test_equal_indicators_give_ideal_weights():
    # sigma_1 = sigma_2 = sigma_3 (nonzero) on linear data
    np.testing.assert_allclose(weno5_weights(1.0, 2.0, 3.0, 4.0, 5.0), (0.1, 0.6, 0.3), rtol=1e-14)


def test_reproduces_quadratics():
    # every candidate is exact for quadratic point data, so the weighted value is too
    x = np.arange(-2, 3, dtype=float)
    q = 0.3 * x ** 2 - 0.7 * x + 2.0
    h = weno5(*q)
    # the flux-difference form needs (h_{s+1/2} - h_{s-1/2}) = q'(x_s) for quadratics
    q2 = 0.3 * (x - 1) ** 2 - 0.7 * (x - 1) + 2.0
    assert float(h - weno5(*q2)) == pytest.approx(-0.7, abs=1e-13)


# smooth monotone data and their derivatives (epsilon-free weights lose accuracy at extrema)
FUNCS = {"exp": (np.exp, np.exp),
         "tanh": (lambda x: np.tanh(0.5 * x) + x, lambda x: 0.5 / np.cosh(0.5 * x) ** 2 + 1.0)}


@pytest.mark.parametrize("name", sorted(FUNCS))
@pytest.mark.parametrize("positive", [True, False])
def test_fifth_order_on_smooth_monotone_data(name, positive):
    """(h_{s+1/2} - h_{s-1/2}) / dx -> F'(x_s) at fifth order on either upwind side: the
    positive side reads (F_{s-2} .. F_{s+2}), the negative side the mirror stencil
    (F_{s+3} .. F_{s-1}) (Sec. III.C).  A stencil shifted by one cell drops to first order."""
    f, df = FUNCS[name]
    errs = []
    for n in (20, 40, 80):
        dx = 1.0 / n
        xs = np.arange(-3, n + 3) * dx  # cells -3 .. n+2: three ghost layers each side
        h = upwind_interfaces(f(xs), positive, axis=0)  # n + 1 interfaces, x_{s+1/2} for s = -1 .. n-1
        d = (h[1:] - h[:-1]) / dx  # at cells 0 .. n-1
        errs.append(np.abs(d - df(xs[3:n + 3])).max())
    order = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert min(order) > 4.5, (errs, order)
    assert errs[-1] < 1e-8


def test_mirror_side_is_the_reflection_of_the_positive_side():
    # the negative-velocity value at x_{s+1/2} is the positive-velocity value of the reflected
    # data at the reflected interface, operand for operand (so bit for bit)
    rng = np.random.default_rng(7)
    G = rng.uniform(0.5, 1.5, size=(40, 3))
    neg = upwind_interfaces(G, False, axis=0)
    pos_reflected = upwind_interfaces(G[::-1], True, axis=0)
    assert np.array_equal(neg, pos_reflected[::-1])
    # and the two sides differ on rough data
    assert not np.allclose(neg, upwind_interfaces(G, True, axis=0))
