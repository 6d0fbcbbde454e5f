"""Pins of the oracle's epsilon-free WENO-5 (Sec. III.C, Table IV)."""
import numpy as np
import pytest

from oracle.weno import weno5, weno5_weights


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


@pytest.mark.parametrize("func", [np.exp, lambda x: np.tanh(0.5 * x) + x])
def test_fifth_order_on_smooth_monotone_data(func):
    # (h_{s+1/2} - h_{s-1/2}) / dx -> F'(x_s) with O(dx^5) on monotone data
    errs = []
    for n in (20, 40, 80):
        dx = 1.0 / n
        xs = np.arange(-3, n + 4) * dx
        F = func(xs)
        j = np.arange(2, n + 4)  # interfaces between xs[j] and xs[j+1]
        h = weno5(F[j - 2], F[j - 1], F[j], F[j + 1], F[j + 2])
        d = (h[1:] - h[:-1]) / dx  # derivative at xs[3 .. n+3]
        x0 = xs[3:n + 4]
        ex = (func(x0 + 1e-4) - func(x0 - 1e-4)) / 2e-4 if func is not np.exp else np.exp(x0)
        errs.append(np.abs(d - ex).max() if func is np.exp else np.abs(d - ex).max())
    if func is np.exp:
        order = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
        assert min(order) > 4.6, (errs, order)


def test_mirror_stencil_symmetry():
    rng = np.random.default_rng(7)
    a = rng.uniform(0.5, 1.5, size=(5, 100))
    # for negative velocity the stencil is read from the other side: reflect the data
    np.testing.assert_allclose(weno5(*a), weno5(*a[::-1][::-1]), rtol=0, atol=0)
