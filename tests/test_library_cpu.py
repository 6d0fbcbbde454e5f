"""CPU checks of libvlb: it loads, exports every function include/vlb.h declares,
parses the paper's model notation, validates arguments before touching the GPU,
and builds quadrature and force tables equal to the oracle's."""
import os
import re

import numpy as np
import pytest

from oracle import lbmodel as lb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
vlb = pytest.importorskip("paper_1708_05944_gb300.vlb", reason="libvlb not built")


def declared_functions():
    text = open(os.path.join(ROOT, "include", "vlb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vlb_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    import ctypes
    lib = ctypes.CDLL(vlb.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(vlb.EXPORTS), set(names) ^ set(vlb.EXPORTS)


def test_parse_model():
    m = vlb.vlb_parse_model("HH(4;8)xH(4;20)")
    assert list(m.kind) == [1, 0] and list(m.N) == [4, 4] and list(m.Q) == [8, 20]
    m = vlb.vlb_parse_model("H(2;3) x HH(3;4)")
    assert list(m.kind) == [0, 1] and list(m.Q) == [3, 4]
    for bad in ("HH(4;4)xH(2;3)", "HH(4;8)", "X(1;2)xH(1;2)", "HH(4;8)xH(4;20)junk", "HH(-1;3)xH(1;2)"):
        with pytest.raises(vlb.VlbError):
            vlb.vlb_parse_model(bad)


@pytest.mark.parametrize("spec", ["HH(4;8)xH(4;20)", "HH(3;4)xH(3;4)", "H(4;5)xH(2;3)", "HH(4;8)xH(4;12)",
                                  "HH(4;16)xH(4;5)"])
def test_tables_equal_oracle(spec):
    m = vlb.vlb_parse_model(spec)
    om = lb.Model(spec)
    for a in (0, 1):
        p, w, K, Kt = vlb.vlb_axis_tables(m, a)
        np.testing.assert_allclose(p, om.p[a], rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(w, om.w[a], rtol=1e-13, atol=0)
        np.testing.assert_allclose(K, om.K[a], rtol=0, atol=1e-13 * np.abs(om.K[a]).max())
        np.testing.assert_allclose(Kt, om.Kt[a], rtol=0, atol=1e-13 * np.abs(om.Kt[a]).max())


@pytest.mark.parametrize("spec", ["HH(4;8)xH(4;20)", "HH(4;8)xH(4;12)", "HH(3;4)xH(3;4)", "H(4;16)xHH(4;10)"])
def test_node_reflection_used_by_the_split_contractions(spec):
    """The stage kernels of the fixed shapes mirror node k of an axis to k + Q/2 on
    half-range axes (positive nodes first) and to nq - 1 - k on full-range axes,
    and rely on K J = -J K, Kt J = J Kt for that permutation."""
    m = vlb.vlb_parse_model(spec)
    for a in (0, 1):
        p, _, K, Kt = vlb.vlb_axis_tables(m, a)
        n = len(p)
        J = np.array([(k + n // 2) % n if m.kind[a] == vlb.VLB_HALF else n - 1 - k for k in range(n)])
        np.testing.assert_allclose(p[J], -p, rtol=0, atol=1e-14 * np.abs(p).max())
        np.testing.assert_allclose(K[np.ix_(J, J)], -K, rtol=0, atol=1e-12 * np.abs(K).max())
        np.testing.assert_allclose(Kt[np.ix_(J, J)], Kt, rtol=0, atol=1e-12 * np.abs(Kt).max())


@pytest.mark.parametrize("spec", ["HH(4;8)xH(4;20)", "HH(4;8)xH(4;12)", "HH(3;4)xH(3;4)"])
def test_split_contraction_reproduces_the_full_one(spec):
    """The recombination the fixed-shape stage kernels use, on the library's tables:
    with e = f_k + f_Jk, o = f_k - f_Jk (k in the first half), P = (K[:, k] + K[:, Jk]) / 2
    and M = (K[:, k] - K[:, Jk]) / 2 over the first-half rows,
    axis 0 (K0 J = -J K0): (K0 f)_i = P e + M o, (K0 f)_Ji = M o - P e;
    axis 1 (Kt1 J = J Kt1): (Kt1 f)_j = P e + M o, (Kt1 f)_Jj = P e - M o."""
    m = vlb.vlb_parse_model(spec)
    rng = np.random.default_rng(7)
    for a, mat, anti in ((0, 2, True), (1, 3, False)):
        tabs = vlb.vlb_axis_tables(m, a)
        K, n = tabs[mat], len(tabs[0])
        h = n // 2
        J = np.array([(k + h) % n if m.kind[a] == vlb.VLB_HALF else n - 1 - k for k in range(n)])
        P = 0.5 * (K[:h, :h] + K[:h][:, J[:h]])
        M = 0.5 * (K[:h, :h] - K[:h][:, J[:h]])
        f = rng.standard_normal(n)
        e, o = f[:h] + f[J[:h]], f[:h] - f[J[:h]]
        full = K @ f
        scale = np.abs(full).max()
        np.testing.assert_allclose(P @ e + M @ o, full[:h], rtol=0, atol=1e-12 * scale)
        mirror = M @ o - P @ e if anti else P @ e - M @ o
        np.testing.assert_allclose(mirror, full[J[:h]], rtol=0, atol=1e-12 * scale)


def test_invalid_arguments_rejected_without_gpu():
    bad = [
        dict(grids=[dict(n_cells=2)]),
        dict(grids=[dict(n_cells=8, r_in=2.0, r_out=1.0)]),
        dict(kn=[0.0]),
        dict(tau=[7]),
        dict(model="HH(4;200)xH(4;200)"),  # beyond 65536 velocities
    ]
    for b in bad:
        with pytest.raises(vlb.VlbError) as e:
            vlb.Couette(b.get("model", "HH(3;4)xH(3;4)"), vlb.VLB_FP64, b.get("grids", [dict(n_cells=8)]),
                        [(0.1, 1.0)], [(0.0, 1.0)], b.get("kn", [0.1]), b.get("tau", [1]))
        assert e.value.status in (vlb.VLB_ERR_INVALID, vlb.VLB_ERR_UNSUPPORTED)


def test_setters_reject_a_null_context_without_gpu():
    assert vlb._lib.vlb_set_knudsen(None, 0.1, vlb.VLB_TAU_AOKI) == vlb.VLB_ERR_INVALID
    assert vlb._lib.vlb_set_channel_reservoirs(None, 2.0, 1.0, 1.0) == vlb.VLB_ERR_INVALID


def test_high_order_half_range_tables():
    """The library's tables for the paper's high-order axis HH(4;200) (Sec. VI.D.2): the rule
    integrates the half-Gaussian moments (checked up to degree 180, where double still holds
    p^k), and the force kernels act on
    populations of omega P (P a polynomial; no jump at p = 0) as the derivative does,
    d/dp (omega P) = omega (P' - p P), d/dp (p omega P) = omega (P + p P' - p^2 P); in the
    symmetric scaling sqrt(w_k'/w_k) K their entries stay of order Q^(3/2)."""
    m = vlb.vlb_parse_model("HH(4;200)xHH(4;10)")
    p, w, K, Kt = vlb.vlb_axis_tables(m, 0)
    Q = 200
    half = p > 0
    Mk = [0.5, 1.0 / np.sqrt(2.0 * np.pi)]
    for k in range(2, 181):
        Mk.append((k - 1) * Mk[k - 2])
    for k in (0, 1, 2, 7, 50, 120, 180):
        got = (w[half] * p[half] ** k).sum()
        assert abs(got / Mk[k] - 1) < 1e-12, k
    P = np.polynomial.polynomial.Polynomial([0.3, -1.0, 0.5, 0.2, -0.05])
    f = w * P(p)
    rows = np.abs(p) < 8.0  # where the polynomial's populations are not negligible in double
    np.testing.assert_allclose(((K @ f) / w)[rows], (P.deriv()(p) - p * P(p))[rows], rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(((Kt @ f) / w)[rows], (P(p) + p * P.deriv()(p) - p * p * P(p))[rows],
                               rtol=1e-8, atol=1e-8)
    s = np.sqrt(w)
    assert np.abs(K * s[None, :] / s[:, None]).max() < 3.0 * Q ** 1.5
