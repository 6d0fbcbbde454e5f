"""The steady-state residual of Eq. (msites_steady) on the GPU (vlb_residual) against
the oracle's on the same moment snapshots, on equidistant and stretched grids."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle.couette import TAU_AOKI, CouetteGrid, CouetteOracle, Wall  # noqa: E402
from paper_1708_05944_gb300 import vlb  # noqa: E402
from paper_1708_05944_gb300.inputs import perturbation  # noqa: E402

MODEL = "HH(4;8)xH(4;20)"
GRIDS = [dict(n_cells=40, r_in=1.0, r_out=2.0, stretch_A=0.0, stretch_delta=0.5),
         dict(n_cells=48, r_in=1.0, r_out=3.0, stretch_A=0.9, stretch_delta=0.5),
         dict(n_cells=33, r_in=1.0, r_out=1.6, stretch_A=0.6, stretch_delta=0.3)]
WALL_U = [0.1, 0.35, 0.2]
KN = [0.1, 1.0, 0.3]


@pytest.mark.parametrize("prec", [vlb.VLB_FP64, vlb.VLB_FP32_BULK])
def test_residual_matches_the_oracle(prec):
    c = vlb.Couette(MODEL, prec, GRIDS, [(u, 1.0) for u in WALL_U], [(0.0, 1.0)] * 3, KN, [vlb.VLB_TAU_AOKI] * 3)
    m = c.model
    _, w0 = vlb.vlb_quadrature(m, 0)
    _, w1 = vlb.vlb_quadrature(m, 1)
    F = np.broadcast_to(np.outer(w0, w1), c.f_shape()) * perturbation(c.f_shape(), seed=31, amplitude=0.02)
    c.set_f(np.ascontiguousarray(F.astype(c.dtype)))
    c.set_dt([2e-4] * 3)
    c.residual()  # stores the first snapshot
    a = c.read_moments()
    c.step(0.0, 40)
    b = c.read_moments()
    l2u, l2n, l2T = c.residual()
    off = np.concatenate([[0], np.cumsum([g["n_cells"] for g in GRIDS])])
    for k, g in enumerate(GRIDS):
        o = CouetteOracle(MODEL, CouetteGrid(g["n_cells"], g["r_in"], g["r_out"], g["stretch_A"], g["stretch_delta"]),
                          Wall(WALL_U[k]), Wall(0.0), KN[k], TAU_AOKI)
        sl = slice(off[k], off[k + 1])
        ref = o.residual(tuple(x[sl] for x in b), tuple(x[sl] for x in a), WALL_U[k])
        got = (l2u[k], l2n[k], l2T[k])
        assert min(ref) > 1e-8  # the snapshots differ
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0, err_msg=str(k))
    c.close()
