"""GPU parity of the f~ formulation of the Couette stage (vlb_set_formulation; Sec. VI.B,
Eqs. boltz_couette_cons, boltz_couette_str_cons) against the oracle's: F~ = sqrt(g) f
reconstructed and differenced over d eta, the walls acting on F~."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle.couette import TAU_AOKI, CouetteGrid, CouetteOracle, Wall  # noqa: E402
from paper_1708_05944_gb300 import vlb  # noqa: E402
from paper_1708_05944_gb300.inputs import perturbation  # noqa: E402
from tests.helpers import rel_err, to_lib, to_oracle  # noqa: E402


def case(spec, n, A, seed=19):
    o = CouetteOracle(spec, CouetteGrid(n, 1.0, 2.0, A=A), Wall(0.15, 1.0), Wall(-0.05, 1.05), 0.2, TAU_AOKI,
                      formulation="ftilde")
    F = o.initial_equilibrium()
    F = F * perturbation(F.shape, seed=seed, amplitude=0.02)
    return o, F, dict(n_cells=n, r_in=1.0, r_out=2.0, stretch_A=A)


def ctx(spec, prec, grid):
    c = vlb.Couette(spec, prec, [grid], [(0.15, 1.0)], [(-0.05, 1.05)], [0.2], [TAU_AOKI])
    c.set_formulation(vlb.VLB_FTILDE)
    return c


@pytest.mark.parametrize("spec,n,A", [("HH(3;4)xH(3;4)", 16, 0.0), ("HH(4;8)xH(4;20)", 12, 0.95),
                                      ("HH(4;20)xHH(3;4)", 10, 0.9)])
def test_fp64_stages_match_oracle(spec, n, A):
    o, F0, grid = case(spec, n, A)
    c = ctx(spec, vlb.VLB_FP64, grid)
    c.set_f(to_lib(F0))
    dt = 5e-4
    F1 = o.stage(1, dt, F0, F0)
    c.stage(dt, 1)
    assert rel_err(to_oracle(c.read_f()), F1) < 1e-12
    nw = c.wall_density()[0]
    assert abs(nw[0] / o.last_nw[0] - 1) < 1e-12 and abs(nw[1] / o.last_nw[1] - 1) < 1e-12
    F2 = o.stage(2, dt, F0, F1)
    c.stage(dt, 2)
    assert rel_err(to_oracle(c.read_f()), F2) < 1e-12
    F3 = o.stage(3, dt, F0, F2)
    c.stage(dt, 3)
    assert rel_err(to_oracle(c.read_f()), F3) < 1e-12
    c.close()


def test_fp32_moments_and_conservation():
    spec, n = "HH(3;4)xH(3;4)", 20
    o, F0, grid = case(spec, n, 0.9)
    c = ctx(spec, vlb.VLB_FP32_BULK, grid)
    c.set_f(to_lib(F0).astype(np.float32))
    F = F0
    for _ in range(5):
        F = o.step(F, 5e-4)
    c.step(5e-4, 5)
    n_, u0, u1, T = c.read_moments()
    on, ou0, ou1, oT = o.m.moments(F)
    assert np.abs(n_ / on - 1).max() < 1e-5 and np.abs(T / oT - 1).max() < 1e-5
    d = ctx(spec, vlb.VLB_FP64, grid)
    d.set_f(to_lib(F0))
    n0 = o.n_tot_ftilde(F0)
    d.step_graph(5e-4, 300)
    assert abs(o.n_tot_ftilde(to_oracle(d.read_f())) / n0 - 1) < 1e-12
    c.close()
    d.close()


def test_switching_back_and_refusals():
    spec, n = "HH(3;4)xH(3;4)", 16
    o, F0, grid = case(spec, n, 0.0)
    chi = CouetteOracle(spec, CouetteGrid(n), Wall(0.15, 1.0), Wall(-0.05, 1.05), 0.2, TAU_AOKI)
    c = ctx(spec, vlb.VLB_FP64, grid)
    c.set_f(to_lib(F0))
    c.step(5e-4, 1)
    F1 = o.step(F0, 5e-4)
    assert rel_err(to_oracle(c.read_f()), F1) < 1e-12
    c.set_formulation(vlb.VLB_CHI)
    c.step(5e-4, 1)
    assert rel_err(to_oracle(c.read_f()), chi.step(F1, 5e-4)) < 1e-13
    with pytest.raises(vlb.VlbError):
        c.set_formulation(3)
    ch = vlb.Channel("HH(3;4)xH(3;4)", vlb.VLB_FP64, 6, 8, 0.1)
    assert vlb._lib.vlb_set_formulation(ch.h, vlb.VLB_FTILDE) == vlb.VLB_ERR_UNSUPPORTED
    c.close()
    ch.close()


def test_fused_kernel_launch_shapes_and_ragged_instances():
    """Velocity sets of the fused stage kernel run f~ on its f~ instance (launch shape 0, plain
    and persistent): two ragged instances (stretched and equidistant) in one context against
    their oracles over three stages; other launch shapes are refused."""
    spec = "HH(4;8)xH(4;20)"
    (oa, Fa, ga), (ob, Fb, gb) = case(spec, 12, 0.95, seed=20), case(spec, 30, 0.0, seed=21)
    c = vlb.Couette(spec, vlb.VLB_FP64, [ga, gb], [(0.15, 1.0)] * 2, [(-0.05, 1.05)] * 2, [0.2, 0.2],
                    [TAU_AOKI] * 2)
    c.set_formulation(vlb.VLB_FTILDE)
    dt = 5e-4
    refs = []
    for o, F0 in ((oa, Fa), (ob, Fb)):
        F1 = o.stage(1, dt, F0, F0)
        F2 = o.stage(2, dt, F0, F1)
        refs.append((F1, F2, o.stage(3, dt, F0, F2)))
    for v in (0, 1):
        c.set_variant(v)
        c.set_f(np.concatenate([to_lib(Fa), to_lib(Fb)], axis=0))
        for k in (1, 2, 3):
            c.stage(dt, k)
            got = c.read_f()
            assert rel_err(to_oracle(got[:12]), refs[0][k - 1]) < 1e-12, (v, k)
            assert rel_err(to_oracle(got[12:]), refs[1][k - 1]) < 1e-12, (v, k)
    with pytest.raises(vlb.VlbError) as e:
        c.set_variant(2)
    assert e.value.status == vlb.VLB_ERR_INVALID
    c.set_formulation(vlb.VLB_CHI)
    c.set_variant(2)  # every launch shape again on the chi formulation
    c.close()


def test_shakhov_on_the_ftilde_formulation():
    """The Shakhov pass composes with the f~ stage of the fused kernel: FP64, three stages,
    against the oracle's f~ operator with Pr = 2/3."""
    spec, n = "HH(4;8)xH(4;20)", 12
    o = CouetteOracle(spec, CouetteGrid(n, 1.0, 2.0, A=0.95), Wall(0.15, 1.0), Wall(-0.05, 1.05), 0.2, TAU_AOKI,
                      formulation="ftilde", prandtl=2.0 / 3.0)
    F0 = o.initial_equilibrium()
    F0 = F0 * perturbation(F0.shape, seed=22, amplitude=0.05)
    c = ctx(spec, vlb.VLB_FP64, dict(n_cells=n, r_in=1.0, r_out=2.0, stretch_A=0.95))
    c.set_collision(vlb.VLB_SHAKHOV, 2.0 / 3.0)
    c.set_f(to_lib(F0))
    F = F0
    for k in (1, 2, 3):
        F = o.stage(k, 5e-4, F0, F)
        c.stage(5e-4, k)
        assert rel_err(to_oracle(c.read_f()), F) < 1e-12
    c.close()
