"""The Couette path for velocity sets beyond 32 nodes on an axis (the high-order half-range
models of Sec. VI.D; vlb_large.cu) against the oracle, and the ballistic case of Sec. VI.D.2
with HH(4;200) x HH(4;10), 8000 velocities, against the free-molecular closed forms."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle.couette import TAU_KN_OVER_NT, CouetteGrid, CouetteOracle, Wall  # noqa: E402
from paper_1708_05944_gb300 import vlb  # noqa: E402
from tests.helpers import make_case, rel_err, to_lib, to_oracle  # noqa: E402


@pytest.mark.parametrize("spec,n,A", [("HH(4;20)xHH(3;4)", 12, 0.0), ("HH(3;20)xH(3;6)", 9, 0.9),
                                      ("H(4;40)xHH(2;3)", 8, 0.0)])
def test_fp64_stages_match_oracle(spec, n, A):
    o, F0, grid = make_case(spec, n, u_in=0.1, u_out=-0.05, T_out=1.05, kn=0.1, A=A)
    c = vlb.Couette(spec, vlb.VLB_FP64, [grid], [(0.1, 1.0)], [(-0.05, 1.05)], [0.1], [1])
    assert c.variants() == [(1, 256, 0)]  # the multi-kernel path
    c.set_f(to_lib(F0))
    dt = 1e-3
    F1 = o.stage(1, dt, F0, F0)
    c.stage(dt, 1)
    assert rel_err(to_oracle(c.read_f()), F1) < 1e-12
    nw = c.wall_density()[0]
    assert abs(nw[0] - o.last_nw[0]) < 1e-12 and abs(nw[1] - o.last_nw[1]) < 1e-12
    F2 = o.stage(2, dt, F0, F1)
    c.stage(dt, 2)
    assert rel_err(to_oracle(c.read_f()), F2) < 1e-12
    F3 = o.stage(3, dt, F0, F2)
    c.stage(dt, 3)
    assert rel_err(to_oracle(c.read_f()), F3) < 1e-12
    n_, u0, u1, T = c.read_moments()
    on, ou0, ou1, oT = o.m.moments(F3)
    assert np.abs(n_ / on - 1).max() < 1e-12 and np.abs(T / oT - 1).max() < 1e-12
    c.close()


def test_fp32_bulk_matches_oracle():
    spec, n = "HH(4;20)xHH(3;4)", 12
    o, F0, grid = make_case(spec, n, u_in=0.2, kn=0.3)
    c = vlb.Couette(spec, vlb.VLB_FP32_BULK, [grid], [(0.2, 1.0)], [(0.0, 1.0)], [0.3], [1])
    c.set_f(to_lib(F0).astype(np.float32))
    F = F0
    for _ in range(5):
        F = o.step(F, 1e-3)
    c.step(1e-3, 5)
    n_, u0, u1, T = c.read_moments()
    on, ou0, ou1, oT = o.m.moments(F)
    assert np.abs(n_ / on - 1).max() < 1e-5 and np.abs(T / oT - 1).max() < 1e-5
    assert np.abs(u1 - ou1).max() < 1e-5
    c.close()


def test_ragged_instances_match_their_oracles():
    spec = "HH(3;20)xHH(2;3)"
    oa, Fa, ga = make_case(spec, 7, u_in=0.1, kn=0.05, tau_mode=0, seed=1)
    ob, Fb, gb = make_case(spec, 11, u_in=-0.2, u_out=0.1, kn=0.7, tau_mode=2, A=0.9, seed=2)
    c = vlb.Couette(spec, vlb.VLB_FP64, [ga, gb], [(0.1, 1.0), (-0.2, 1.0)], [(0.0, 1.0), (0.1, 1.0)],
                    [0.05, 0.7], [0, 2])
    c.set_dt([1e-3, 5e-4])
    c.set_f(np.concatenate([to_lib(Fa), to_lib(Fb)]))
    c.step(0.0, 2)
    got = to_oracle(c.read_f())
    assert rel_err(got[:, :7], oa.step(oa.step(Fa, 1e-3), 1e-3)) < 1e-12
    assert rel_err(got[:, 7:], ob.step(ob.step(Fb, 5e-4), 5e-4)) < 1e-12
    c.close()


def test_graph_stepping_mass_and_restrictions():
    spec, n = "HH(4;20)xHH(3;4)", 16
    o, F0, grid = make_case(spec, n, u_in=0.2, kn=0.2)
    a = vlb.Couette(spec, vlb.VLB_FP64, [grid], [(0.2, 1.0)], [(0.0, 1.0)], [0.2], [1])
    b = vlb.Couette(spec, vlb.VLB_FP64, [grid], [(0.2, 1.0)], [(0.0, 1.0)], [0.2], [1])
    for c in (a, b):
        c.set_f(to_lib(F0))
    a.step_graph(1e-3, 9)
    b.step(1e-3, 9)
    assert np.array_equal(a.read_f(), b.read_f())
    n0 = o.n_tot(F0)
    a.step_graph(1e-3, 300)
    assert abs(o.n_tot(to_oracle(a.read_f())) / n0 - 1) < 1e-12
    a.residual()
    a.step(1e-3, 3)
    assert all(np.isfinite(x).all() for x in a.residual())
    for call in (lambda: a.init_from_moments(np.ones(n), np.zeros(n), np.zeros(n), np.ones(n)),
                 lambda: a.set_collision(vlb.VLB_SHAKHOV, 2.0 / 3.0)):
        with pytest.raises(vlb.VlbError) as e:
            call()
        assert e.value.status == vlb.VLB_ERR_UNSUPPORTED
    a.close()
    b.close()


def test_ballistic_couette_with_200_nodes_per_half_axis():
    """Sec. VI.D.2 with the paper's model HH(4;200) x HH(4;10) (8000 velocities), N_R = 16
    stretched cells (A = 0.95, delta = 0.75), dt = 2e-5, 10 time units (500 000 steps, the
    paper's run), FP32, inner wall speed 0.1, Kn = 1000.  Without collisions the
    angular-momentum flux R^2 T^{R phi} and the energy flux R (q^R + u^phi T^{R phi}) are the
    same at every radius and equal the closed forms of Eqs. (bal_TRp, bal_Q) to O(Omega^2),
    and u^phi follows Willis' profile, Eq. (bal_u_willis).  The small velocity sets of the
    oracle pins miss the fluxes by 6-16 % (discrete-velocity error); with 200 nodes per
    half-axis the paper removes that error."""
    spec, n, uw = "HH(4;200)xHH(4;10)", 16, 0.1
    grid = dict(n_cells=n, r_in=1.0, r_out=2.0, stretch_A=0.95, stretch_delta=0.75)
    c = vlb.Couette(spec, vlb.VLB_FP32_BULK, [grid], [(uw, 1.0)], [(0.0, 1.0)], [1000.0], [TAU_KN_OVER_NT])
    c.init_equilibrium()
    c.step_graph(2e-5, 500_000)
    n_, u0, u1, T, Tab, q = c.read_moments(full=True)
    R = CouetteGrid(n, 1.0, 2.0, A=0.95, delta=0.75).Rc
    om = uw / math.sqrt(2.0)
    flux = R ** 2 * Tab[:, 1]
    energy = R * (q[:, 0] + u1 * Tab[:, 1])
    for x, exact in ((flux, om / math.sqrt(math.pi)), (energy, om ** 2 / math.sqrt(2.0 * math.pi))):
        assert (x.max() - x.min()) / abs(x.mean()) < 0.02, (x, exact)
        assert abs(x.mean() / exact - 1) < 0.03, (x.mean(), exact)
    willis = uw * R / math.pi * (np.arcsin(1.0 / R) - np.sqrt(1.0 - R ** -2) / R)
    assert np.abs(u1 - willis).max() / uw < 0.03
    c.close()
