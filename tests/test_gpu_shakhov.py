"""GPU parity of the Shakhov collision (vlb_set_collision) against the oracle's: the library
adds cc dt (1 - Pr) G[F_prev] / tau to each BGK stage, G built on the device from closed-form
projections of xi^k g; the oracle builds G by numerical integration of the same functions."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle.channel import ChannelGrid, ChannelOracle  # noqa: E402
from oracle.couette import CouetteGrid, CouetteOracle, Wall  # noqa: E402
from paper_1708_05944_gb300 import vlb  # noqa: E402
from paper_1708_05944_gb300.inputs import perturbation  # noqa: E402
from tests.helpers import rel_err, to_lib, to_oracle  # noqa: E402

PR = 2.0 / 3.0


def couette_case(spec, n, kn, mode, seed, u_in=0.2, A=0.0):
    o = CouetteOracle(spec, CouetteGrid(n, 1.0, 2.0, A=A), Wall(u_in, 1.0), Wall(0.0, 1.05), kn, mode, prandtl=PR)
    F = o.initial_equilibrium()
    F = F * perturbation(F.shape, seed=seed, amplitude=0.03)
    return o, F, dict(n_cells=n, r_in=1.0, r_out=2.0, stretch_A=A)


@pytest.mark.parametrize("prec", [vlb.VLB_FP64, vlb.VLB_FP32_BULK])
@pytest.mark.parametrize("spec,n,A", [("HH(3;4)xH(3;4)", 12, 0.0), ("HH(4;8)xH(4;20)", 9, 0.9)])
def test_couette_stages_match_oracle(prec, spec, n, A):
    o, F0, grid = couette_case(spec, n, 0.1, 1, 13, A=A)
    c = vlb.Couette(spec, prec, [grid], [(0.2, 1.0)], [(0.0, 1.05)], [0.1], [1])
    c.set_collision(vlb.VLB_SHAKHOV, PR)
    c.set_f(to_lib(F0).astype(np.float64 if prec == vlb.VLB_FP64 else np.float32))
    dt = 1e-3
    tol = 1e-12 if prec == vlb.VLB_FP64 else 1e-6
    F1 = o.stage(1, dt, F0, F0)
    c.stage(dt, 1)
    assert rel_err(to_oracle(c.read_f()), F1) < tol
    F2 = o.stage(2, dt, F0, F1)
    c.stage(dt, 2)
    assert rel_err(to_oracle(c.read_f()), F2) < tol
    F3 = o.stage(3, dt, F0, F2)
    c.stage(dt, 3)
    assert rel_err(to_oracle(c.read_f()), F3) < tol
    # and the correction is not negligible: BGK differs from it
    b = vlb.Couette(spec, prec, [grid], [(0.2, 1.0)], [(0.0, 1.05)], [0.1], [1])
    b.set_f(to_lib(F0).astype(np.float64 if prec == vlb.VLB_FP64 else np.float32))
    b.step(dt, 1)
    assert rel_err(to_oracle(b.read_f()), F3) > 1e-5  # one step's correction: about 4e-5 of F
    c.close()
    b.close()


def test_ragged_instances_use_their_own_kn_and_tau():
    """Two instances with different Kn, tau convention and dt in one context: each cell's
    correction takes its own instance's (the kernel finds it by the instances' first cells)."""
    spec = "HH(3;4)xH(3;4)"
    oa, Fa, ga = couette_case(spec, 7, 0.05, 0, 3)
    ob, Fb, gb = couette_case(spec, 10, 0.5, 2, 4)
    c = vlb.Couette(spec, vlb.VLB_FP64, [ga, gb], [(0.2, 1.0)] * 2, [(0.0, 1.05)] * 2, [0.05, 0.5], [0, 2])
    c.set_collision(vlb.VLB_SHAKHOV, PR)
    c.set_dt([1e-3, 5e-4])
    c.set_f(np.concatenate([to_lib(Fa), to_lib(Fb)]))
    c.step(0.0, 1)
    got = to_oracle(c.read_f())
    assert rel_err(got[:, :7], oa.step(Fa, 1e-3)) < 1e-12
    assert rel_err(got[:, 7:], ob.step(Fb, 5e-4)) < 1e-12
    c.close()


def test_channel_stage_matches_oracle():
    spec, nl, nx = "HH(3;4)xH(3;4)", 6, 8
    o = ChannelOracle(spec, ChannelGrid(nl, nx), 0.1, prandtl=PR)
    F0 = o.initial_state()
    F0 = F0 * perturbation(F0.shape, seed=14, amplitude=0.03)
    c = vlb.Channel(spec, vlb.VLB_FP64, nl, nx, 0.1)
    c.set_collision(vlb.VLB_SHAKHOV, PR)
    lib = np.ascontiguousarray(F0.transpose(2, 1, 0, 3, 4).reshape(nx * nl, 2, F0.shape[3], F0.shape[4]))
    c.set_f(lib)
    dt = 1e-3
    c.stage(dt, 1)
    got = np.asarray(c.read_f()).reshape(nx, nl, 2, F0.shape[3], F0.shape[4]).transpose(2, 1, 0, 3, 4)
    assert rel_err(got, o.stage(1, dt, F0, F0)) < 1e-12
    c.close()


def test_graph_stepping_and_switching_back():
    spec = "HH(3;4)xH(3;4)"
    o, F0, grid = couette_case(spec, 16, 0.1, 1, 5)
    a = vlb.Couette(spec, vlb.VLB_FP32_BULK, [grid], [(0.2, 1.0)], [(0.0, 1.05)], [0.1], [1])
    b = vlb.Couette(spec, vlb.VLB_FP32_BULK, [grid], [(0.2, 1.0)], [(0.0, 1.05)], [0.1], [1])
    for c in (a, b):
        c.set_f(to_lib(F0).astype(np.float32))
    a.step_graph(1e-3, 3)  # a BGK graph captured first
    b.step(1e-3, 3)
    for c in (a, b):
        c.set_collision(vlb.VLB_SHAKHOV, PR)
    a.step_graph(1e-3, 6)
    b.step(1e-3, 6)
    assert np.array_equal(a.read_f(), b.read_f())
    for c in (a, b):
        c.set_collision(vlb.VLB_BGK)
    a.step_graph(1e-3, 3)
    b.step(1e-3, 3)
    assert np.array_equal(a.read_f(), b.read_f())
    with pytest.raises(vlb.VlbError):
        a.set_collision(vlb.VLB_SHAKHOV, -1.0)
    with pytest.raises(vlb.VlbError):
        a.set_collision(7)
    a.close()
    b.close()


def test_mass_momentum_and_energy_of_the_correction():
    """The correction carries no particles (nor momentum or energy, pinned on the oracle):
    the particle number of a wall-bounded instance stays conserved over many stages."""
    spec = "HH(4;8)xH(4;20)"
    o, F0, grid = couette_case(spec, 24, 0.2, 1, 8)
    c = vlb.Couette(spec, vlb.VLB_FP64, [grid], [(0.2, 1.0)], [(0.0, 1.05)], [0.2], [1])
    c.set_collision(vlb.VLB_SHAKHOV, PR)
    c.set_f(to_lib(F0))
    n0 = o.n_tot(F0)
    c.step(5e-4, 20)
    assert abs(o.n_tot(to_oracle(c.read_f())) / n0 - 1) < 1e-12
    c.close()
