"""GPU parity of the Cartesian-split channel (vlb_set_formulation VLB_CARTESIAN; Sec. VII.G,
Eqs. canalie_coord_beq_cons, canalie_coord_nw) against the oracle's ClbChannelOracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle.channel import ChannelGrid, ChannelOracle, ClbChannelOracle  # noqa: E402
from paper_1708_05944_gb300 import vlb  # noqa: E402
from paper_1708_05944_gb300.inputs import perturbation  # noqa: E402
from tests.helpers import rel_err  # noqa: E402


def to_lib(F):
    nl, nx = F.shape[1], F.shape[2]
    return np.ascontiguousarray(np.asarray(F).transpose(2, 1, 0, 3, 4).reshape(nx * nl, 2, F.shape[3], F.shape[4]))


def to_oracle(f, nl, nx):
    f = np.asarray(f, dtype=np.float64).reshape(nx, nl, 2, f.shape[2], f.shape[3])
    return np.ascontiguousarray(f.transpose(2, 1, 0, 3, 4))


@pytest.mark.parametrize("spec,nl,nx,xi", [("HH(3;4)xHH(3;4)", 7, 12, (-10.0, 40.0)),
                                          ("HH(4;8)xH(4;12)", 9, 16, (0.0, 12.0))])
def test_fp64_stages_match_oracle(spec, nl, nx, xi):
    o = ClbChannelOracle(spec, ChannelGrid(nl, nx, xi_in=xi[0], xi_out=xi[1]), 0.05, n_in=1.5, n_out=1.0)
    F0 = o.initial_state()
    F0 = F0 * perturbation(F0.shape, seed=31, amplitude=0.02)
    c = vlb.Channel(spec, vlb.VLB_FP64, nl, nx, 0.05, n_in=1.5, n_out=1.0, xi_in=xi[0], xi_out=xi[1])
    c.set_formulation(vlb.VLB_CARTESIAN)
    c.set_f(to_lib(F0))
    dt = 1e-3
    F1 = o.stage(1, dt, F0, F0)
    c.stage(dt, 1)
    assert rel_err(to_oracle(c.read_f(), nl, nx), F1) < 1e-12
    np.testing.assert_allclose(c.wall_density(), o.last_nw, rtol=1e-12, atol=0)
    F2 = o.stage(2, dt, F0, F1)
    c.stage(dt, 2)
    assert rel_err(to_oracle(c.read_f(), nl, nx), F2) < 1e-12
    F3 = o.stage(3, dt, F0, F2)
    c.stage(dt, 3)
    assert rel_err(to_oracle(c.read_f(), nl, nx), F3) < 1e-12
    c.close()


def test_fp32_moments_and_switching_back():
    spec, nl, nx = "HH(3;4)xHH(3;4)", 8, 12
    o = ClbChannelOracle(spec, ChannelGrid(nl, nx), 0.05)
    F0 = o.initial_state()
    F0 = F0 * perturbation(F0.shape, seed=32, amplitude=0.02)
    c = vlb.Channel(spec, vlb.VLB_FP32_BULK, nl, nx, 0.05)
    c.set_formulation(vlb.VLB_CARTESIAN)
    c.set_f(to_lib(F0).astype(np.float32))
    F = F0
    for _ in range(5):
        F = o.step(F, 1e-3)
    c.step_graph(1e-3, 3)
    c.step(1e-3, 2)
    n, ux, uy, T = (x.reshape(nx, nl).T for x in c.read_moments())
    on, oux, ouy, oT = o.moments(F)
    assert np.abs(n / on - 1).max() < 1e-5 and np.abs(T / oT - 1).max() < 1e-5
    assert np.abs(uy - ouy).max() < 1e-5
    # HH(3;4) on the xi axis has no vielbein kernel: the context runs only the Cartesian split
    e = vlb.Channel(spec, vlb.VLB_FP64, nl, nx, 0.05)
    for call in (lambda: e.step(1e-3, 1), lambda: e.set_formulation(vlb.VLB_CHI)):
        with pytest.raises(vlb.VlbError) as ei:
            call()
        assert ei.value.status == vlb.VLB_ERR_UNSUPPORTED
    e.close()
    # a velocity set with both: switch to the Cartesian split and back to the vielbein stage
    spec2 = "HH(4;8)xH(4;12)"
    o2 = ChannelOracle(spec2, ChannelGrid(nl, nx), 0.05)
    G0 = o2.initial_state()
    G0 = G0 * perturbation(G0.shape, seed=33, amplitude=0.02)
    d = vlb.Channel(spec2, vlb.VLB_FP64, nl, nx, 0.05)
    d.set_formulation(vlb.VLB_CARTESIAN)
    d.set_formulation(vlb.VLB_CHI)
    d.set_f(to_lib(G0))
    d.step(1e-3, 1)
    assert rel_err(to_oracle(d.read_f(), nl, nx), o2.step(G0, 1e-3)) < 1e-12
    d.set_formulation(vlb.VLB_CARTESIAN)
    for call, status in ((lambda: d.set_flow_rate(0.1), vlb.VLB_ERR_STATE), (lambda: d.postprocess(), vlb.VLB_ERR_STATE),
                         (lambda: d.set_formulation(vlb.VLB_FTILDE), vlb.VLB_ERR_UNSUPPORTED)):
        with pytest.raises(vlb.VlbError) as ei:
            call()
        assert ei.value.status == status
    c.close()
    d.close()


def test_shakhov_on_the_cartesian_split():
    """vlb_set_collision(VLB_SHAKHOV) on a Cartesian-split channel: the correction pass after each
    stage, against ClbChannelOracle(prandtl=2/3), FP64, three stages."""
    spec, nl, nx = "HH(3;4)xHH(3;4)", 7, 12
    o = ClbChannelOracle(spec, ChannelGrid(nl, nx), 0.05, n_in=1.5, n_out=1.0, prandtl=2.0 / 3.0)
    F0 = o.initial_state()
    F0 = F0 * perturbation(F0.shape, seed=34, amplitude=0.05)
    c = vlb.Channel(spec, vlb.VLB_FP64, nl, nx, 0.05, n_in=1.5, n_out=1.0)
    c.set_formulation(vlb.VLB_CARTESIAN)
    c.set_collision(vlb.VLB_SHAKHOV, 2.0 / 3.0)
    c.set_f(to_lib(F0))
    F = F0
    for k in (1, 2, 3):
        F = o.stage(k, 1e-3, F0, F)
        c.stage(1e-3, k)
        assert rel_err(to_oracle(c.read_f(), nl, nx), F) < 1e-12
    bgk = ClbChannelOracle(spec, ChannelGrid(nl, nx), 0.05, n_in=1.5, n_out=1.0).step(F0, 1e-3)
    assert rel_err(F, bgk) > 1e-9  # the heat-flux term is not negligible here
    c.close()


@pytest.mark.parametrize("spec,nl,nx", [("HH(4;8)xH(4;12)", 11, 12), ("HH(3;4)xH(3;4)", 13, 16),
                                      ("HH(4;8)xHH(4;6)", 9, 12)])
def test_marching_kernel_every_launch_shape(spec, nl, nx):
    """Velocity sets with a vielbein kernel run the Cartesian split on the same march (the
    geometry records read as V^lambda per face, no force, fluxes of F): every launch shape
    against the oracle, FP64 over three stages with n_w per column, FP32 moments after one step."""
    o = ClbChannelOracle(spec, ChannelGrid(nl, nx), 0.05, n_in=1.5, n_out=1.0)
    F0 = o.initial_state()
    F0 = F0 * perturbation(F0.shape, seed=35, amplitude=0.03)
    dt = 1e-3
    F1 = o.stage(1, dt, F0, F0)
    nw1 = o.last_nw.copy()
    F2 = o.stage(2, dt, F0, F1)
    F3 = o.stage(3, dt, F0, F2)
    on, oux, ouy, oT = o.moments(F3)
    c = vlb.Channel(spec, vlb.VLB_FP64, nl, nx, 0.05, n_in=1.5, n_out=1.0)
    c.set_formulation(vlb.VLB_CARTESIAN)
    d = vlb.Channel(spec, vlb.VLB_FP32_BULK, nl, nx, 0.05, n_in=1.5, n_out=1.0)
    d.set_formulation(vlb.VLB_CARTESIAN)
    nvar = len(c.channel_variants())
    assert nvar >= 2
    assert len(d.channel_variants()) >= 1
    for v in range(nvar):
        c.set_variant(v)
        c.set_f(to_lib(F0))
        c.stage(dt, 1)
        assert rel_err(to_oracle(c.read_f(), nl, nx), F1) < 1e-12, v
        np.testing.assert_allclose(c.wall_density(), nw1, rtol=1e-12, atol=0)
        c.stage(dt, 2)
        c.stage(dt, 3)
        assert rel_err(to_oracle(c.read_f(), nl, nx), F3) < 1e-12, v
        d.set_variant(v % len(d.channel_variants()))
        d.set_f(to_lib(F0).astype(np.float32))
        d.step(dt, 1)
        n, ux, uy, T = (x.reshape(nx, nl).T for x in d.read_moments())
        assert np.abs(n / on - 1).max() < 1e-5 and np.abs(T / oT - 1).max() < 1e-5, v
        assert np.abs(ux - oux).max() < 1e-5 and np.abs(uy - ouy).max() < 1e-5, v
    c.close()
    d.close()


def test_shakhov_on_the_marching_cartesian_split():
    spec, nl, nx = "HH(4;8)xH(4;12)", 9, 12
    o = ClbChannelOracle(spec, ChannelGrid(nl, nx), 0.05, n_in=1.5, n_out=1.0, prandtl=2.0 / 3.0)
    F0 = o.initial_state()
    F0 = F0 * perturbation(F0.shape, seed=36, amplitude=0.05)
    c = vlb.Channel(spec, vlb.VLB_FP64, nl, nx, 0.05, n_in=1.5, n_out=1.0)
    c.set_formulation(vlb.VLB_CARTESIAN)
    c.set_collision(vlb.VLB_SHAKHOV, 2.0 / 3.0)
    c.set_f(to_lib(F0))
    F = F0
    for k in (1, 2, 3):
        F = o.stage(k, 1e-3, F0, F)
        c.stage(1e-3, k)
        assert rel_err(to_oracle(c.read_f(), nl, nx), F) < 1e-12
    c.close()
