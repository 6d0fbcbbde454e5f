"""GPU parity of the chi-formulation Couette RK3 stage (libvlb through the C ABI)
against the fp64 CPU oracle on the same seeded inputs.

Tolerances: FP64 path 1e-10 relative (single stages 1e-13); FP32-bulk path
1e-5 relative on the moments n, u, T.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1708_05944_gb300 import vlb  # noqa: E402
from paper_1708_05944_gb300.inputs import perturbation  # noqa: E402
from tests.helpers import make_case, rel_err, to_lib, to_oracle  # noqa: E402

CONFIG1 = "HH(3;4)xH(3;4)"
CONFIG2 = "HH(4;8)xH(4;20)"


def ctx_for(spec, prec, grids, walls_in, walls_out, kns, modes):
    return vlb.Couette(spec, prec, grids, walls_in, walls_out, kns, modes)


@pytest.mark.parametrize("spec,n", [(CONFIG1, 32), (CONFIG2, 37), ("H(4;5)xH(4;5)", 19), ("HH(2;3)xH(3;4)", 3)])
@pytest.mark.parametrize("A", [0.0, 0.95])
def test_fp64_stages_match_oracle(spec, n, A):
    o, F0, grid = make_case(spec, n, u_in=0.1, u_out=-0.05, T_out=1.05, kn=0.1, A=A)
    c = ctx_for(spec, vlb.VLB_FP64, [grid], [(0.1, 1.0)], [(-0.05, 1.05)], [0.1], [1])
    dt = 1e-3
    c.set_f(to_lib(F0))
    F1 = o.stage(1, dt, F0, F0)
    c.stage(dt, 1)
    assert rel_err(to_oracle(c.read_f()), F1) < 1e-13
    nw = c.wall_density()[0]
    assert abs(nw[0] - o.last_nw[0]) < 1e-13 and abs(nw[1] - o.last_nw[1]) < 1e-13
    F2 = o.stage(2, dt, F0, F1)
    c.stage(dt, 2)
    assert rel_err(to_oracle(c.read_f()), F2) < 1e-13
    F3 = o.stage(3, dt, F0, F2)
    c.stage(dt, 3)
    assert rel_err(to_oracle(c.read_f()), F3) < 1e-13
    c.close()


def test_fp64_many_steps_config1():
    o, F0, grid = make_case(CONFIG1, 32)
    c = ctx_for(CONFIG1, vlb.VLB_FP64, [grid], [(0.1, 1.0)], [(0.0, 1.0)], [0.1], [1])
    c.set_f(to_lib(F0))
    F = F0
    for _ in range(150):
        F = o.step(F, 1e-3)
    c.step(1e-3, 150)
    assert rel_err(to_oracle(c.read_f()), F) < 1e-10
    n, u0, u1, T = c.read_moments()
    on, ou0, ou1, oT = o.m.moments(F)
    assert np.abs(n / on - 1).max() < 1e-10 and np.abs(T / oT - 1).max() < 1e-10
    c.close()


@pytest.mark.parametrize("kn", [1e-3, 1.0, 10.0])
def test_fp64_config2_full_size_stage(kn):
    o, F0, grid = make_case(CONFIG2, 1024, kn=kn, tau_mode=1)
    c = ctx_for(CONFIG2, vlb.VLB_FP64, [grid], [(0.1, 1.0)], [(0.0, 1.0)], [kn], [1])
    c.set_f(to_lib(F0))
    dt = 5e-5
    F1 = o.stage(1, dt, F0, F0)
    c.stage(dt, 1)
    assert rel_err(to_oracle(c.read_f()), F1) < 1e-12
    c.close()


@pytest.mark.parametrize("kn", [1e-3, 0.1, 10.0])
def test_fp32_bulk_moments_config2(kn):
    o, F0, grid = make_case(CONFIG2, 1024, kn=kn, tau_mode=1)
    c = ctx_for(CONFIG2, vlb.VLB_FP32_BULK, [grid], [(0.1, 1.0)], [(0.0, 1.0)], [kn], [1])
    c.set_f(to_lib(F0).astype(np.float32))
    dt = 5e-5
    F = F0
    for _ in range(4):
        F = o.step(F, dt)
    c.step(dt, 4)
    n, u0, u1, T = c.read_moments()
    on, ou0, ou1, oT = o.m.moments(F)
    assert np.abs(n / on - 1).max() < 1e-5
    assert np.abs(T / oT - 1).max() < 1e-5
    assert np.abs(u1 - ou1).max() < 1e-5 * max(1.0, np.abs(ou1).max())
    assert np.abs(u0 - ou0).max() < 1e-5
    c.close()


def test_batched_instances_equal_single_runs():
    # uneven instance sizes (tile remainders, the 3-cell minimum) in one context
    specs = [dict(n=37, u=0.1, kn=0.1, ro=2.0), dict(n=3, u=0.3, kn=1.0, ro=1.5),
             dict(n=16, u=0.05, kn=0.01, ro=3.0), dict(n=17, u=0.2, kn=10.0, ro=4.0)]
    cases = [make_case(CONFIG1, s["n"], u_in=s["u"], kn=s["kn"], r_out=s["ro"], seed=100 + k)
             for k, s in enumerate(specs)]
    c = ctx_for(CONFIG1, vlb.VLB_FP64, [g for _, _, g in cases], [(s["u"], 1.0) for s in specs],
                [(0.0, 1.0)] * 4, [s["kn"] for s in specs], [1] * 4)
    c.set_f(np.concatenate([to_lib(F0) for _, F0, _ in cases]))
    c.step(1e-3, 5)
    got = c.read_f()
    off = 0
    for (o, F0, g), s in zip(cases, specs):
        F = F0
        for _ in range(5):
            F = o.step(F, 1e-3)
        assert rel_err(to_oracle(got[off:off + s["n"]]), F) < 1e-12
        off += s["n"]
    c.close()


def test_rest_state_and_mass_on_gpu():
    spec = CONFIG2
    o, F0, grid = make_case(spec, 64, u_in=0.0, amplitude=0.0)
    c = ctx_for(spec, vlb.VLB_FP64, [grid], [(0.0, 1.0)], [(0.0, 1.0)], [0.1], [1])
    c.init_equilibrium()
    ref = c.read_f()
    c.step(1e-4, 20)
    assert rel_err(c.read_f(), ref) < 1e-13
    # moving wall: particle number conserved to round-off
    c.set_walls([(0.3, 1.0)], [(0.0, 1.0)])
    c.step(1e-4, 200)
    F = to_oracle(c.read_f())
    assert abs(o.n_tot(F) / o.n_tot(to_oracle(ref)) - 1) < 1e-12
    c.close()


def test_save_load_continues_bitwise(tmp_path):
    o, F0, grid = make_case(CONFIG1, 32)
    c = ctx_for(CONFIG1, vlb.VLB_FP32_BULK, [grid], [(0.1, 1.0)], [(0.0, 1.0)], [0.1], [1])
    c.set_f(to_lib(F0).astype(np.float32))
    c.step(1e-3, 10)
    p = str(tmp_path / "state.vlb")
    c.save(p)
    c.step(1e-3, 10)
    a = c.read_f().copy()
    c.load(p)
    c.step(1e-3, 10)
    assert np.array_equal(a, c.read_f())
    c.close()


def test_kernel_launch_count():
    o, F0, grid = make_case(CONFIG1, 32)
    c = ctx_for(CONFIG1, vlb.VLB_FP64, [grid], [(0.1, 1.0)], [(0.0, 1.0)], [0.1], [1])
    c.step(1e-3, 7)
    assert c.kernel_launches() == 21
    c.close()


@pytest.mark.parametrize("prec", [vlb.VLB_FP64, vlb.VLB_FP32_BULK])
def test_every_launch_shape_matches_oracle(prec):
    # 37 cells: a remainder tile for every tile size; two instances
    cases = [make_case(CONFIG2, 37, u_in=0.2, kn=0.05, seed=9), make_case(CONFIG2, 21, u_in=0.1, kn=2.0, seed=10)]
    c = ctx_for(CONFIG2, prec, [g for _, _, g in cases], [(0.2, 1.0), (0.1, 1.0)], [(0.0, 1.0)] * 2, [0.05, 2.0],
                [1, 1])
    dtype = np.float64 if prec == vlb.VLB_FP64 else np.float32
    f0 = np.concatenate([to_lib(F0) for _, F0, _ in cases]).astype(dtype)
    refs = []
    for o, F0, _ in cases:
        F = F0
        for _ in range(2):
            F = o.step(F, 1e-4)
        refs.append(F)
    shapes = c.variants()
    assert len(shapes) >= 1
    for v in range(len(shapes)):
        c.set_variant(v)
        c.set_f(f0)
        c.step(1e-4, 2)
        got = c.read_f()
        off = 0
        for (o, F0, g), ref in zip(cases, refs):
            n = g["n_cells"]
            if prec == vlb.VLB_FP64:
                assert rel_err(to_oracle(got[off:off + n]), ref) < 1e-12, shapes[v]
            else:
                c_n = to_oracle(got[off:off + n]).astype(np.float64)
                on = o.m.moments(ref)[0]
                assert np.abs(o.m.moments(c_n)[0] / on - 1).max() < 1e-5, shapes[v]
            off += n
    best, ms = c.autotune(1e-4, reps=5)
    assert 0 <= best < len(shapes) and ms > 0
    c.close()


def test_knudsen_set_after_creation():
    o, F0, grid = make_case("HH(3;4)xH(3;4)", 24, kn=2.0, tau_mode=vlb.VLB_TAU_KN_OVER_NT)
    c = vlb.Couette("HH(3;4)xH(3;4)", vlb.VLB_FP64, [grid], [(0.1, 1.0)], [(0.0, 1.0)], [0.1], [vlb.VLB_TAU_AOKI])
    c.set_knudsen(2.0, vlb.VLB_TAU_KN_OVER_NT)
    c.set_f(to_lib(F0))
    dt = 1e-3
    c.stage(dt, 1)
    F1 = o.stage(1, dt, F0, F0)
    assert rel_err(to_oracle(c.read_f()), F1) < 1e-13
    with pytest.raises(vlb.VlbError):
        c.set_knudsen(0.0)
    with pytest.raises(vlb.VlbError):
        vlb._check(vlb._lib.vlb_set_channel_reservoirs(c.h, 2.0, 1.0, 1.0), c.h)
    c.close()


def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


def test_fp64_config1_ten_thousand_steps():
    # the whole configured run: 32 cells, HH(3;4)xH(3;4), Kn = 0.1, dt = 1e-3, 10^4 steps, against
    # the oracle's run (tests/golden/make_oracle_references.py); 1e-10 relative
    ref = _golden("couette_config1_10000_steps.json")
    o, F0, grid = make_case(CONFIG1, 32)
    c = ctx_for(CONFIG1, vlb.VLB_FP64, [grid], [(0.1, 1.0)], [(0.0, 1.0)], [0.1], [1])
    c.set_f(to_lib(F0))
    c.step_graph(1e-3, 10000)
    assert rel_err(to_oracle(c.read_f()), np.asarray(ref["F"])) < 1e-10
    n, u0, u1, T = c.read_moments()
    assert np.abs(n / np.asarray(ref["n"]) - 1).max() < 1e-10
    assert np.abs(T / np.asarray(ref["T"]) - 1).max() < 1e-10
    assert np.abs(u1 - np.asarray(ref["u1"])).max() < 1e-10 * 0.1
    c.close()


@pytest.mark.parametrize("kn", [1e-3, 0.1, 10.0])
def test_fp32_bulk_one_stage_and_hundred_steps(kn):
    # FP32-bulk storage and stencil arithmetic against the FP64 oracle: moments within 1e-5
    # after a single stage and after 100 steps (64 cells of the scale-up model)
    o, F0, grid = make_case(CONFIG2, 64, kn=kn, tau_mode=1, u_in=0.2)
    dt = 5e-4 if kn > 1e-2 else 1e-4
    c = ctx_for(CONFIG2, vlb.VLB_FP32_BULK, [grid], [(0.2, 1.0)], [(0.0, 1.0)], [kn], [1])
    c.set_f(to_lib(F0).astype(np.float32))
    F1 = o.stage(1, dt, F0, F0)
    c.stage(dt, 1)

    def check(F):
        n, u0, u1, T = c.read_moments()
        on, ou0, ou1, oT = o.m.moments(F)
        assert np.abs(n / on - 1).max() < 1e-5
        assert np.abs(T / oT - 1).max() < 1e-5
        assert np.abs(u0 - ou0).max() < 1e-5 and np.abs(u1 - ou1).max() < 1e-5

    check(F1)
    c.stage(dt, 2)
    c.stage(dt, 3)
    F = o.step(F0, dt)
    for _ in range(99):
        F = o.step(F, dt)
    c.step(dt, 99)
    check(F)
    c.close()


def test_fp32_bulk_steady_state():
    # the steady state of a small instance of the scale-up model, FP32 bulk against the
    # oracle's (tests/golden/make_oracle_references.py): moments within 1e-5
    ref = _golden("couette_steady_16x320.json")
    grid = dict(n_cells=16, r_in=1.0, r_out=2.0, stretch_A=0.0, stretch_delta=0.5)
    c = ctx_for(CONFIG2, vlb.VLB_FP32_BULK, [grid], [(0.2, 1.0)], [(0.0, 1.0)], [0.1], [1])
    c.init_equilibrium()
    c.step_graph(ref["dt"], ref["steps"])
    n, u0, u1, T = c.read_moments()
    assert np.abs(n / np.asarray(ref["n"]) - 1).max() < 1e-5
    assert np.abs(T / np.asarray(ref["T"]) - 1).max() < 1e-5
    assert np.abs(u1 - np.asarray(ref["u1"])).max() < 1e-5
    assert np.abs(u0 - np.asarray(ref["u0"])).max() < 1e-5
    c.close()


def plateau_input(o, seed, run=4, amplitude=0.02):
    """Equilibrium populations times 1 + amplitude * a_ij * k(s), with a_ij = +-1 drawn from the
    seeded generator and k(s) piecewise constant in runs of `run` cells: every five-point stencil
    holds at most one jump, so its indicators vanish in every combination of Table IV (one, two
    or all three), in either precision."""
    F = o.initial_equilibrium()
    a = np.sign(perturbation(F.shape[2:], seed=seed, amplitude=1.0) - 1.0)
    k = ((np.arange(F.shape[1]) // run) % 3 - 1).astype(np.float64)
    return F * (1.0 + amplitude * a[None, None] * k[None, :, None, None])


@pytest.mark.parametrize("prec", [vlb.VLB_FP64, vlb.VLB_FP32_BULK])
def test_table_iv_rows(prec):
    spec, n = CONFIG2, 40
    o, _, grid = make_case(spec, n, kn=0.3, tau_mode=1, u_in=0.15)
    F0 = plateau_input(o, seed=77)
    c = ctx_for(spec, prec, [grid], [(0.15, 1.0)], [(0.0, 1.0)], [0.3], [1])
    dtype = np.float64 if prec == vlb.VLB_FP64 else np.float32
    c.set_f(to_lib(F0).astype(dtype))
    dt = 4e-4
    F = o.step(F0, dt)
    c.step(dt, 1)
    got = to_oracle(c.read_f())
    if prec == vlb.VLB_FP64:
        assert rel_err(got, F) < 1e-13
    else:
        assert rel_err(got, F) < 1e-6
        n_, u0, u1, T = c.read_moments()
        on, ou0, ou1, oT = o.m.moments(F)
        assert np.abs(n_ / on - 1).max() < 1e-6 and np.abs(T / oT - 1).max() < 1e-6
    c.close()


def test_kn_over_n_relaxation_time():
    # tau = Kn / n (vlb_tau_mode 2), three stages against the oracle
    o, F0, grid = make_case(CONFIG1, 20, kn=0.05, tau_mode=2, u_in=0.1)
    c = ctx_for(CONFIG1, vlb.VLB_FP64, [grid], [(0.1, 1.0)], [(0.0, 1.0)], [0.05], [2])
    c.set_f(to_lib(F0))
    dt = 1e-3
    F = o.step(F0, dt)
    c.step(dt, 1)
    assert rel_err(to_oracle(c.read_f()), F) < 1e-13
    c.close()
