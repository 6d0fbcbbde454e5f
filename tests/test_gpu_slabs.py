"""Radial slabs on the GPU: Couette contexts holding cells [begin, end) of one grid, their
halo ends filled with vlb_read_edge / vlb_write_halo before every stage, step bitwise as
the whole grid does (the stage kernel's result does not depend on how cells are cut into
tiles), and against the oracle's slab path.  Several slabs live in one process here; the
rank-to-rank exchange itself is covered on the CPU (tests/test_slabs_cpu.py)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle.couette import CouetteOracle, Wall  # noqa: E402
from paper_1708_05944_gb300 import vlb  # noqa: E402
from paper_1708_05944_gb300.slabs import LibrarySlab, slab_bounds  # noqa: E402
from tests.helpers import make_case, rel_err, to_lib, to_oracle  # noqa: E402

CONFIG1 = "HH(3;4)xH(3;4)"
CONFIG2 = "HH(4;8)xH(4;20)"
WIN, WOUT = (0.15, 1.0), (-0.05, 1.1)


def contexts(spec, prec, grid, bounds, F0):
    dtype = np.float64 if prec == vlb.VLB_FP64 else np.float32
    out = []
    for b, e in bounds:
        c = vlb.Couette(spec, prec, [dict(grid, cell_begin=b, cell_end=e)], [WIN], [WOUT], [0.2], [1])
        c.set_f(to_lib(F0[:, b:e]).astype(dtype))
        out.append(c)
    return out


def exchange(slabs, on_device):
    """Each slab's edge blocks into its neighbours' halos (host or device buffers)."""
    nb = slabs[0].halo_bytes()
    buf = (lambda: torch.empty(nb, dtype=torch.uint8, device="cuda")) if on_device else (
        lambda: np.empty(nb, dtype=np.uint8))
    edges = [(c.read_edge(0, 0, buf()), c.read_edge(0, 1, buf())) for c in slabs]
    for r, c in enumerate(slabs):
        if r > 0:
            c.write_halo(0, 0, edges[r - 1][1])
        if r < len(slabs) - 1:
            c.write_halo(0, 1, edges[r + 1][0])


def run(slabs, dt, steps, on_device=False):
    for _ in range(steps):
        for k in (1, 2, 3):
            exchange(slabs, on_device)
            for c in slabs:
                c.stage(dt, k)


@pytest.mark.parametrize("prec", [vlb.VLB_FP64, vlb.VLB_FP32_BULK])
@pytest.mark.parametrize("spec,n,parts,A", [(CONFIG1, 32, 2, 0.0), (CONFIG2, 64, 3, 0.95), (CONFIG2, 47, 4, 0.0)])
def test_slabs_step_bitwise_as_the_whole_grid(prec, spec, n, parts, A):
    o, F0, grid = make_case(spec, n, u_in=WIN[0], u_out=WOUT[0], T_out=WOUT[1], kn=0.2, A=A)
    dtype = np.float64 if prec == vlb.VLB_FP64 else np.float32
    dt = 5e-4
    full = vlb.Couette(spec, prec, [grid], [WIN], [WOUT], [0.2], [1])
    full.set_f(to_lib(F0).astype(dtype))
    full.step(dt, 5)
    slabs = contexts(spec, prec, grid, slab_bounds(n, parts), F0)
    run(slabs, dt, 5, on_device=(parts == 3))
    got = np.concatenate([c.read_f() for c in slabs], axis=0)
    assert np.array_equal(got, full.read_f())
    nw_full = full.wall_density()[0]
    assert slabs[0].wall_density()[0][0] == nw_full[0] and slabs[-1].wall_density()[0][1] == nw_full[1]
    assert slabs[0].wall_density()[0][1] == 0.0  # a halo end has no wall
    for c in slabs + [full]:
        c.close()


def test_slabs_match_the_oracle_slab_path():
    spec, n = CONFIG1, 30
    o, F0, grid = make_case(spec, n, u_in=WIN[0], u_out=WOUT[0], T_out=WOUT[1], kn=0.2, A=0.9)
    bounds = slab_bounds(n, 3)
    slabs = contexts(spec, vlb.VLB_FP64, grid, bounds, F0)
    dt = 1e-3
    os_ = [CouetteOracle(spec, o.g.slab(b, e), Wall(*WIN), Wall(*WOUT), 0.2, 1) for b, e in bounds]
    Fl = [F0[:, b:e].copy() for b, e in bounds]
    Fin = list(Fl)
    for k in (1, 2, 3):
        for r, oo in enumerate(os_):
            oo.set_halo(Fin[r - 1][:, -3:] if r > 0 else None, Fin[r + 1][:, :3] if r < 2 else None)
        Fin = [oo.stage(k, dt, Fl[r], Fin[r]) for r, oo in enumerate(os_)]
    run(slabs, dt, 1)
    for r, c in enumerate(slabs):
        assert rel_err(to_oracle(c.read_f()), Fin[r]) < 1e-13
    for c in slabs:
        c.close()


def test_residual_sums_add_up_over_slabs():
    spec, n = CONFIG2, 48
    o, F0, grid = make_case(spec, n, u_in=WIN[0], u_out=WOUT[0], T_out=WOUT[1], kn=0.2)
    full = vlb.Couette(spec, vlb.VLB_FP64, [grid], [WIN], [WOUT], [0.2], [1])
    full.set_f(to_lib(F0))
    slabs = contexts(spec, vlb.VLB_FP64, grid, slab_bounds(n, 3), F0)
    full.residual()
    for c in slabs:
        c.residual_sums()
    full.step(5e-4, 4)
    run(slabs, 5e-4, 4)
    ref = np.array(full.residual()).ravel()
    tot = np.sum([np.array(c.residual_sums()).ravel() for c in slabs], axis=0)
    np.testing.assert_allclose(np.sqrt(tot), ref, rtol=1e-12)
    for c in slabs + [full]:
        c.close()


def test_slab_contexts_refuse_whole_steps_and_wall_halos():
    spec, n = CONFIG1, 20
    o, F0, grid = make_case(spec, n)
    a, b = contexts(spec, vlb.VLB_FP64, grid, [(0, 10), (10, 20)], F0)
    for call in (lambda: a.step(1e-3, 1), lambda: a.step_graph(1e-3, 3), lambda: a.run_to_steady(1e-3, 10, 1e-6, 20)):
        with pytest.raises(vlb.VlbError) as ei:
            call()
        assert ei.value.status == vlb.VLB_ERR_STATE
    with pytest.raises(vlb.VlbError) as ei:
        a.write_halo(0, 0, np.zeros(a.halo_bytes(), dtype=np.uint8))  # the inner end of slab 0 is the wall
    assert ei.value.status == vlb.VLB_ERR_STATE
    with pytest.raises(vlb.VlbError):
        vlb.Couette(spec, vlb.VLB_FP64, [dict(grid, cell_begin=18, cell_end=20)], [WIN], [WOUT], [0.2], [1])
    a.close()
    b.close()


def test_library_slab_runner_on_one_rank():
    """SlabRunner over LibrarySlab with a one-rank gloo group: the whole grid as one slab
    (no exchange), stepped and reduced through the same host path the ranks use."""
    import os
    import socket
    import torch.distributed as dist
    from paper_1708_05944_gb300.slabs import HaloExchange, SlabRunner
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        spec, n = CONFIG1, 24
        o, F0, grid = make_case(spec, n, u_in=WIN[0], u_out=WOUT[0], T_out=WOUT[1], kn=0.2)
        ls = LibrarySlab(spec, vlb.VLB_FP64, grid, WIN, WOUT, 0.2, 1, 0, n, on_device=False)
        ls.ctx.set_f(to_lib(F0))
        runner = SlabRunner(ls, HaloExchange(0, 1))
        runner.residual()
        runner.step(1e-3, 3)
        res = runner.residual()
        full = vlb.Couette(spec, vlb.VLB_FP64, [grid], [WIN], [WOUT], [0.2], [1])
        full.set_f(to_lib(F0))
        full.residual()
        full.step(1e-3, 3)
        assert np.array_equal(ls.ctx.read_f(), full.read_f())
        np.testing.assert_allclose(res, np.array(full.residual()).ravel(), rtol=1e-14)
        ls.close()
        full.close()
    finally:
        dist.destroy_process_group()
