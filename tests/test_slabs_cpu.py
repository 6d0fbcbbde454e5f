"""Radial slab decomposition on the CPU: the oracle's slab path (halo ghosts at the
ends that are not walls) against the whole grid, and the host logic of
paper_1708_05944_gb300.slabs (cutting, point-to-point halo exchange over gloo
ranks, the all-reduced residual) driving oracle slabs: every rank's cells are
bitwise those of the single-rank run."""
import math
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle.couette import TAU_AOKI, CouetteGrid, CouetteOracle, Wall  # noqa: E402
from paper_1708_05944_gb300.inputs import perturbation  # noqa: E402
from paper_1708_05944_gb300.slabs import slab_bounds  # noqa: E402

SPEC = "HH(3;4)xH(3;4)"
N, DT, STEPS = 20, 1e-3, 6
WALLS = (Wall(0.2, 1.0), Wall(-0.05, 1.1))


def whole(A):
    return CouetteOracle(SPEC, CouetteGrid(N, 1.0, 2.0, A=A), *WALLS, 0.3, TAU_AOKI)


def start(o):
    F = o.initial_equilibrium()
    return F * perturbation(F.shape, seed=31)


class OracleSlab:
    """One rank's slab on the oracle, with the interface of slabs.LibrarySlab: edge
    blocks are float64 tensors (2, 3, nq0, nq1) of the next stage's input."""

    def __init__(self, A, begin, end, F0):
        g = CouetteGrid(N, 1.0, 2.0, A=A).slab(begin, end)
        self.o = CouetteOracle(SPEC, g, *WALLS, 0.3, TAU_AOKI)
        self.F_l = F0[:, begin:end].copy()
        self.F_in = self.F_l  # what the next stage reads as F_prev
        self.halo = [None, None]
        self.prev_mom = None

    def read_edge(self, end):
        blk = self.F_in[:, 0:3] if end == 0 else self.F_in[:, -3:]
        return torch.from_numpy(np.ascontiguousarray(blk))

    def write_halo(self, end, rows):
        self.halo[end] = rows.numpy()

    def stage(self, dt, k):
        self.o.set_halo(*self.halo)
        out = self.o.stage(k, dt, self.F_l, self.F_in)
        if k == 3:
            self.F_l = out
        self.F_in = out

    def residual_sums(self):
        mom = self.o.m.moments(self.F_in)
        if self.prev_mom is None:
            self.prev_mom = mom
            return [0.0, 0.0, 0.0]
        n1, _, u1, T1 = mom
        n0, _, u0, T0 = self.prev_mom
        w = self.o.g.wres
        uw = WALLS[0].u_tangential
        self.prev_mom = mom
        return [float((w * ((u1 - u0) / uw) ** 2).sum()), float((w * (n1 / n0 - 1.0) ** 2).sum()),
                float((w * (T1 / T0 - 1.0) ** 2).sum())]


def test_slab_bounds():
    assert slab_bounds(20, 3) == [(0, 7), (7, 14), (14, 20)]
    assert slab_bounds(9, 3) == [(0, 3), (3, 6), (6, 9)]
    for n, w in ((1024, 8), (37, 5), (3, 1)):
        b = slab_bounds(n, w)
        assert b[0][0] == 0 and b[-1][1] == n and all(e - s >= 3 for s, e in b)
        assert all(b[i][1] == b[i + 1][0] for i in range(w - 1))
    with pytest.raises(ValueError):
        slab_bounds(8, 3)


@pytest.mark.parametrize("A", [0.0, 0.9])
def test_oracle_slabs_step_as_the_whole_grid(A):
    """Three slabs exchanging halos in one process, against the whole grid: bitwise,
    n_w included (each wall belongs to the slab that holds it)."""
    o = whole(A)
    F0 = start(o)
    F = F0
    for _ in range(STEPS):
        F = o.step(F, DT)
    slabs = [OracleSlab(A, b, e, F0) for b, e in slab_bounds(N, 3)]
    for _ in range(STEPS):
        for k in (1, 2, 3):
            edges = [(s.read_edge(0), s.read_edge(1)) for s in slabs]
            for r, s in enumerate(slabs):
                if r > 0:
                    s.write_halo(0, edges[r - 1][1])
                if r < 2:
                    s.write_halo(1, edges[r + 1][0])
            for s in slabs:
                s.stage(DT, k)
    got = np.concatenate([s.F_in for s in slabs], axis=1)
    assert np.array_equal(got, F)
    assert slabs[0].o.last_nw[0] == o.last_nw[0] and slabs[-1].o.last_nw[1] == o.last_nw[1]


def test_a_shifted_halo_is_caught():
    """The decomposition test can fail: ghosts taken one cell off change the result."""
    o = whole(0.0)
    F0 = start(o)
    ref = o.step(F0, DT)
    a, b = OracleSlab(0.0, 0, 10, F0), OracleSlab(0.0, 10, N, F0)
    for k in (1, 2, 3):
        a.write_halo(1, torch.from_numpy(np.ascontiguousarray(b.F_in[:, 1:4])))  # one cell too far
        b.write_halo(0, a.read_edge(1))
        a.stage(DT, k)
        b.stage(DT, k)
    assert not np.array_equal(np.concatenate([a.F_in, b.F_in], axis=1), ref)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, A, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1708_05944_gb300.slabs import HaloExchange, SlabRunner, slab_bounds
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        o = whole(A)
        b, e = slab_bounds(N, world)[rank]
        run = SlabRunner(OracleSlab(A, b, e, start(o)), HaloExchange(rank, world))
        run.residual()  # stores the starting moments
        run.step(DT, STEPS)
        res = run.residual()
        q.put((rank, b, e, run.slab.F_in, res, run.slab.o.last_nw, run.messages))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,A", [(2, 0.0), (3, 0.9)])
def test_gloo_ranks_step_as_one(world, A):
    """world gloo ranks, one slab each, halos exchanged by HaloExchange before every
    stage: the assembled state equals the single-rank run bitwise, each wall's n_w comes
    from the rank that holds it, and the all-reduced residual equals the whole grid's
    (the sums are added in another order, so to rounding)."""
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, A, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    o = whole(A)
    F0 = start(o)
    F = F0
    for _ in range(STEPS):
        F = o.step(F, DT)
    assembled = np.concatenate([g[3] for g in got], axis=1)
    assert np.array_equal(assembled, F)
    assert got[0][5][0] == o.last_nw[0] and got[-1][5][1] == o.last_nw[1]
    # each inner boundary: two blocks received per stage (one per side)
    assert sum(g[6] for g in got) == 2 * (world - 1) * 3 * STEPS
    ref = o.residual(o.m.moments(F), o.m.moments(F0), WALLS[0].u_tangential)
    for g in got:
        assert g[4] == pytest.approx(ref, rel=1e-12)
    assert all(math.isfinite(x) for x in got[0][4])
