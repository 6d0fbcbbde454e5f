"""Radial slab decomposition of a circular Couette instance over ranks.

The cells of one radial grid (Sec. VI.A.1) are cut into contiguous slabs, one
per rank.  A stage of Eq. (rk3) needs, at each cell, the WENO-5 stencils of
Sec. III.C, which reach three cells across an interface; everything else in
the stage (moments, equilibrium, force, relaxation) is local to the cell.  So
before every stage each rank sends the three cells at each inner end of its
slab to the neighbour on that side and writes the three it receives into its
halo; the diffuse-wall density n_w (Eq. nw) is computed by the rank whose slab
holds the wall, from its own cells.  The steady-state norms of Eq.
(msites_steady) are sums over cells: the ranks add their sums of squares (one
all-reduce of three numbers per instance) before the square root.

`slab_bounds` cuts the grid, `HaloExchange` moves the three-cell blocks with
torch.distributed point-to-point messages (gloo: host tensors, nccl: device
tensors), `SlabRunner` drives one rank, and `LibrarySlab` is a rank's slab as
a library context (vlb_couette_grid with cell_begin / cell_end).  A runner
takes any slab object with the methods of `LibrarySlab`.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def slab_bounds(n_cells: int, world: int):
    """[(begin, end)] of `world` contiguous slabs of n_cells cells, sizes differing by at
    most one, each at least three cells (the wall extrapolation and the three-cell halo)."""
    if world < 1 or n_cells < 3 * world:
        raise ValueError(f"{n_cells} cells cannot be cut into {world} slabs of at least 3 cells")
    base, extra = divmod(n_cells, world)
    out, b = [], 0
    for r in range(world):
        e = b + base + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


class HaloExchange:
    """Point-to-point exchange of edge blocks between ranks r - 1, r, r + 1 of a group."""

    def __init__(self, rank: int, world: int, group=None):
        self.rank, self.world, self.group = rank, world, group

    def _peer(self, r):
        return r if self.group is None else dist.get_global_rank(self.group, r)

    def exchange(self, lo_edge, hi_edge):
        """Send lo_edge to rank - 1 and hi_edge to rank + 1; return the blocks received
        from them (lo_halo from rank - 1, hi_halo from rank + 1; None at the ends)."""
        reqs, lo_halo, hi_halo = [], None, None
        if self.rank > 0:
            lo_halo = torch.empty_like(lo_edge)
            reqs.append(dist.isend(lo_edge, self._peer(self.rank - 1), group=self.group))
            reqs.append(dist.irecv(lo_halo, self._peer(self.rank - 1), group=self.group))
        if self.rank < self.world - 1:
            hi_halo = torch.empty_like(hi_edge)
            reqs.append(dist.isend(hi_edge, self._peer(self.rank + 1), group=self.group))
            reqs.append(dist.irecv(hi_halo, self._peer(self.rank + 1), group=self.group))
        for q in reqs:
            q.wait()
        return lo_halo, hi_halo


class SlabRunner:
    """One rank's slab: halo exchange before each stage, residual norms over all ranks."""

    def __init__(self, slab, exchange: HaloExchange):
        self.slab, self.ex = slab, exchange
        self.messages = 0  # blocks sent so far

    def stage(self, dt: float, k: int):
        lo = self.slab.read_edge(0) if self.ex.rank > 0 else None
        hi = self.slab.read_edge(1) if self.ex.rank < self.ex.world - 1 else None
        lo_halo, hi_halo = self.ex.exchange(lo, hi)
        if lo_halo is not None:
            self.slab.write_halo(0, lo_halo)
            self.messages += 1
        if hi_halo is not None:
            self.slab.write_halo(1, hi_halo)
            self.messages += 1
        self.slab.stage(dt, k)

    def step(self, dt: float, nsteps: int = 1):
        for _ in range(nsteps):
            for k in (1, 2, 3):
                self.stage(dt, k)

    def residual(self):
        """(L2_u, L2_n, L2_T) of Eq. (msites_steady) over the whole grid (every rank gets
        them): the ranks' sums of squares added by one all-reduce, then the square root."""
        s = torch.tensor(np.asarray(self.slab.residual_sums(), dtype=np.float64).reshape(3))
        dist.all_reduce(s, op=dist.ReduceOp.SUM, group=self.ex.group)
        return tuple(float(x) for x in torch.sqrt(s))


class LibrarySlab:
    """A rank's slab of one Couette instance as a library context.  Edge blocks are
    device tensors (nccl) or pinned host tensors (gloo) of vlb_halo_bytes bytes."""

    def __init__(self, model, precision, grid: dict, inner, outer, kn: float, tau_mode: int,
                 begin: int, end: int, on_device: bool, stream=None):
        from . import vlb
        g = dict(grid, cell_begin=begin, cell_end=end)
        self.ctx = vlb.Couette(model, precision, [g], [inner], [outer], [kn], [tau_mode], stream=stream)
        self.begin, self.end = begin, end
        nb = self.ctx.halo_bytes()
        if on_device:
            self._edge = [torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2)]
        else:
            self._edge = [torch.empty(nb, dtype=torch.uint8).pin_memory() for _ in range(2)]

    def read_edge(self, end: int):
        return self.ctx.read_edge(0, end, self._edge[end])

    def write_halo(self, end: int, rows):
        self.ctx.write_halo(0, end, rows)

    def stage(self, dt: float, k: int):
        self.ctx.stage(dt, k)

    def residual_sums(self):
        return [float(x[0]) for x in self.ctx.residual_sums()]

    def close(self):
        self.ctx.close()
