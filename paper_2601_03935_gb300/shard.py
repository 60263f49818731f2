"""Velocity-space sharding of the GSIS outer iteration over several GPUs.

With the macroscopic fields fixed, each discrete velocity's (and photon direction's)
kinetic sweep is independent, so the velocity and direction sets are cut into one
contiguous range per rank.  Every rank holds all cells; per outer iteration the ranks
sum one exchange buffer (per-cell moment sums and wall outflow; GSIS adds a second
exchange with the kinetic boundary-flux sums), and the synthetic equations are solved
on every rank from identical inputs.  The arithmetic runs in the library
(gsis_shard_* entry points); this module only partitions the sets and drives the phase
calls and the sums.

``allreduce_`` sums a list of equally shaped buffers: those held by this process (one
per shard it drives, several when shards are emulated on one GPU) and, when
torch.distributed is initialised with more than one rank, those of every rank (NCCL on
GPUs, gloo on CPU tensors).  Every buffer ends with the total.
"""
from __future__ import annotations

import numpy as np

from . import gsis as G


def split_range(n, rank, world):
    """Contiguous [lo, hi) of n items for `rank` of `world`: sizes differ by at most one,
    earlier ranks take the larger ones, every rank gets at least one item."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank %r of %r" % (rank, world))
    if n < world:
        raise ValueError("%d items cannot feed %d ranks" % (n, world))
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allreduce_(bufs, group=None):
    """Sum the tensors in `bufs` (same shape, dtype and device) in place: over this
    process's list first, then over the ranks of torch.distributed if it is initialised
    with a world larger than one."""
    import torch
    import torch.distributed as dist
    total = bufs[0] if len(bufs) == 1 else torch.stack(list(bufs)).sum(0)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        if total is bufs[0] and len(bufs) == 1:
            dist.all_reduce(bufs[0], op=dist.ReduceOp.SUM, group=group)
            return bufs
        dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
    for b in bufs:
        if b is not total:
            b.copy_(total)
    return bufs


class _DeviceDoubles:
    """A borrowed device array of doubles, for torch.as_tensor (no copy, no stream sync)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 2}


class VelocityShard:
    """One rank's context: the velocities xi[lo:hi] and directions omega[olo:ohi] of a
    workload, every cell.  `buf` is the context's exchange buffer as a torch tensor."""

    def __init__(self, mesh, xi, w, omega, wo, model, solver, rank, world, stream=0):
        import torch
        dim = mesh.dim
        xi = np.asarray(xi, np.float64)[:, :dim]
        self.lo, self.hi = split_range(xi.shape[0], rank, world)
        self.olo, self.ohi = split_range(np.asarray(wo).shape[0], rank, world)
        self.ctx = G.gsis_create(dim, mesh.face_owner, mesh.face_nbr, mesh.face_normal, mesh.face_area,
                                 mesh.face_centroid, mesh.cell_volume, mesh.cell_centroid, mesh.patches,
                                 xi[self.lo:self.hi], np.asarray(w)[self.lo:self.hi], np.asarray(omega)[self.olo:self.ohi],
                                 np.asarray(wo)[self.olo:self.ohi], model, solver, stream,
                                 period=getattr(mesh, "period", 0.0))
        try:
            G.gsis_shard_setup(self.ctx, xi, w, omega, wo)
            ptr, n = G.gsis_shard_buffer(self.ctx)
            self.buf = torch.as_tensor(_DeviceDoubles(ptr, n), device="cuda")
        except Exception:
            G.gsis_destroy(self.ctx)
            raise
        self.n_cells = mesh.n_cells

    def set_distributions(self, f_all, I_all):
        """This shard's slice of full distributions f [n_cells][n_xi][4], I [n_cells][n_omega]
        (host, FP64); follow with refresh()."""
        G.gsis_set_distributions(self.ctx, np.ascontiguousarray(f_all[:, self.lo:self.hi]),
                                 np.ascontiguousarray(I_all[:, self.olo:self.ohi]))

    def destroy(self):
        if self.ctx:
            G.gsis_destroy(self.ctx)
            self.ctx = None


def _sum(shards, reduce, stream):
    import torch
    if stream is not None:
        with torch.cuda.stream(stream):
            reduce([s.buf for s in shards])
    else:
        reduce([s.buf for s in shards])


def refresh(shards, reduce=allreduce_, stream=None):
    """Fields of the current distributions on every shard (two exchanges)."""
    for p in (0, 1):
        for s in shards:
            G.gsis_shard_refresh(s.ctx, p)
        _sum(shards, reduce, stream)
        for s in shards:
            G.gsis_shard_end(s.ctx)


def step(shards, mode=G.GSIS_MODE_CIS, reduce=allreduce_, stream=None):
    """One outer iteration on every shard this process drives; returns eps (the same on
    every shard)."""
    for s in shards:
        G.gsis_shard_begin(s.ctx, mode)
    _sum(shards, reduce, stream)
    if mode == G.GSIS_MODE_GSIS:
        for s in shards:
            G.gsis_shard_mid(s.ctx)
        _sum(shards, reduce, stream)
    return [G.gsis_shard_end(s.ctx) for s in shards][0]
