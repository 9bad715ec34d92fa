"""Slabs of one grid on several ranks: ghost-plane exchange between processes.

This is the multi-process form of the library's domain decomposition
(spider_domain_*).  The layout comes from the library: the grid is cut along
its slowest axis into one slab per rank, each with g ghost planes on every
side that has a neighbour (g = steps per exchange x radius, rounded to the
multiple that keeps points in place inside the tensor-core tiles).  A run
alternates E time steps on the local slab with an exchange: rank p sends its
outermost g owned planes to ranks p - 1 and p + 1 and receives their
outermost owned planes into its ghost planes.  The exchange is a pair of
point-to-point send / receive with each neighbour (torch.distributed: NCCL
for device tensors, gloo for host tensors), not a collective.

The local time steps are the caller's `step(slab, n)`: on a GPU, a
spider_run of the slab's plan.  This module moves planes between ranks and
computes nothing itself.
"""
from __future__ import annotations

import ctypes

from . import _native
from ._native import check


class SlabLayout:
    """Slab `rank` of `world` for a plan's grid (spider_domain_create with one
    part per rank, read back through spider_domain_slab; host work only)."""

    def __init__(self, plan, world: int, rank: int, steps_per_exchange: int):
        lib = _native.load()
        h = ctypes.c_void_p()
        check(lib.spider_domain_create(plan.handle, int(world), int(steps_per_exchange), ctypes.byref(h)),
              "spider_domain_create")
        try:
            v = [ctypes.c_int64() for _ in range(4)]
            check(lib.spider_domain_slab(h, int(rank), *[ctypes.byref(x) for x in v]), "spider_domain_slab")
            self.first, self.owned, self.ghost_lo, self.ghost_hi = (x.value for x in v)
            g = [ctypes.c_int64() for _ in range(4)]
            # every interior side has the same depth: read it from a slab that has one
            probe = 1 if world > 1 else 0
            check(lib.spider_domain_slab(h, probe, *[ctypes.byref(x) for x in g]), "spider_domain_slab")
            self.ghost = g[2].value
        finally:
            lib.spider_domain_destroy(h)
        self.world, self.rank = int(world), int(rank)
        self.steps_per_exchange = int(steps_per_exchange)

    @property
    def planes(self) -> int:
        """Planes of the local slab: ghost planes below, owned, ghost planes above."""
        return self.ghost_lo + self.owned + self.ghost_hi

    def local_range(self):
        """[start, stop) of the slab's planes (ghosts included) in the global grid."""
        return self.first - self.ghost_lo, self.first + self.owned + self.ghost_hi


def exchange_ghosts(slab, layout: SlabLayout, group=None) -> None:
    """Fills the ghost planes of `slab` (a tensor whose first axis is the
    layout's planes) with the neighbouring ranks' outermost owned planes."""
    import torch.distributed as dist
    g, rank, world = layout.ghost, layout.rank, layout.world
    if world == 1 or g == 0:
        return
    lo_owned = slab[layout.ghost_lo:layout.ghost_lo + g]
    hi_owned = slab[layout.ghost_lo + layout.owned - g:layout.ghost_lo + layout.owned]
    reqs = []
    recv_lo = recv_hi = None
    if rank > 0:
        recv_lo = slab[:layout.ghost_lo].clone()
        reqs.append(dist.isend(lo_owned.contiguous(), rank - 1, group=group))
        reqs.append(dist.irecv(recv_lo, rank - 1, group=group))
    if rank + 1 < world:
        recv_hi = slab[layout.ghost_lo + layout.owned:].clone()
        reqs.append(dist.isend(hi_owned.contiguous(), rank + 1, group=group))
        reqs.append(dist.irecv(recv_hi, rank + 1, group=group))
    for r in reqs:
        r.wait()
    if recv_lo is not None:
        slab[:layout.ghost_lo] = recv_lo
    if recv_hi is not None:
        slab[layout.ghost_lo + layout.owned:] = recv_hi


def run_slab(slab, layout: SlabLayout, steps: int, step, group=None):
    """Advances the local slab by `steps` time steps in periods of the
    layout's steps per exchange, exchanging ghost planes between periods.
    `step(slab, n)` returns the slab after n steps (zero halo at the slab's
    ends).  Returns the final slab; its owned planes are those of the
    undivided run."""
    done = 0
    while done < steps:
        n = min(layout.steps_per_exchange, steps - done)
        slab = step(slab, n)
        done += n
        if done < steps:
            exchange_ghosts(slab, layout, group)
    return slab
