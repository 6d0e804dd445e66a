"""Domain decomposition of a 2D or 3D problem along its last axis (slabs).

The conservation form (Sec. 2, Eq. 1DWENOFD) makes each cell's update need
the G = order/2 + 2 cells beyond it on each side, per Runge-Kutta stage, and
the global Lax-Friedrichs splitting takes alpha as the maximum of |f'(u)| over
the whole mesh (Sec. 2).  Split over ranks, a step is therefore one maximum
over all ranks (alpha) and, before each of the three stages, one exchange of
G layers with each neighbouring slab.  This module holds that host-side
bookkeeping -- slab ranges, which layers go where, the global alpha and the
time step -- over any object with the sub-domain interface of
``paper_2108_12742_gb300.SubDomain`` (``halo_export``, ``halo_import``,
``halo_fill_transmissive``, ``local_alpha``, ``set_step_alpha``, ``rk_stage``),
and two ways of moving the layers: ``TorchComm`` (torch.distributed, one rank
per process: gloo with host buffers, NCCL with device buffers) and
``LocalGroup`` (several sub-domains driven from one process, e.g. on one GPU).
"""
from __future__ import annotations

import numpy as np

PERIODIC, TRANSMISSIVE = 0, 1
UP, DOWN = 0, 1  # a slab's high-side layers go up to its upper neighbour, low-side ones down


def halo_width(order):
    return order // 2 + 2


def slab_ranges(n, nranks, G):
    """(offset, n_local) of each rank's slab of n layers: sizes differ by at
    most one, and every slab owns at least G layers (its neighbours' ghosts)."""
    if nranks < 1 or n < nranks * G:
        raise ValueError(f"{n} layers cannot be split into {nranks} slabs of at least {G}")
    base, extra = divmod(n, nranks)
    out, off = [], 0
    for r in range(nranks):
        m = base + (1 if r < extra else 0)
        out.append((off, m))
        off += m
    return out


def neighbours(rank, size, bc):
    """(lower, upper) neighbour ranks along the split axis; None at a
    transmissive edge of the global grid (periodic edges wrap around)."""
    lo = rank - 1 if rank > 0 else (size - 1 if bc == PERIODIC else None)
    hi = rank + 1 if rank < size - 1 else (0 if bc == PERIODIC else None)
    return lo, hi


def exchange_plan(rank, size, bc):
    """The messages of one halo exchange for this rank, in the fixed order in
    which every rank posts them (so that unmatched tags pair up in order):
      sends: (peer, tag, side) -- export the G interior layers next to side;
      recvs: (peer, tag, side) -- import into the G ghost layers beyond side;
      fills: sides at a transmissive edge (zero-gradient ghosts, no message).
    tag UP carries a slab's high-side layers to the slab above (its low
    ghosts), tag DOWN its low-side layers to the slab below."""
    lo, hi = neighbours(rank, size, bc)
    sends, recvs, fills = [], [], []
    if hi is not None:
        sends.append((hi, UP, 1))
    if lo is not None:
        sends.append((lo, DOWN, 0))
    if lo is not None:
        recvs.append((lo, UP, 0))
    else:
        fills.append(0)
    if hi is not None:
        recvs.append((hi, DOWN, 1))
    else:
        fills.append(1)
    return sends, recvs, fills


def step_dt(alpha, dx, cfl):
    """dt = cfl / sum_d alpha_d / dx_d, in the order the library's step takes it."""
    s = 0.0
    for d in range(len(dx)):
        s += alpha[d] / dx[d]
    return cfl / s


class TorchComm:
    """Halo messages and the alpha maximum over torch.distributed (one slab per
    rank).  ``device`` is where the message buffers live ("cpu" for gloo,
    "cuda" for NCCL)."""

    def __init__(self, device="cpu"):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()
        self.device = device

    def allreduce_max(self, a):
        import torch
        t = torch.as_tensor(np.asarray(a, dtype=np.float64), device=self.device).clone()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return t.cpu().numpy()

    def exchange(self, sends, recvs):
        """sends: [(peer, tag, tensor)], recvs: [(peer, tag, tensor)]; returns
        when every receive buffer is filled."""
        ops = [self.dist.P2POp(self.dist.isend, t, peer, tag=tag) for peer, tag, t in sends]
        ops += [self.dist.P2POp(self.dist.irecv, t, peer, tag=tag) for peer, tag, t in recvs]
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()


class Slab:
    """One rank's slab of a decomposed problem: ``dom`` is its sub-domain
    (interior layers [offset, offset + n_local) of the split axis), ``comm`` a
    TorchComm.  step() takes one Runge-Kutta step of the whole decomposed
    problem, collectively over the ranks."""

    def __init__(self, dom, comm, bc, dx):
        self.dom, self.comm, self.bc, self.dx = dom, comm, bc, tuple(dx)

    def _buf(self):
        import torch
        return torch.empty(self.dom.halo_shape, dtype=torch.float64, device=self.comm.device)

    def fill_halos(self, k):
        sends, recvs, fills = exchange_plan(self.comm.rank, self.comm.size, self.bc)
        out = [(peer, tag, self.dom.halo_export(k, side, self._buf())) for peer, tag, side in sends]
        inc = [(peer, tag, self._buf(), side) for peer, tag, side in recvs]
        self.comm.exchange(out, [(p, t, b) for p, t, b, _ in inc])
        for _, _, buf, side in inc:
            self.dom.halo_import(k, side, buf)
        for side in fills:
            self.dom.halo_fill_transmissive(k, side)

    def step(self, cfl):
        alpha = self.comm.allreduce_max(self.dom.local_alpha())
        self.dom.set_step_alpha(alpha)
        dt = step_dt(alpha, self.dx, cfl)
        for k in range(3):
            self.fill_halos(k)
            self.dom.rk_stage(k, dt)
        return dt


class LocalGroup:
    """All slabs of a decomposed problem driven from one process (the layers
    staged through host buffers): for several sub-domains on one GPU, or in
    tests.  doms[r] is the slab of rank r."""

    def __init__(self, doms, bc, dx):
        self.doms, self.bc, self.dx = list(doms), bc, tuple(dx)

    def fill_halos(self, k):
        size = len(self.doms)
        posted = {}
        for r, dom in enumerate(self.doms):  # every export first, then every import
            sends, _, _ = exchange_plan(r, size, self.bc)
            for peer, tag, side in sends:
                posted[(r, peer, tag)] = dom.halo_export(k, side)
        for r, dom in enumerate(self.doms):
            _, recvs, fills = exchange_plan(r, size, self.bc)
            for peer, tag, side in recvs:
                dom.halo_import(k, side, posted[(peer, r, tag)])
            for side in fills:
                dom.halo_fill_transmissive(k, side)

    def step(self, cfl):
        alpha = np.max([d.local_alpha() for d in self.doms], axis=0)
        for d in self.doms:
            d.set_step_alpha(alpha)
        dt = step_dt(alpha, self.dx, cfl)
        for k in range(3):
            self.fill_halos(k)
            for d in self.doms:
                d.rk_stage(k, dt)
        return dt
