"""Domain decomposition of one ADG problem: contiguous PE ranges per rank, and the
exchange of the PE boundary elements between neighbouring subdomains.

The method (Sec. 3.1, Fig. 1) cuts the domain into the subdomains of the PEs;
each sends the DoFs of its boundary elements to the buffer elements of its
neighbours. Sec. 3.2: the buffers may hold delayed levels, and the flux at a PE
face is taken at the common delayed level (the AT flux of Eq. 7 over several of
them). Sec. 3.3: the limiter's neighbour data is exchanged after every stage,
and across a delayed face the AT-WENO neighbour of Eq. (11) extrapolates the
delayed levels. Sec. 4: CAA and SAA decide the delays; here they are drawn by
the whole domain's face numbers, so that a decomposed run follows the same
delays as the whole domain run.

A subdomain is an instance of its own (``pe_begin``, ``pe_end`` on the workload)
holding its elements plus one buffer element at each cut side. Per RK stage:

1. the stage inputs of the boundary elements go to the neighbours' buffers,
2. half 0 of the stage (the stage kernels: Eq. 5 and the RK update),
3. the pre-limit outputs of the boundary elements go to the neighbours' buffers
   (and into the history of the cut faces, for the delayed AT-WENO neighbours),
4. half 1 (troubled-cell indicator and limiter).

Every delayed level that a stage reads was written by an earlier exchange, so
the owned elements advance exactly as in the whole-domain run. With real
network delays the same buffers would simply hold older levels; here the delays
are the emulated ones of Sec. 4.

The stage work and the block moves come from a backend (the CUDA library
through ``adg.ADG``, or anything with the same calls); this module holds only
the partition and the message schedule.
"""
from __future__ import annotations

import dataclasses

PART_INPUT, PART_PRELIMIT = 0, 1


def split_pes(n_pe, world):
    """Contiguous PE ranges [(pe_begin, pe_end)] of `world` ranks, as even as the
    PE count allows (rank r: [floor(r P / W), floor((r+1) P / W)))."""
    if world < 1 or n_pe < world:
        raise ValueError("%d PEs cannot be split over %d ranks" % (n_pe, world))
    return [((r * n_pe) // world, ((r + 1) * n_pe) // world) for r in range(world)]


def subdomain(wl, pe_begin, pe_end):
    """A copy of the workload restricted to the PEs [pe_begin, pe_end)."""
    return dataclasses.replace(wl, pe_begin=int(pe_begin), pe_end=int(pe_end))


def neighbours(rank, world, periodic):
    """(left rank, right rank) of a rank's subdomain; None past a physical
    boundary."""
    left = rank - 1 if rank > 0 else (world - 1 if periodic and world > 1 else None)
    right = rank + 1 if rank < world - 1 else (0 if periodic and world > 1 else None)
    return left, right


def local_slice(arr, n_elem, elem0, n_local, axis):
    """The elements [elem0, elem0 + n_local) (modulo n_elem) of a whole-domain
    array along `axis`: a subdomain's initial data, buffers included."""
    import numpy as np
    idx = (np.arange(n_local) + elem0) % n_elem
    return np.take(arr, idx, axis=axis)


def owned(arr, cut_left, cut_right, axis):
    """A subdomain array without its buffer elements."""
    import numpy as np
    n = arr.shape[axis]
    return np.take(arr, range(int(cut_left), n - int(cut_right)), axis=axis)


def advance(n_steps, n_stages, stage, exchange):
    """n_steps steps of a decomposed run: `stage(s, half)` runs one half of RK
    stage s (of every subdomain the caller holds), `exchange(what, s)` moves the
    boundary blocks (PART_INPUT before half 0, PART_PRELIMIT before half 1)."""
    for _ in range(int(n_steps)):
        for s in range(int(n_stages)):
            exchange(PART_INPUT, s)
            stage(s, 0)
            exchange(PART_PRELIMIT, s)
            stage(s, 1)


def capture_step(n_stages, stage, exchange, device=None):
    """One step of a decomposed run (the sequence of `advance`) captured into a
    torch CUDA graph on the current device, for runs whose stage and exchange
    calls only enqueue work on PyTorch's current stream (``adg.ADG.step_stage``
    and ``AdgPart``): the graph's replay is one step. Capturing enqueues nothing
    that runs; the blocks the exchange allocates come from the graph's pool."""
    import torch
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        advance(1, n_stages, stage, exchange)
    return g


class LocalExchange:
    """The exchange between subdomains held by one process, listed in PE order.

    Each part has ``cut`` (left, right) and ``export(what, side, s)`` /
    ``import_(what, side, s, blk)``. All exports come first, so a part's buffer
    is written only after every boundary block of the stage has been read."""

    def __init__(self, parts):
        self.parts = list(parts)

    def __call__(self, what, s):
        n = len(self.parts)
        out = {}
        for i, p in enumerate(self.parts):
            for side in (0, 1):
                if p.cut[side]:
                    out[(i, side)] = p.export(what, side, s)
        for i, p in enumerate(self.parts):
            if p.cut[0]:
                p.import_(what, 0, s, out[((i - 1) % n, 1)])
            if p.cut[1]:
                p.import_(what, 1, s, out[((i + 1) % n, 0)])


class DistExchange:
    """The exchange of one rank's subdomain with its neighbour ranks over
    torch.distributed point-to-point messages (gloo or NCCL).

    A block sent to the left neighbour fills that rank's right buffer and has
    tag 2 what; a block sent to the right fills the left buffer, tag 2 what + 1.
    Every rank posts its sends leftward first, then rightward, and its receives
    from the right neighbour first, then from the left one: when both
    neighbours are the same rank (two ranks, periodic), the messages between
    them then pair up in posting order too, for backends that ignore tags.

    ``to_wire(blk)`` turns an exported block into a tensor the backend sends
    (a CPU tensor for gloo, a CUDA tensor for NCCL), ``empty()`` makes a
    receive tensor of the same shape, and ``from_wire(t)`` gives what the
    part imports."""

    def __init__(self, dist, part, rank, world, periodic, to_wire, empty, from_wire,
                 group=None):
        self.dist, self.part, self.group = dist, part, group
        self.left, self.right = neighbours(rank, world, periodic)
        if part.cut[0] != (self.left is not None) or part.cut[1] != (self.right is not None):
            raise ValueError("the subdomain's cut sides do not match its neighbour ranks")
        self.to_wire, self.empty, self.from_wire = to_wire, empty, from_wire

    def __call__(self, what, s):
        d, p = self.dist, self.part
        reqs, keep = [], []
        if self.left is not None:
            t = self.to_wire(p.export(what, 0, s))
            keep.append(t)
            reqs.append(d.isend(t, self.left, group=self.group, tag=2 * what))
        if self.right is not None:
            t = self.to_wire(p.export(what, 1, s))
            keep.append(t)
            reqs.append(d.isend(t, self.right, group=self.group, tag=2 * what + 1))
        rbuf = lbuf = None
        if self.right is not None:
            rbuf = self.empty()
            reqs.append(d.irecv(rbuf, self.right, group=self.group, tag=2 * what))
        if self.left is not None:
            lbuf = self.empty()
            reqs.append(d.irecv(lbuf, self.left, group=self.group, tag=2 * what + 1))
        for r in reqs:
            r.wait()
        if lbuf is not None:
            p.import_(what, 0, s, self.from_wire(lbuf))
        if rbuf is not None:
            p.import_(what, 1, s, self.from_wire(rbuf))


class AdgPart:
    """One subdomain instance of an ``adg.ADG`` context as a part: its blocks
    are CUDA tensors [nv, p+1] moved by adg_part_block on the context's stream."""

    def __init__(self, ctx, k, stream=None):
        from . import adg
        self.ctx, self.k, self.stream = ctx, int(k), stream
        wl = ctx.workloads[self.k]
        n_local, elem0, cl, cr = adg.part_layout(wl)
        self.n_local, self.elem0 = n_local, elem0
        self.cut = (bool(cl), bool(cr))
        self.block_shape = (ctx.nv, wl.p + 1)

    def export(self, what, side, s):
        import torch
        blk = torch.empty(self.block_shape, dtype=torch.float64, device=self.ctx.device)
        self.ctx.part_block(self.k, what, side, s, blk, False, self.stream)
        return blk

    def import_(self, what, side, s, blk):
        self.ctx.part_block(self.k, what, side, s, blk.contiguous(), True, self.stream)
