"""Partition of a workload's instances over ranks, one process per GPU.

The instances of an ensemble are independent problems (each has its own mesh,
PEs and delays), so rank r of N runs instances r, r + N, r + 2N, ... and no data
moves between ranks. A workload with fewer instances than ranks (a single
problem) runs whole on every rank: replicas. The only collectives are the
reductions of a measured run: the longest rank's time and the sum of the units
that the ranks processed."""


def assign(n_items, rank, world):
    """(indices of the instances rank `rank` runs, "sharded" or "replicas")."""
    if world < 1 or not 0 <= rank < world or n_items < 1:
        raise ValueError("bad partition: %d items, rank %d of %d" % (n_items, rank, world))
    if n_items >= world:
        return list(range(rank, n_items, world)), "sharded"
    return list(range(n_items)), "replicas"


def reduce_rate(dist, ms, units, device):
    """(the longest rank's ms, the sum over ranks of units): two all-reduces on
    `dist` (torch.distributed, or None for one process) with tensors on
    `device` (the GPU for NCCL, the CPU for gloo)."""
    if dist is None:
        return float(ms), float(units)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
