"""The multi-rank path of the benchmark on CPU: two gloo ranks (spawned
processes, rendezvous on 127.0.0.1) partition the 512-instance ensemble with
`shard.assign` and reduce their timings with `shard.reduce_rate`, the calls
`bench.py` makes under torchrun. The shards are disjoint and cover every
instance; the summed units are the whole ensemble's DOF-stages per step; the
reduced time is the longest rank's. A single problem runs whole on every rank
(replicas), and the units then count every replica. Two ranks that step their
shards of a small ensemble (through the oracle, on the CPU) gather the same
states as one process that steps every instance."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from paper_2501_01747_gb300 import inputs as I
    from paper_2501_01747_gb300 import shard as SH
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cpu = torch.device("cpu")
        ens = I.ensemble_workloads()
        idx, mode = SH.assign(len(ens), rank, world)
        units = bench.dof_stages_per_step([ens[i] for i in idx])
        ms, total = SH.reduce_rate(dist, 1.0 + 2.5 * rank, units, cpu)
        shards = [None] * world
        dist.all_gather_object(shards, idx)
        one = [I.load_workloads()["ignition-9sp-4096x4"]]
        idx1, mode1 = SH.assign(len(one), rank, world)
        _, total1 = SH.reduce_rate(dist, 1.0, bench.dof_stages_per_step([one[i] for i in idx1]), cpu)
        q.put((rank, mode, ms, total, shards, mode1, idx1, total1))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_ensemble_and_replicate_a_single_problem():
    import torch.multiprocessing as mp

    sys.path.insert(0, ROOT)
    import bench
    from paper_2501_01747_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    try:
        for _ in range(2):
            r = q.get(timeout=240)
            res[r[0]] = r
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    ens = I.ensemble_workloads()
    whole = bench.dof_stages_per_step(ens)
    one = bench.dof_stages_per_step([I.load_workloads()["ignition-9sp-4096x4"]])
    for rank in (0, 1):
        _, mode, ms, total, shards, mode1, idx1, total1 = res[rank]
        assert mode == "sharded" and mode1 == "replicas" and idx1 == [0]
        assert ms == 3.5  # the longest rank's
        assert total == whole
        assert total1 == 2 * one
        s0, s1 = set(shards[0]), set(shards[1])
        assert not (s0 & s1) and s0 | s1 == set(range(len(ens)))
        assert abs(len(s0) - len(s1)) <= 1


def test_assign_rejects_a_bad_partition():
    from paper_2501_01747_gb300 import shard as SH
    for args in ((10, 2, 2), (10, -1, 2), (0, 0, 1), (10, 0, 0)):
        with pytest.raises(ValueError):
            SH.assign(*args)
    assert SH.assign(5, 1, 2) == ([1, 3], "sharded")
    assert SH.assign(1, 1, 4) == ([0], "replicas")


def _mini_ensemble():
    """The first six ensemble instances (their degrees, temperatures, fuel
    fractions, delay seeds and dt), each cut to 24 + 4 i elements in 2 PEs so
    that the oracle steps them in seconds."""
    from paper_2501_01747_gb300 import inputs as I
    return [I.scaled(wl, 24 + 4 * i, 2) for i, wl in enumerate(I.ensemble_workloads(6))]


def _run_instance(wl, mech, steps):
    import oracle as O
    from paper_2501_01747_gb300 import inputs as I
    o = O.Oracle(wl, mech)
    o.set_primitive(I.primitive_ic(wl, mech))
    o.step(steps)
    return o.state(), o.flags()[1]


def _step_rank(rank, world, port, steps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2501_01747_gb300 import shard as SH
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ens = _mini_ensemble()
        mech = ens[0].mechanism()
        idx, mode = SH.assign(len(ens), rank, world)
        mine = {i: _run_instance(ens[i], mech, steps) for i in idx}
        every = [None] * world
        dist.all_gather_object(every, mine)
        q.put((rank, mode, every))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_step_their_shards_like_one_process():
    """Each rank advances only the instances `shard.assign` gives it (here
    through the oracle, the CPU stand-in for a rank's GPU), and the gathered
    states and troubled-cell counts equal a single-process run of every
    instance bit for bit: sharding an ensemble moves no data and changes no
    result."""
    import torch.multiprocessing as mp

    steps = 6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_step_rank, args=(r, 2, port, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    try:
        for _ in range(2):
            r = q.get(timeout=240)
            res[r[0]] = r
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    ens = _mini_ensemble()
    mech = ens[0].mechanism()
    for rank in (0, 1):
        _, mode, every = res[rank]
        assert mode == "sharded"
        got = {}
        for part in every:
            assert not (set(part) & set(got))
            got.update(part)
        assert sorted(got) == list(range(len(ens)))
        for i, wl in enumerate(ens):
            w, cnt = _run_instance(wl, mech, steps)
            assert np.array_equal(got[i][0], w), i
            assert np.array_equal(got[i][1], cnt), i
