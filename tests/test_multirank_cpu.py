"""The multi-rank paths on CPU (gloo ranks): the plain workload's independent replicas agree on
the slowest rank's time, and the batched sweep / warm-start split hands every instance to
exactly one rank in contiguous, node-balanced ranges and gathers the per-instance results on
rank 0 in instance order."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.rank_workload(rank)
    local_ms = 10.0 + 5.0 * rank
    got = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (got, w.name, w.mu_rel_circle)
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_distinct_instances():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 15.0          # slowest rank's time on every rank
    assert out[0][1] != out[1][1]                    # independent instances (seed = rank)
    assert out[0][2] != out[1][2]


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5


def _shard_worker(rank, world, port, n_inst, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2202_06516_gb300 import shard, workloads as W
    ws = W.batched(n_inst, seed=0)
    nodes = [w.nx * w.ny for w in ws]
    lo, hi = shard.partition(nodes, world, rank)
    # a host stand-in for each instance's result: (index, nodes, name) plus the rank that ran it
    local = [(i, nodes[i], ws[i].name, rank) for i in range(lo, hi)]
    rows = shard.gather(local, dist)
    slow = shard.max_over_ranks(1.0 + rank, dist)
    got = shard.broadcast({"from": rank, "w": [1.5, 2.5]} if rank == 0 else None, dist)
    out[rank] = (lo, hi, rows, slow, got)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_inst", [(2, 64), (3, 2)])
def test_instance_split_and_gather_over_gloo_ranks(world, n_inst):
    """world gloo ranks split the batched sweep's instances: contiguous ranges in rank order that
    cover every instance exactly once (a rank may get none when instances are fewer than ranks),
    node-balanced to within one instance, and the gathered rows come back on rank 0 in instance
    order; the slowest rank's time and rank 0's broadcast reach every rank."""
    from paper_2202_06516_gb300 import workloads as W
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, n_inst, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    ranges = [out[r][:2] for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n_inst
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and a <= b
    rows = out[0][2]
    assert [r[0] for r in rows] == list(range(n_inst))
    ws = W.batched(n_inst, seed=0)
    assert [r[2] for r in rows] == [w.name for w in ws]
    for i, r in enumerate(rows):
        lo, hi = ranges[r[3]]
        assert lo <= i < hi  # the rank that reported it owns it
    for r in range(1, world):
        assert out[r][2] is None  # only rank 0 holds the gathered rows
    nodes = [w.nx * w.ny for w in ws]
    share = sum(nodes) / world
    for lo, hi in ranges:
        if n_inst >= world:
            assert abs(sum(nodes[lo:hi]) - share) <= max(nodes)
    assert all(out[r][3] == float(world) for r in range(world))
    assert all(out[r][4] == {"from": 0, "w": [1.5, 2.5]} for r in range(world))


def test_partition_without_process_group():
    from paper_2202_06516_gb300 import shard
    assert shard.partition([5.0, 1.0, 1.0, 1.0], 1, 0) == (0, 4)
    parts = [shard.partition([1.0] * 10, 4, r) for r in range(4)]
    assert parts[0][0] == 0 and parts[-1][1] == 10
    assert all(b == c for (_, b), (c, _) in zip(parts, parts[1:]))
    assert sorted(b - a for a, b in parts) == [2, 2, 3, 3]
    assert shard.partition([], 3, 1) == (0, 0)
    assert shard.gather([1, 2], None) == [1, 2]
    assert shard.max_over_ranks(3.0, None) == 3.0
    with pytest.raises(ValueError):
        shard.partition([1.0], 2, 2)
