"""The multi-rank bench path on CPU: two gloo ranks, each with its own seeded instance, agree on
the slowest rank's time (max over ranks) without any data-path collective."""
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
