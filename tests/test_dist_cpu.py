"""Multi-rank host logic on CPU (gloo, world size 2): equation sharding and the
max/sum-over-ranks reductions bench.py uses (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2412_15840_gb300.dist import max_over_ranks, shard, sum_over_ranks


def test_shard_partitions_and_balances():
    costs = [float(c) for c in (5, 1, 9, 3, 3, 7, 2, 8, 6, 4)]
    for world in (1, 2, 3, 4):
        parts = [shard(costs, r, world) for r in range(world)]
        flat = sorted(e for p in parts for e in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[e] for e in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)
    assert shard(costs, 0, 1) == list(range(len(costs)))
    with pytest.raises(ValueError):
        shard(costs, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [float(i % 7 + 1) for i in range(23)]
        mine = shard(costs, rank, world)
        # per-rank "time": proportional to the rank's load
        t = sum(costs[e] for e in mine)
        tmax = max_over_ranks(t)
        done = sum_over_ranks(len(mine))
        dist.barrier()
        out[rank] = (tmax, done, mine)
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_reductions():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    (t0, n0, m0), (t1, n1, m1) = out[0], out[1]
    assert t0 == t1 == max(sum(float(i % 7 + 1) for i in m) for m in (m0, m1))
    assert n0 == n1 == 23
    assert sorted(m0 + m1) == list(range(23)) and not set(m0) & set(m1)


def test_reductions_without_a_group_are_identity():
    assert max_over_ranks(3.5) == 3.5 and sum_over_ranks(2.0) == 2.0
