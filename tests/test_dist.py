"""Multi-process host logic on CPU (gloo, world size 2): instance sharding
covers every unit exactly once and balances the load; the max-over-ranks
timing and the aggregate throughput see every rank."""
import os
import socket

import pytest

from paper_2012_08208_gb300 import dist as D


def test_shard_partitions_and_balances():
    import workloads as W
    ws = W.batch2d()
    weights = [w.n_nodes for w in ws]
    for world in (1, 2, 3, 4, 8):
        parts = [D.shard(weights, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(ws)))
        loads = [sum(weights[i] for i in p) for p in parts]
        # greedy LPT: the heaviest rank exceeds the mean by less than the largest unit
        assert max(loads) - sum(loads) / world <= max(weights)
    with pytest.raises(ValueError):
        D.shard(weights, 2, 2)


def test_throughput_uses_the_slowest_rank():
    assert D.throughput([10, 10], [1.0, 2.0]) == pytest.approx(10.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import workloads as W
        weights = [w.n_nodes for w in W.batch2d()]
        mine = D.shard(weights, world, rank)
        t = 1.0 + rank  # this rank's "time"
        tmax = D.max_over_ranks([t, -t])
        units = D.sum_over_ranks([len(mine)])
        dist.barrier()
        q.put((rank, D.env(), mine, tmax, units))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, env0, m0, tmax0, u0), (r1, env1, m1, tmax1, u1) = res
    assert env0 == (2, 0, 0) and env1 == (2, 1, 1)
    assert sorted(m0 + m1) == list(range(64)) and not set(m0) & set(m1)
    assert tmax0 == tmax1 == [2.0, -1.0]
    assert u0 == u1 == [64.0]
