"""The multi-rank bench path (independent replicas, max-over-ranks time, summed units)
with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    t_local = [10.0, 14.0][rank]          # rank 1 is the slow one
    units = [1000, 1000][rank]
    t, n, rate = bench.aggregate(t_local, units, dist, device="cpu")
    q.put((rank, t, n, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n, rate in res:
        assert t == 14.0 and n == 2000.0
        assert abs(rate - 2000.0 / 0.014) < 1e-6


def test_single_rank_aggregation():
    import bench
    t, n, rate = bench.aggregate(5.0, 100)
    assert (t, n) == (5.0, 100) and abs(rate - 100 / 0.005) < 1e-9
