"""Multi-rank host logic of bench.py with gloo on CPU (world size 2, no GPU).

bench.py runs independent replicas (one per GPU): the only cross-rank operations are the
barrier and the max over ranks of the timed region; the whole-job value is all ranks'
units over the slowest rank's time.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank           # rank 1 is the slow one
    ms_max = bench.reduce_max(ms_local)
    dist.barrier()
    q.put((rank, ms_max, bench.replica_throughput(world, 10, ms_max)))
    dist.destroy_process_group()


def test_reduce_max_and_replica_value_world2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, val in res:
        assert ms_max == 150.0
        assert abs(val - 2 * 10 / 0.150) < 1e-9


def test_single_process_identity():
    import bench
    assert bench.reduce_max(12.5) == 12.5
    assert abs(bench.replica_throughput(1, 5, 250.0) - 20.0) < 1e-12
