"""The several-GPU form is independent replicas: every rank runs its own CPMA
and the job's time is the slowest rank's.  The aggregation bench.py uses is
checked here with two gloo ranks on the CPU (no GPU)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate(10.0 * (rank + 1), 1000.0, dist)
    out.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_the_slowest_rank_and_sums_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 20.0                         # max over ranks
        assert value == pytest.approx(2 * 1000.0 / 0.020)


def test_aggregate_single_process():
    import bench
    ms, value = bench.aggregate(4.0, 100.0, None)
    assert ms == 4.0 and value == pytest.approx(100.0 / 0.004)
