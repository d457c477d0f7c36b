"""The N > 1 benchmark path on CPU: two gloo ranks, each with its own replica, combine their
timings only through the barrier and the max over ranks (no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r = bench.Ranks(dist, torch.device("cpu"))
    r.barrier()
    my_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
    out[rank] = (r.max(my_ms), r.job_rate(4, my_ms), r.world)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    # the manager process is spawned, not forked: this process may already run OpenMP threads
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        mx, rate, w = res[rank]
        assert w == 2
        assert mx == 200.0
        assert rate == pytest.approx(8 / 0.2)  # 4 solves per rank x 2 ranks / slowest 200 ms


def test_single_process_needs_no_collective():
    import bench
    r = bench.Ranks(None)
    assert r.world == 1 and r.max(3.0) == 3.0 and r.job_rate(4, 500.0) == pytest.approx(8.0)
