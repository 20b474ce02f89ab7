"""Multi-rank logic of bench.py on CPU (gloo, world size 2): each rank advances
its own replica, the job's time is the slowest rank's, and the value counts the
site-steps of all ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank
    t = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (t, bench.whole_job_value(world, 512 * 512, 1000, t))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, v = out[r]
        assert t == 150.0
        assert v == pytest.approx(2 * 512 * 512 * 1000 / 0.150 / 1e6)


def test_single_rank_value():
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.whole_job_value(1, 100, 10, 1000.0) == pytest.approx(1e-3)
