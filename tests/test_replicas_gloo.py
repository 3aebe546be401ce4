"""Multi-rank timing of bench.py's replica mode, on CPU with gloo (world
size 2): every rank gets the slowest rank's time and the same whole-job
rate. No GPU is used."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(torch, dist, times[rank], "cpu")
    value = bench.job_mlups(1000, 10, world, ms)
    dist.barrier()
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    times = [3.0, 5.0]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 5.0
    expected = 1000 * 10 * world / (5.0e-3) / 1e6
    assert out[0][1] == pytest.approx(expected) and out[1][1] == pytest.approx(expected)
