"""The whole-job rate of bench.py over replicas (CPU only): two gloo ranks
with different local times must both report the slowest rank's time and
world * steps / that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [120.0, 200.0][rank]
    out[rank] = bench.job_rate(local, 10, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    import bench
    assert bench.job_rate(50.0, 5, 1) == (50.0, 100.0)
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        for r in range(world):
            ms, rate = out[r]
            assert ms == 200.0
            assert rate == pytest.approx(world * 10 / 0.2)
