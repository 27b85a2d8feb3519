"""The multi-GPU path of the benchmark is replicas only (one independent system per rank; no
collective on the data path).  Its host logic -- barrier, max-over-ranks timing and the
whole-job aggregate -- is exercised here with two gloo ranks on the CPU."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    local_ms = [400.0, 500.0][rank]          # rank 1 is the slowest
    value, ms_per_step = bench.aggregate(local_ms, world, 600_000, 5, torch.device("cpu"))
    out[rank] = (value, ms_per_step)
    dist.destroy_process_group()


def test_two_rank_aggregate_takes_the_slowest_rank():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    # 2 ranks x 600k dofs x 5 steps in 0.5 s
    for r in range(world):
        value, ms = out[r]
        assert ms == 100.0
        assert abs(value - 2 * 600_000 * 5 / 0.5) < 1e-6


def test_single_rank_aggregate():
    import bench
    value, ms = bench.aggregate(250.0, 1, 600_000, 5, torch.device("cpu"))
    assert ms == 50.0 and abs(value - 600_000 * 5 / 0.25) < 1e-6
