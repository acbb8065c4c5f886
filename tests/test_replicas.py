"""Multi-rank path of bench.py on CPU: world_size-2 gloo process group, replicas
only (no collective in the method's data path; the one all-reduce is the
max-over-ranks timing)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r timed 3 units in (r + 1) seconds: the job is as slow as rank 1
    out[rank] = bench.replica_rate(1000.0 * (rank + 1), 3, world)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_takes_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        slowest, value = out[r]
        assert slowest == pytest.approx(2000.0)
        assert value == pytest.approx(world * 3 / 2.0)


def test_replica_rate_single_process():
    slowest, value = __import__("bench").replica_rate(500.0, 4, 1)
    assert slowest == 500.0 and value == pytest.approx(8.0)
