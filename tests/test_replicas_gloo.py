"""The bench's multi-rank aggregation (replicas: one independent solve stream
per GPU, no collective on the data path) over two CPU ranks on gloo: every
rank reports the slowest rank's time and the whole-job solves/s."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sys.path.insert(0, ROOT)
        import bench
        steps = 5
        own_ms = 100.0 * (rank + 1)          # rank 1 is the slower replica
        value, total_ms = bench.replicas_value(own_ms, steps, world, dist, "cpu")
        assert total_ms == 100.0 * world, (rank, total_ms)
        assert abs(value - world * steps / (total_ms / 1e3)) < 1e-12
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_value_two_ranks_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)


def test_replicas_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    value, total_ms = bench.replicas_value(250.0, 5, 1)
    assert total_ms == 250.0 and value == 20.0
