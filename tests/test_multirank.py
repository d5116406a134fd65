"""The multi-rank path of bench.py on CPU (gloo, world size 2).

Under torchrun every rank builds its own replica of the workload (fragments are
independent given X and V^q, so replicas need no collective on the data path);
the only collective is the max over ranks of the step timings, checked here.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    res = bench.reduce_max_over_ranks([1.0 + rank, 10.0 - rank], dist, "cpu")
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_timings_reduce_to_the_slowest_rank():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == [2.0, 10.0]


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max_over_ranks([3.5, 4.25], None, "cpu") == [3.5, 4.25]
