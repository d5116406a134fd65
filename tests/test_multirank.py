"""The multi-rank path on CPU (gloo, world size 2).

Fragments are independent given X and V^q, so under torchrun every rank holds
X and V^q, contracts its share of the fragments and the traces are gathered by
one sum-reduction; bench.py also takes the max over ranks of the step timings.
A CPU stand-in (the oracle) takes the place of the per-fragment library call,
so no GPU is needed.
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


def _any_rank_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank 1 alone runs out of budget: every rank stops; nobody out of budget: nobody stops
    out[rank] = (bench.any_rank(rank == 1, dist, "cpu"), bench.any_rank(False, dist, "cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_budget_decisions_agree_across_ranks():
    """Each bench step ends in a collective, so the wall-clock budget that stops the
    warm-up and timed loops is decided jointly: one rank out of budget stops all."""
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_any_rank_worker, args=(world, port, out), nprocs=world, join=True)
    assert [out[r] for r in range(world)] == [(True, False)] * world


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max_over_ranks([3.5, 4.25], None, "cpu") == [3.5, 4.25]
    assert bench.any_rank(True, None, "cpu") is True and bench.any_rank(False, None, "cpu") is False


# ------------------------------------------------- fragment partition
def test_partition_covers_every_fragment_once_and_balances():
    from paper_2601_16379_gb300.partition import fragment_cost, fragment_partition
    sizes = [40, 200, 73, 120, 41, 199, 88, 150, 60, 60, 130]
    for world in (1, 2, 3, 4, 8):
        parts = fragment_partition(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(fragment_cost(sizes[i]) for i in p) for p in parts]
        # greedy longest-first: no rank exceeds the mean by more than the largest fragment
        assert max(loads) <= sum(loads) / world + max(fragment_cost(s) for s in sizes)
    assert fragment_partition(sizes, 2) == fragment_partition(list(sizes), 2)   # deterministic


def _tiny_fragments():
    import oracle as O
    from paper_2601_16379_gb300 import workloads as W
    cell = W.custom_cell(5.0, [[0, 0, 0], [0.37, 0.52, 0.21]],
                         [W.Shell(0, 0, (0.6,), (1.0,)), W.Shell(1, 0, (0.9,), (1.0,))], 2, 8)
    r = O.run_isdf(cell, 16, 7, solve_tol=1e-10)
    sizes = [2, 4, 3, 5, 2]
    frags = [W.make_fragment(cell, 11, i, n) for i, n in enumerate(sizes)]
    return cell, r, sizes, frags


def _contract_on_cpu(cell, r, frags, idx):
    """CPU stand-in for the per-fragment library call: the oracle's ERIs and traces."""
    import oracle as O
    ej, ek = [], []
    for i in idx:
        eri = O.fragment_eri(r["X"], r["V"], frags[i].C, cell.kmesh)
        a, b = O.traces(eri, frags[i].gamma)
        ej.append(a)
        ek.append(b)
    return ej, ek


def _partition_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2601_16379_gb300.partition import run_partitioned
    cell, r, sizes, frags = _tiny_fragments()   # every rank holds X and V^q
    ej, ek, mine = run_partitioned(sizes, lambda idx: _contract_on_cpu(cell, r, frags, idx), rank, world, dist)
    out[rank] = (list(ej), list(ek), mine)
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_traces_equal_one_rank():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_partition_worker, args=(world, port, out), nprocs=world, join=True)
    cell, r, sizes, frags = _tiny_fragments()
    ej1, ek1 = _contract_on_cpu(cell, r, frags, range(len(sizes)))
    mine = sorted(i for k in range(world) for i in out[k][2])
    assert mine == list(range(len(sizes)))
    assert all(len(out[k][2]) > 0 for k in range(world))
    for k in range(world):
        assert out[k][0] == list(ej1) and out[k][1] == list(ek1)
