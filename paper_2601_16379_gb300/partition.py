"""Fragment partition across ranks (one process per GPU).

The fragment ERIs of Eqs. 19-20 are independent of one another once X^k and
V^q are known, so the fragment step shards by fragment: every rank holds the
same X and V^q (it runs the points, the fit and the Coulomb metric itself, or
receives them) and contracts its own share of the fragments.  The only
exchange is the gather of the per-fragment J/K traces at the end.  The paper
distributes its own work over MPI ranks (Section III); this is the same idea
applied to the fragment loop.

The assignment is longest-processing-time first on the cost of each fragment,
n_f^4 (the E = sum_q B^q B^q^H contraction dominates, Section II.C's
O(Nk N_EO^4 N_IP) term): fragments in decreasing cost go to the rank with the
least work so far (ties to the lower rank), which is deterministic and keeps
the ranks within one fragment of each other.
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import numpy as np


def fragment_cost(n_orb: int) -> float:
    """Relative cost of one fragment: the n_f^4 term of the contraction."""
    return float(n_orb) ** 4


def fragment_partition(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Fragment indices of each rank (each list in increasing index order)."""
    if world < 1:
        raise ValueError("world size must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-fragment_cost(sizes[i]), i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += fragment_cost(sizes[i])
    return [sorted(p) for p in parts]


def gather_traces(n_frag: int, mine: Sequence[int], ej: Sequence[float], ek: Sequence[float],
                  dist=None) -> Tuple[np.ndarray, np.ndarray]:
    """Full E_J, E_K arrays from every rank's share: each rank writes its own
    entries into zero arrays and one sum-reduction combines them (every
    fragment belongs to exactly one rank)."""
    import torch

    buf = torch.zeros((2, n_frag), dtype=torch.float64)
    for j, i in enumerate(mine):
        buf[0, i] = float(ej[j])
        buf[1, i] = float(ek[j])
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = buf.to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        buf = t.cpu()
    return buf[0].numpy().copy(), buf[1].numpy().copy()


def run_partitioned(sizes: Sequence[int], contract: Callable[[List[int]], Tuple[Sequence[float], Sequence[float]]],
                    rank: int = 0, world: int = 1, dist=None) -> Tuple[np.ndarray, np.ndarray, List[int]]:
    """Contract this rank's fragments with `contract(indices) -> (ej, ek)` and
    gather the traces of all fragments.  Returns (E_J, E_K, this rank's indices)."""
    mine = fragment_partition(sizes, world)[rank]
    ej, ek = contract(mine) if mine else ([], [])
    full_j, full_k = gather_traces(len(sizes), mine, ej, ek, dist)
    return full_j, full_k, mine
