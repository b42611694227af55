"""Placement of independent cavity solves on several GPUs.

The batched sweep and the solve server advance many independent cavities; no
step of the method couples two of them, so a multi-GPU run places whole
cavities on ranks (one process per GPU) and needs no collective on the data
path, only a final gather of the per-instance results on rank 0.

Placement balances the expected work of each rank: the bytes one step of a
cavity moves (nodes times the storage's bytes per node: 9 populations read and
written) times the steps it is expected to take.  The step estimate is a
heuristic of this library, not a result of the paper: the viscous time H^2 / nu
of the cavity (H = ny r in lattice units), shortened by gamma because the
preconditioned momentum equation advances its spatial terms 1/gamma faster
(Eqs. 5-6), and capped at the solve's step limit.  The greedy
longest-first rule then puts each cavity, largest cost first, on the rank with
the least work so far.  Its largest rank load is at most the mean load plus
the largest single cost (and within 4/3 of the best possible placement).
"""
from __future__ import annotations

from typing import Callable, List, Sequence

BYTES_PER_NODE = {"f64": 144, "f32": 72, "f16": 36}


def expected_steps(cav) -> float:
    """Heuristic steps to steady state of an ``inputs.Cavity``: gamma H^2 / nu,
    at least one residual block (20 steps), at most its step limit."""
    h = cav.ny * cav.r
    return float(min(max(cav.gamma * h * h / cav.nu, 20.0), cav.max_steps))


def cost(cav) -> float:
    """Expected device bytes of a whole solve: bytes per step times steps."""
    return cav.nodes * BYTES_PER_NODE[cav.dtype] * expected_steps(cav)


def partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Indices of the items each of `world` ranks takes, by the greedy
    longest-first rule (largest cost first, to the least-loaded rank; ties to
    the lower cost index and the lower rank).  Every index appears on exactly
    one rank; each rank's list is ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += float(costs[i])
    for lst in out:
        lst.sort()
    return out


def loads(costs: Sequence[float], parts: Sequence[Sequence[int]]) -> List[float]:
    return [sum(float(costs[i]) for i in p) for p in parts]


def run_sharded(items: Sequence, costs: Sequence[float], solve: Callable[[List], List], rank: int, world: int,
                dist=None):
    """Solve `items` across `world` ranks: this rank solves its share with
    `solve(list_of_items) -> list_of_results` (same order), and rank 0
    gathers every rank's results over `dist` (torch.distributed, any
    backend; None when world == 1).  Returns the results in the order of
    `items` on rank 0 and None on the other ranks."""
    parts = partition(costs, world)
    mine = parts[rank]
    local = list(solve([items[i] for i in mine]))
    if len(local) != len(mine):
        raise ValueError("solve returned %d results for %d items" % (len(local), len(mine)))
    if world == 1:
        return local_in_order(len(items), [mine], [local])
    gathered = [None] * world if rank == 0 else None
    dist.gather_object((mine, local), gathered, dst=0)
    if rank != 0:
        return None
    return local_in_order(len(items), [g[0] for g in gathered], [g[1] for g in gathered])


def local_in_order(n: int, index_lists, result_lists):
    """Reassemble per-rank results into the original item order; every index
    must appear exactly once."""
    out = [None] * n
    seen = [False] * n
    for idx, res in zip(index_lists, result_lists):
        for i, r in zip(idx, res):
            if seen[i]:
                raise ValueError("item %d placed twice" % i)
            seen[i] = True
            out[i] = r
    if not all(seen):
        raise ValueError("items not placed: %s" % [i for i, s in enumerate(seen) if not s])
    return out
