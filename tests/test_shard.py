"""Placement of independent cavities on several ranks (``shard.py``).

Host logic only: the greedy longest-first placement is checked for exact
coverage and for its balance bounds (against brute force on small cases), and
the sharded run with a gather on rank 0 is checked on two and three gloo ranks
on CPU, with the FP64 oracle as the per-cavity solver standing in for the
batch engine: the gathered results must equal a single-rank run bitwise.
"""
import itertools
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2208_03562_gb300 import inputs as I
from paper_2208_03562_gb300 import shard as SH

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_every_cavity_of_the_sweep_is_placed_once_and_loads_balance(world):
    mix = I.batched_sweep(seed=0, n=256)
    costs = [SH.cost(c) for c in mix]
    parts = SH.partition(costs, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(mix)))
    ld = SH.loads(costs, parts)
    mean = sum(costs) / world
    assert max(ld) <= mean + max(costs) + 1e-9 * mean
    # the sweep has many more cavities than ranks: within 10 % of the mean
    assert max(ld) <= 1.10 * mean


def _opt(costs, world):
    best = float("inf")
    for assign in itertools.product(range(world), repeat=len(costs)):
        ld = [0.0] * world
        for c, r in zip(costs, assign):
            ld[r] += c
        best = min(best, max(ld))
    return best


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("world", [2, 3])
def test_greedy_is_within_the_longest_first_bound_of_the_best_placement(seed, world):
    g = I.rng(500 + seed)
    costs = list(g.uniform(1.0, 10.0, 7))
    ld = max(SH.loads(costs, SH.partition(costs, world)))
    opt = _opt(costs, world)
    assert ld <= (4.0 / 3.0 - 1.0 / (3.0 * world)) * opt + 1e-12


def test_cost_grows_with_nodes_and_with_gamma():
    a = I.Cavity(100, 50, 1.0, 0.5, 1000.0, 0.05)
    b = I.Cavity(200, 50, 1.0, 0.5, 1000.0, 0.05)
    c = I.Cavity(100, 50, 1.0, 0.1, 1000.0, 0.05)
    assert SH.cost(b) == pytest.approx(2 * SH.cost(a))
    assert SH.cost(c) < SH.cost(a)
    d = I.Cavity(100, 50, 1.0, 0.5, 1000.0, 0.05, "f16")
    assert SH.cost(d) == pytest.approx(SH.cost(a) / 2)
    # capped at the step limit
    e = I.Cavity(100, 50, 1.0, 0.5, 1000.0, 0.05, max_steps=100)
    assert SH.expected_steps(e) == 100


def test_reassembly_rejects_a_double_or_missing_placement():
    with pytest.raises(ValueError):
        SH.local_in_order(3, [[0, 1], [1, 2]], [["a", "b"], ["c", "d"]])
    with pytest.raises(ValueError):
        SH.local_in_order(3, [[0], [2]], [["a"], ["c"]])


def _tiny_mix():
    """Small cavities of the sweep's kind (uneven grids, r, gamma, Re)."""
    g = I.rng(11)
    out = []
    for _ in range(7):
        nx, ny = int(g.integers(4, 12)), int(g.integers(3, 9))
        r = float(g.choice([0.5, 1.0, 2.0]))
        gamma = float(g.uniform(0.2, 1.0))
        out.append(I.Cavity(nx, ny, r, gamma, 50.0, 0.03, "f32", 0.0, 40))
    return out


def _solve_with_oracle(cavs):
    """CPU stand-in for the batch engine: 40 FP64 oracle steps per cavity,
    returning the residual and the velocity field."""
    from oracle import stepper as S
    out = []
    for c in cavs:
        o = S.Oracle(S.OracleParams(nx=c.nx, ny=c.ny, r=c.r, gamma=c.gamma, nu=c.nu, u_lid=c.u_lid))
        steps, res = o.run(0.0, c.max_steps)
        _, ux, uy = o.fields()
        out.append((steps, res, ux, uy))
    return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2208_03562_gb300 import shard
        mix = _tiny_mix()
        res = shard.run_sharded(mix, [shard.cost(c) for c in mix], _solve_with_oracle, rank, world, dist)
        out[rank] = None if res is None else [(s, r, ux.tolist(), uy.tolist()) for s, r, ux, uy in res]
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_run_gathers_the_single_rank_results(world):
    single = SH.run_sharded(_tiny_mix(), [SH.cost(c) for c in _tiny_mix()], _solve_with_oracle, 0, 1)
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        got = dict(out)
    assert all(got[r] is None for r in range(1, world))
    assert len(got[0]) == len(single)
    for (s, r, ux, uy), (s1, r1, ux1, uy1) in zip(got[0], single):
        assert s == s1 and r == r1
        assert np.array_equal(np.array(ux), ux1) and np.array_equal(np.array(uy), uy1)
    # every rank had work
    parts = SH.partition([SH.cost(c) for c in _tiny_mix()], world)
    assert all(parts)
