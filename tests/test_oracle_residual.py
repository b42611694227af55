"""Pins of the oracle's convergence residual and total mass.

The residual of Sec. 5.2 (reading A8) is the unnormalised L2 norm of the change
of u_x over 20 steps, ``sqrt(sum((u_x(t) - u_x(t - 20))**2))``, evaluated at
t = 20, 40, ...; every steps-to-steady-state figure rests on it.  The total
mass is the sum of every population of every node.

Here both are recomputed in numpy from the oracle's post-collision populations
alone: u_x = (sum_i f~_i e_ix - F_x / (2 gamma)) / sum_i f~_i, the velocity the
collision used (its first moment gains F/gamma, Sec. 4.2).  The oracle's own
residual, its run-to-residual loop and its mass must equal those values, and
each plausible slip (u_y in place of u_x, a missing square root, a snapshot
that is not advanced, a population left out of the mass) is shown to give a
value that the comparison rejects.  No CUDA code is involved.
"""
import math

import numpy as np
import pytest

from oracle import stepper as S
from paper_2208_03562_gb300 import inputs as I

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
EYB = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)

RTOL = 1e-13
# u from the populations in another summation order than the oracle's:
# a few units of FP64 round-off of the O(1) density, per node
U_ABS = 4e-15


def _velocity(ft, p):
    """(u_x, u_y) of a post-collision population set, from its moments."""
    rho = np.sum(ft, axis=0)
    jx = np.tensordot(EX, ft, axes=1) - p.fx / (2 * p.gamma)
    jy = np.tensordot(p.r * EYB, ft, axes=1) - p.fy / (2 * p.gamma)
    return jx / rho, jy / rho


def _norm(a):
    return math.sqrt(math.fsum((a * a).ravel()))


def _start(p, seed):
    """Rest populations w_i(r) with a seeded perturbation that carries mass
    and momentum, so that the flow moves from the first step."""
    g = I.rng(seed)
    w = S.rest_weights(p)
    ft = w[:, None, None] * (1.0 + 0.02 * g.standard_normal((9, p.ny, p.nx)))
    return ft


CASES = [
    dict(nx=13, ny=9, r=0.5, gamma=0.5, nu=0.02, u_lid=0.05),
    dict(nx=10, ny=14, r=2.0, gamma=0.1, nu=0.01, u_lid=0.03),
    dict(nx=12, ny=8, r=1.0, gamma=1.0, nu=0.05, u_lid=0.0, fx=1e-5, fy=-2e-5, bc=S.BC_PERIODIC),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_residual_is_the_l2_change_of_u_x_over_20_steps(case):
    p = S.OracleParams(**CASES[case])
    o = S.Oracle(p)
    o.set_populations(_start(p, 40 + case))
    ux0, uy0 = _velocity(o.populations(), p)
    o.step(20)
    ux20, uy20 = _velocity(o.populations(), p)
    # the fields the oracle keeps are the same velocity
    f = o.fields()
    assert np.max(np.abs(f[1] - ux20)) <= U_ABS
    tol = lambda v: RTOL * v + 2 * U_ABS * math.sqrt(p.nx * p.ny)
    r20 = o.residual_update()
    want20 = _norm(ux20 - ux0)
    assert want20 > 0
    assert abs(r20 - want20) <= tol(want20)
    o.step(20)
    ux40, uy40 = _velocity(o.populations(), p)
    r40 = o.residual_update()
    want40 = _norm(ux40 - ux20)
    assert want40 > 1e4 * tol(0.0)
    assert abs(r40 - want40) <= tol(want40)
    # the slips each of which the comparison must reject
    slips = {
        "u_y in place of u_x": _norm(uy40 - uy20),
        "no square root": want40 ** 2,
        "snapshot not advanced": _norm(ux40 - ux0),
        "normalised by sqrt(N)": want40 / math.sqrt(p.nx * p.ny),
    }
    for name, v in slips.items():
        assert abs(v - r40) > 100 * tol(want40), name
    # the snapshot is advanced: an immediate second evaluation sees no change
    assert o.residual_update() == 0.0


@pytest.mark.parametrize("case", range(len(CASES)))
def test_run_returns_the_residual_of_its_last_block(case):
    """The run loop evaluates the residual after every block of 20 steps and
    returns the last one with the step count; its stop rule is R < tol."""
    p = S.OracleParams(**CASES[case])
    start = _start(p, 40 + case)
    o = S.Oracle(p)
    o.set_populations(start)
    seq = [_velocity(o.populations(), p)[0]]
    for _ in range(3):
        o.step(20)
        seq.append(_velocity(o.populations(), p)[0])
    norms = [_norm(b - a) for a, b in zip(seq, seq[1:])]
    tol = lambda v: RTOL * v + 2 * U_ABS * math.sqrt(p.nx * p.ny)
    o2 = S.Oracle(p)
    o2.set_populations(start)
    steps, res = o2.run(0.0, 60)
    assert steps == 60
    assert abs(res - norms[-1]) <= tol(norms[-1])
    # stop rule: with a tolerance between the first and the second norms
    # (the flow settles from the perturbed start), the run ends after 40 steps
    assert norms[1] < norms[0]
    o3 = S.Oracle(p)
    o3.set_populations(start)
    steps, res = o3.run(0.5 * (norms[0] + norms[1]), 60)
    assert steps == 40
    assert abs(res - norms[1]) <= tol(norms[1])


@pytest.mark.parametrize("case", range(len(CASES)))
def test_total_mass_is_the_sum_of_every_population(case):
    p = S.OracleParams(**CASES[case])
    o = S.Oracle(p)
    o.set_populations(_start(p, 40 + case))
    o.step(37)
    ft = o.populations()
    want = math.fsum(ft.ravel())
    m = o.total_mass()
    assert abs(m - want) <= 1e-13 * abs(want)
    # the density field the oracle keeps sums to the same mass
    assert abs(math.fsum(o.fields()[0].ravel()) - want) <= 1e-13 * abs(want)
    # slips: one population set left out, or the rest weights instead of
    # the populations
    for i in range(9):
        assert abs(math.fsum(np.delete(ft, i, axis=0).ravel()) - m) > 1e-6 * abs(want)
    w = S.rest_weights(p)
    assert abs(w.sum() * p.nx * p.ny - m) > 1e-6 * abs(want)
