"""The batched-sweep workload (256 uneven cavities, seed 0) against the FP64
oracle: the eight smallest cavities of the mix, advanced 1000 steps inside
one batch (FP32 storage and collision), must match independent oracle runs
to the FP32 parity bar, 1e-5 relative L2 of the velocity. A cavity whose
sampled Re, gamma and r put it beyond the scheme's stability diverges on both
sides and is counted, not compared."""
import numpy as np
import pytest

from oracle import stepper as S
from paper_2208_03562_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = pytest.importorskip("paper_2208_03562_gb300.lbm")

STEPS = 1000


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L.load()


def test_smallest_cavities_of_the_sweep_match_the_oracle():
    mix = I.batched_sweep(seed=0, n=256)
    small = sorted(mix, key=lambda c: c.nodes)[:8]
    b = L.Batch(len(small), L.F32)
    slots = [b.add(L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid, L.F32), 0.0, STEPS) for c in small]
    while b.run(STEPS):
        pass
    compared = 0
    for c, s in zip(small, slots):
        info, st = b.query(s)
        o = S.Oracle(S.OracleParams(nx=c.nx, ny=c.ny, r=c.r, gamma=c.gamma, nu=c.nu, u_lid=c.u_lid))
        o.step(STEPS)
        _, oux, ouy = o.fields()
        if not (np.all(np.isfinite(oux)) and np.all(np.isfinite(ouy))):
            assert st == L.SLOT_DIVERGED, (c, st)
            continue
        assert st == L.SLOT_MAXSTEPS and info.step == STEPS, (c, st, info.step)
        _, ux, uy = b.fields(s)
        err = np.sqrt(np.sum((ux - oux) ** 2 + (uy - ouy) ** 2) / np.sum(oux ** 2 + ouy ** 2))
        assert err <= 1e-5, (c, err)
        compared += 1
    assert compared >= 6
