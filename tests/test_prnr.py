"""PRNR-LBM (raw moments, Sec. 4.1 and Sec. 5.3) on the GPU.

The raw-moment scheme runs on the general kernel and the cluster engine. It
must match the oracle's raw-moment mode (FP64 to 1e-10, FP32 to 1e-5), and
the cluster engine must match the general kernel bitwise. Sec. 5.3's claim
that the central and raw schemes converge at the same rate for a fixed gamma
(the shallow cavity, AR = 0.25, r = 0.5, 100 x 50, Re = 100, Ma = 0.06,
gamma = 0.1 and 0.5) must also hold.
"""
import math

import numpy as np
import pytest

from oracle import stepper as S
from paper_2208_03562_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = pytest.importorskip("paper_2208_03562_gb300.lbm")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L.load()


CASES = [
    # nx, ny, r, gamma, nu, u_lid, bc, drho, fx
    (40, 24, 0.5, 0.3, 0.01, 0.03, L.BC_CAVITY, L.DRHO_CURRENT, 0.0),
    (33, 40, 1.0, 1.0, 0.02, 0.05, L.BC_CHANNEL, L.DRHO_OFF, 1e-5),
    (64, 20, 0.25, 0.6, 0.002, 0.0, L.BC_PERIODIC, L.DRHO_CURRENT, 2e-6),
    (70, 19, 2.0, 0.1, 0.01, 0.02, L.BC_CAVITY, L.DRHO_CURRENT, 0.0),
]


def pair(case, dtype, variant):
    nx, ny, r, gamma, nu, u, bc, drho, fx = case
    p = L.lbm_params_init(nx, ny, r, gamma, nu, u, dtype, bc=bc, drho=drho, fx=fx, model=L.MODEL_PRNR)
    g = L.Lbm(p)
    g.variant = variant
    o = S.Oracle(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=u, bc=bc,
                                drho_off=int(drho == L.DRHO_OFF), fx=fx, model=1))
    w = S.rest_weights(o.p if hasattr(o, "p") else S.OracleParams(nx=nx, ny=ny, r=r))
    f0 = w[:, None, None] + I.noise(11 + nx, (9, ny, nx), 1e-3)
    g.set_populations(f0)
    o.set_populations(f0)
    return g, o


@pytest.mark.parametrize("variant", [L.VARIANT_GENERAL, L.VARIANT_CLUSTER])
@pytest.mark.parametrize("dtype,tol", [(L.F64, 1e-10), (L.F32, 1e-5)])
@pytest.mark.parametrize("k", range(len(CASES)))
def test_prnr_matches_oracle(k, dtype, tol, variant):
    g, o = pair(CASES[k], dtype, variant)
    g.step(200)
    o.step(200)
    a, b = g.populations(), o.populations()
    w = S.rest_weights(S.OracleParams(nx=1, ny=1, r=CASES[k][2]))[:, None, None]
    e = np.sqrt(np.sum((a - b) ** 2) / np.sum((b - w) ** 2))
    assert e < tol, e


@pytest.mark.parametrize("dtype", [L.F64, L.F32, L.F16])
def test_prnr_cluster_bitwise_equals_general(dtype):
    for case in CASES:
        g, _ = pair(case, dtype, L.VARIANT_GENERAL)
        c, _ = pair(case, dtype, L.VARIANT_CLUSTER)
        g.step(57)
        c.step(57)
        assert np.array_equal(g.populations(), c.populations())


def test_prnr_differs_from_prc():
    case = CASES[0]
    nx, ny, r, gamma, nu, u, bc, drho, fx = case
    a = L.Lbm(L.lbm_params_init(nx, ny, r, gamma, nu, u, L.F64, model=L.MODEL_PRNR))
    b = L.Lbm(L.lbm_params_init(nx, ny, r, gamma, nu, u, L.F64, model=L.MODEL_PRC))
    a.step(300)
    b.step(300)
    assert np.max(np.abs(a.populations() - b.populations())) > 1e-9
    with pytest.raises(L.LbmError):
        a.variant = 0  # the interior kernel is the central scheme only


@pytest.mark.parametrize("gamma", [0.1, 0.5])
def test_same_convergence_rate_as_prc(gamma):
    """Sec. 5.3: AR = 0.25, r = 0.5, 100 x 50, Re = 100, Ma = 0.06: for a fixed
    gamma both collision models converge at the same rate."""
    nx, ny, r, re, mach = 100, 50, 0.5, 100.0, 0.06
    u = mach * 0.5 / math.sqrt(3.0)
    nu = u * ny * r / re
    steps = {}
    for model in (L.MODEL_PRC, L.MODEL_PRNR):
        h = L.Lbm(L.lbm_params_init(nx, ny, r, gamma, nu, u, L.F32, model=model))
        st, n = h.run(1e-6, 2_000_000)
        assert st == L.OK
        steps[model] = n
    assert abs(steps[L.MODEL_PRC] - steps[L.MODEL_PRNR]) <= 0.1 * steps[L.MODEL_PRC], steps
