"""Cluster-resident engine for small grids (variant LBM_VARIANT_CLUSTER).

One thread-block cluster keeps the whole state in distributed shared memory
and runs many steps per launch. It performs the same per-node arithmetic as
the general kernel (scalar FP64; pairs of neighbouring nodes in packed FP32x2
for the FP32 collision), so its populations must be bitwise those of the
general kernel, step for step, across wall types, the density-gradient mode,
body forces and storage types. It must also stop on the device at the same step
when run to a residual.
"""
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
    (77, 45, 2.0, 0.1, 0.01, 0.02, L.BC_CAVITY, L.DRHO_CURRENT, 0.0),
    (33, 40, 1.0, 1.0, 0.02, 0.05, L.BC_CHANNEL, L.DRHO_OFF, 1e-5),
    (96, 32, 0.25, 0.6, 0.002, 0.01, L.BC_PERIODIC, L.DRHO_CURRENT, 2e-6),
    (128, 128, 2.0, 0.1, 0.0128, 0.0346, L.BC_CAVITY, L.DRHO_CURRENT, 0.0),
    (5, 7, 1.6, 0.2, 0.005, 0.01, L.BC_CAVITY, L.DRHO_CURRENT, 0.0),
]


def params(case, dtype):
    nx, ny, r, gamma, nu, u, bc, drho, fx = case
    return L.lbm_params_init(nx, ny, r, gamma, nu, u, dtype, bc=bc, drho=drho, fx=fx)


def start(case, seed):
    nx, ny, r, gamma, nu, u, bc, drho, fx = case
    w = S.rest_weights(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=u))
    return w[:, None, None] + I.noise(seed, (9, ny, nx), 1e-3)


def handle(case, dtype, variant, f0):
    h = L.Lbm(params(case, dtype))
    h.variant = variant
    h.set_populations(f0)
    return h


@pytest.mark.parametrize("dtype", [L.F64, L.F32, L.F16])
@pytest.mark.parametrize("k", range(len(CASES)))
def test_cluster_bitwise_equals_general(dtype, k):
    case = CASES[k]
    f0 = start(case, 300 + k)
    c = handle(case, dtype, L.VARIANT_CLUSTER, f0)
    g = handle(case, dtype, L.VARIANT_GENERAL, f0)
    for n in (1, 19, 37):  # split launches, crossing residual steps
        c.step(n)
        g.step(n)
        assert np.array_equal(c.populations(), g.populations())
        ic, ig = c.info(), g.info()
        assert ic.step == ig.step and ic.residual_step == ig.residual_step
        if ic.residual_step:
            assert abs(ic.residual - ig.residual) <= 1e-9 * ig.residual
            assert abs(ic.mass - ig.mass) <= 1e-12 * ig.mass


def test_cluster_is_the_default_for_small_grids():
    assert L.Lbm(L.lbm_params_init(128, 128, 2.0, 0.1, 0.0128, 0.0346, L.F32)).variant == L.VARIANT_CLUSTER
    big = L.Lbm(L.lbm_params_init(1024, 1024, 1.0, 1.0, 0.05, 0.05, L.F32))
    assert big.variant == 0
    with pytest.raises(L.LbmError):
        big.variant = L.VARIANT_CLUSTER


@pytest.mark.parametrize("dtype", [L.F64, L.F32])
def test_cluster_run_stops_where_the_general_kernel_stops(dtype):
    cav = I.Cavity(48, 24, 0.5, 0.5, 20.0, 0.02, "f32")
    p = L.lbm_params_init(cav.nx, cav.ny, cav.r, cav.gamma, cav.nu, cav.u_lid, dtype)
    c, g = L.Lbm(p), L.Lbm(p)
    assert c.variant == L.VARIANT_CLUSTER
    g.variant = L.VARIANT_GENERAL
    sc, nc = c.run(1e-6, 400000)
    sg, ng = g.run(1e-6, 400000)
    assert sc == sg == L.OK and nc == ng and nc % 20 == 0
    assert np.array_equal(c.populations(), g.populations())
    # stepping on after convergence continues from the stopped state
    c.step(40)
    g.step(40)
    assert np.array_equal(c.populations(), g.populations())


def test_cluster_autotune_restores_state():
    p = L.lbm_params_init(64, 64, 1.0, 1.0, 0.064, 0.1, L.F32)
    h = L.Lbm(p)
    h.step(33)
    before = h.populations()
    best, ms = h.autotune(20)
    nv = L.lbm_variant_count(L.F32)
    assert len(ms) == nv + 2 and ms[nv] > 0 and ms[nv + 1] > 0
    assert np.array_equal(h.populations(), before) and h.info().step == 33


@pytest.mark.parametrize("model", [L.MODEL_PRC, L.MODEL_PRNR])
def test_handles_of_different_sizes_coexist(model):
    """The engine's shared-memory opt-in is a property of the kernel, not of a
    handle: creating a handle with smaller slabs (and of either scheme) after
    one with larger slabs must leave the larger one runnable."""
    def mk(nx, ny, m):
        h = L.Lbm(L.lbm_params_init(nx, ny, 4.0 / 3.0, 0.5, 0.007, 0.0346, L.F32, model=m))
        assert h.variant == L.VARIANT_CLUSTER
        return h
    big = mk(100, 150, L.MODEL_PRC)
    small = mk(100, 125, model)
    big.step(40)
    small.step(40)
    big.step(40)
    ref = mk(100, 150, L.MODEL_PRC)
    ref.step(80)
    assert np.array_equal(big.populations(), ref.populations())
    for h in (big, small, ref):
        h.close()
