"""Degenerate and edge cases of the method on every engine.

- The uniform rest state with a resting lid is a fixed point of the step
  (Sec. 5.1 cavity, u_lid = 0): the stored deviations f_i - w_i(r) stay
  exactly zero, the residual exactly zero and the mass exactly nx * ny, in
  every storage format and on every engine.
- The smallest grids (3 x 3 and odd widths, whose last node pair holds one
  node) match the FP64 oracle on the cluster engine and on the general
  kernel, in every storage format.
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


def rest_weights(nx, ny, r, gamma, nu):
    return S.rest_weights(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=0.0))


@pytest.mark.parametrize("dtype", [L.F64, L.F32, L.F16])
@pytest.mark.parametrize("variant", [L.VARIANT_CLUSTER, L.VARIANT_GENERAL, 0])
def test_rest_is_a_fixed_point(dtype, variant):
    nx, ny, r, gamma, nu = 200, 100, 0.5, 0.3, 0.01
    if variant == 0 and dtype == L.F64:
        pytest.skip("no interior kernel for FP64 storage")
    h = L.Lbm(L.lbm_params_init(nx, ny, r, gamma, nu, 0.0, dtype))
    h.variant = variant
    p0 = h.populations()
    w = rest_weights(nx, ny, r, gamma, nu)[:, None, None]
    assert np.max(np.abs(p0 - w)) < 1e-15  # the library's rest state is w_i(r)
    h.step(60)
    assert np.array_equal(h.populations(), p0)
    info = h.info()
    assert info.residual == 0.0 and info.mass == float(nx * ny)
    h.close()


@pytest.mark.parametrize("dtype", [L.F64, L.F32, L.F16])
def test_rest_is_a_fixed_point_in_a_batch(dtype):
    shapes = [(3, 3), (77, 45), (130, 64)]
    b = L.Batch(len(shapes), dtype)
    slots = [b.add(L.lbm_params_init(nx, ny, 1.0, 0.5, 0.02, 0.0, dtype), 0.0, 10 ** 6) for nx, ny in shapes]
    p0 = [b.populations(s) for s in slots]
    b.run(60)
    for (nx, ny), s, p in zip(shapes, slots, p0):
        w = rest_weights(nx, ny, 1.0, 0.5, 0.02)[:, None, None]
        assert np.max(np.abs(p - w)) < 1e-15
        assert np.array_equal(b.populations(s), p)
        info, st = b.query(s)
        assert st == L.SLOT_ACTIVE and info.residual == 0.0 and info.mass == float(nx * ny)


TINY = [
    # nx, ny, r, gamma, nu, u_lid
    (3, 3, 1.0, 1.0, 0.05, 0.05),
    (4, 3, 0.5, 0.4, 0.02, 0.02),
    (3, 5, 2.0, 0.2, 0.01, 0.02),
    (5, 7, 0.5, 0.25, 0.01, 0.02),
    (9, 4, 1.6, 0.6, 0.01, 0.03),
]


@pytest.mark.parametrize("variant", [L.VARIANT_CLUSTER, L.VARIANT_GENERAL])
@pytest.mark.parametrize("dtype,tol", [(L.F64, 1e-13), (L.F32, 2e-7), (L.F16, 2e-5)])
@pytest.mark.parametrize("case", TINY)
def test_smallest_grids_match_the_oracle(case, dtype, tol, variant):
    nx, ny, r, gamma, nu, u = case
    h = L.Lbm(L.lbm_params_init(nx, ny, r, gamma, nu, u, dtype))
    h.variant = variant
    o = S.Oracle(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=u))
    w = S.rest_weights(o.p)[:, None, None]
    f0 = w + I.noise(nx * 31 + ny, (9, ny, nx), 1e-3)
    h.set_populations(f0)
    o.set_populations(f0)
    for n in (1, 4, 15):
        h.step(n)
        o.step(n)
        d = np.max(np.abs((h.populations() - w) - (o.populations() - w)))
        assert d < tol * max(1.0, n / 4), (n, d)
    h.close()
