"""lbm_step_noalloc: the time step for callers that cannot allocate device
memory (under another allocator that owns the GPU's memory, with a memory
budget fixed at start-up, or in loops that cannot take the synchronisation of
cudaMalloc/cudaFree).  Its scratch is a fixed device array inside the library;
this file checks, for every storage type, that consecutive calls through the C
ABI give the same populations, residual and mass as the ordinary handle-based
lbm_step, and that oversized grids, aliased buffers and null buffers are
refused.  It is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

L = pytest.importorskip("paper_2208_03562_gb300.lbm")
torch = pytest.importorskip("torch")

from oracle import stepper as S  # noqa: E402
from paper_2208_03562_gb300 import inputs as I  # noqa: E402

# storage type -> (torch type of the populations, of the snapshot, largest
# population difference against the handle's step).  Both sides run the same
# general kernel, so the differences are those of adding and removing w_i(r)
# in FP64 on the handle's side: far below one unit in the last place of the
# storage type.
DTYPES = {
    "f64": (L.F64, "float64", "float64", 1e-14),
    "f32": (L.F32, "float32", "float32", 1e-7),
    "f16": (L.F16, "float16", "float32", 1e-6),
}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L.load()


def _setup(code, pop_t, snap_t, nx=200, ny=100, r=0.5, gamma=0.3, nu=0.01, u=0.04):
    p = L.lbm_params_init(nx, ny, r, gamma, nu, u, code)
    pitch = (nx + 31) // 32 * 32
    g0 = I.noise(77, (9, ny, nx), 1e-3).astype(pop_t)
    w = S.rest_weights(S.OracleParams(nx=nx, ny=ny, r=r, gamma=gamma, nu=nu, u_lid=u))
    # the handle-based reference, on the same general kernel everywhere
    h = L.Lbm(p)
    h.variant = -1
    h.set_populations(w[:, None, None] + g0.astype(np.float64))
    ux0 = h.fields()[1]
    dev = torch.device("cuda")
    tt = getattr(torch, pop_t)
    bufs = [torch.zeros((9, ny, pitch), dtype=tt, device=dev) for _ in range(2)]
    bufs[0][:, :, :nx] = torch.from_numpy(g0).to(dev)
    snap = torch.zeros((ny, pitch), dtype=getattr(torch, snap_t), device=dev)
    snap[:, :nx] = torch.from_numpy(ux0.astype(snap_t)).to(dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    return p, h, w, bufs, snap, out


def _call(p, bufs, t, snap, out, with_residual):
    stream = torch.cuda.current_stream().cuda_stream
    L.lbm_step_noalloc(p, bufs[t & 1].data_ptr(), bufs[(t + 1) & 1].data_ptr(), snap.data_ptr(), with_residual,
                       out.data_ptr(), stream)


@pytest.mark.parametrize("dtype", list(DTYPES))
def test_consecutive_calls_match_lbm_step(dtype):
    code, pop_t, snap_t, tol = DTYPES[dtype]
    p, h, w, bufs, snap, out = _setup(code, pop_t, snap_t)
    nx = p.nx
    t = 0
    # two calls in a row, each compared with one ordinary step
    for _ in range(2):
        _call(p, bufs, t, snap, out, False)
        t += 1
        h.step(1)
        torch.cuda.synchronize()
        got = bufs[t & 1][:, :, :nx].double().cpu().numpy()
        ref = h.populations() - w[:, None, None]
        assert np.max(np.abs(got - ref)) < tol
    # residual-evaluating calls at steps 20 and 40 against the handle's
    for target in (20, 40):
        while t < target - 1:
            _call(p, bufs, t, snap, out, False)
            t += 1
        _call(p, bufs, t, snap, out, True)
        t += 1
        h.step(target - h.info().step)
        torch.cuda.synchronize()
        res, mass = out.cpu().numpy()
        info = h.info()
        assert info.step == target and info.residual_step == target
        assert abs(res - info.residual) <= 1e-5 * info.residual
        assert abs(mass - info.mass) <= 1e-9 * p.nx * p.ny
        got = bufs[t & 1][:, :, :nx].double().cpu().numpy()
        assert np.max(np.abs(got - (h.populations() - w[:, None, None]))) < tol
    h.close()


def test_oversized_grid_is_refused():
    p = L.lbm_params_init(4096, 4096, 1.0, 1.0, 0.05, 0.05, L.F32)
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(L.LbmError) as e:
        L.lbm_step_noalloc(p, dummy.data_ptr(), dummy.data_ptr() + 16, dummy.data_ptr(), False, 0,
                           torch.cuda.current_stream().cuda_stream)
    assert e.value.status == L.EINVAL


@pytest.mark.parametrize("dtype", list(DTYPES))
def test_aliased_and_null_buffers_are_refused(dtype):
    """The call checks its arguments before it touches the GPU: src == dst,
    a null population or snapshot buffer, and a residual call without an
    output each return LBM_EINVAL and launch nothing."""
    code, pop_t, snap_t, _ = DTYPES[dtype]
    p = L.lbm_params_init(64, 32, 1.0, 1.0, 0.05, 0.05, code)
    a = torch.zeros((9, 32, 64), dtype=getattr(torch, pop_t), device="cuda")
    b = torch.zeros_like(a)
    snap = torch.zeros((32, 64), dtype=getattr(torch, snap_t), device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    before = a.clone()
    for args in ((a.data_ptr(), a.data_ptr(), snap.data_ptr(), False, 0),
                 (0, b.data_ptr(), snap.data_ptr(), False, 0),
                 (a.data_ptr(), 0, snap.data_ptr(), False, 0),
                 (a.data_ptr(), b.data_ptr(), 0, False, 0),
                 (a.data_ptr(), b.data_ptr(), snap.data_ptr(), True, 0)):
        with pytest.raises(L.LbmError) as e:
            L.lbm_step_noalloc(p, *args[:4], args[4], stream)
        assert e.value.status == L.EINVAL
    torch.cuda.synchronize()
    assert torch.equal(a, before) and not torch.any(b) and not torch.any(out)
