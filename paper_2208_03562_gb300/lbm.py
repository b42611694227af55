"""Python binding of the C ABI in ``include/prc_lbm.h`` (``libprc_lbm.so``).

Argument marshalling only: every step of the method runs in the CUDA kernels of
the library.  Module-level functions carry the C names (``lbm_create``,
``lbm_step``, ``lbm_run``, ``lbm_residual``, ``lbm_fields`` ...); the ``Lbm``
class is a convenience wrapper around one handle.  Loading fails loudly when the
library cannot be built or loaded -- there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

F64, F32, F16 = 0, 1, 2
DTYPE_CODES = {"f64": F64, "f32": F32, "f16": F16}
BC_CAVITY, BC_CHANNEL, BC_PERIODIC = 0, 1, 2
DRHO_CURRENT, DRHO_OFF = 0, 1
MODEL_PRC, MODEL_PRNR = 0, 1

OK, EINVAL, ENOMEM, ECUDA, EDIVERGED, ETIMEOUT, ENOTCONVERGED = range(7)
VARIANT_GENERAL, VARIANT_CLUSTER = -1, -2
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EDIVERGED", "ETIMEOUT", "ENOTCONVERGED"]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status


class lbm_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32),
                ("r", C.c_double), ("gamma", C.c_double), ("nu", C.c_double), ("u_lid", C.c_double),
                ("omega_xi", C.c_double), ("fx", C.c_double), ("fy", C.c_double),
                ("dtype", C.c_int32), ("bc", C.c_int32), ("drho", C.c_int32), ("model", C.c_int32)]


class lbm_info_t(C.Structure):
    _fields_ = [("step", C.c_int64), ("residual_step", C.c_int64), ("residual", C.c_double),
                ("mass", C.c_double), ("converged", C.c_int32), ("diverged", C.c_int32)]


_lib = None
_D = C.POINTER(C.c_double)
_H = C.c_void_p


def load():
    """Build (if stale) and load libprc_lbm.so; raise if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise ImportError("libprc_lbm.so missing at %s" % path)
    L = C.CDLL(path)
    P = C.POINTER(lbm_params)
    sig = {
        "lbm_params_init": [P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int],
        "lbm_params_check": [P],
        "lbm_workspace_bytes": [P, C.POINTER(C.c_size_t)],
        "lbm_omega_nu": [P, _D],
        "lbm_create": [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.POINTER(_H)],
        "lbm_create_p": [P, C.POINTER(_H)],
        "lbm_create_ex": [P, C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(_H)],
        "lbm_set_stream": [_H, C.c_void_p],
        "lbm_step": [_H, C.c_long],
        "lbm_run": [_H, C.c_double, C.c_long, C.POINTER(C.c_long)],
        "lbm_residual": [_H, _D],
        "lbm_mass": [_H, _D],
        "lbm_set_mass": [_H, C.c_double],
        "lbm_info": [_H, C.POINTER(lbm_info_t)],
        "lbm_sync": [_H],
        "lbm_fields": [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int],
        "lbm_init_fields": [_H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int],
        "lbm_set_populations": [_H, C.c_void_p, C.c_int],
        "lbm_get_populations": [_H, C.c_void_p, C.c_int],
        "lbm_variant_count": [C.c_int, C.POINTER(C.c_int)],
        "lbm_variant_info": [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                             C.POINTER(C.c_int)],
        "lbm_get_variant": [_H, C.POINTER(C.c_int)],
        "lbm_set_variant": [_H, C.c_int],
        "lbm_autotune": [_H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)],
        "lbm_step_noalloc": [P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
        "lbm_save_bytes": [_H, C.POINTER(C.c_size_t)],
        "lbm_save": [_H, C.c_void_p, C.c_size_t],
        "lbm_load": [_H, C.c_void_p, C.c_size_t],
    }
    B = C.c_void_p
    sig.update({
        "lbm_batch_create": [C.c_int, C.c_int, C.c_void_p, C.POINTER(B)],
        "lbm_batch_instance_bytes": [P, C.POINTER(C.c_size_t)],
        "lbm_batch_add": [B, P, C.c_double, C.c_long, C.POINTER(C.c_int)],
        "lbm_batch_remove": [B, C.c_int],
        "lbm_batch_set_stall": [B, C.c_int, C.c_long, C.c_double],
        "lbm_batch_set_wait_limit": [B, C.c_longlong, C.c_int],
        "lbm_batch_set_ctas_per_sm": [B, C.c_int],
        "lbm_batch_set_body": [B, C.c_int],
        "lbm_batch_get_body": [B, C.POINTER(C.c_int)],
        "lbm_batch_get_ctas_per_sm": [B, C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "lbm_batch_autotune": [B, C.c_int, C.POINTER(C.c_int), _D],
        "lbm_batch_launch": [B, C.c_long, C.c_int],
        "lbm_batch_wait": [B, C.POINTER(C.c_int)],
        "lbm_batch_run": [B, C.c_long, C.POINTER(C.c_int)],
        "lbm_batch_query": [B, C.c_int, C.POINTER(lbm_info_t), C.POINTER(C.c_int)],
        "lbm_batch_fields": [B, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int],
        "lbm_batch_set_populations": [B, C.c_int, C.c_void_p, C.c_int],
        "lbm_batch_get_populations": [B, C.c_int, C.c_void_p, C.c_int],
        "lbm_batch_mass": [B, C.c_int, _D],
        "lbm_batch_set_mass": [B, C.c_int, C.c_double],
    })
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.lbm_destroy.argtypes = [_H]
    L.lbm_destroy.restype = None
    L.lbm_last_error.argtypes = [_H]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_batch_destroy.argtypes = [C.c_void_p]
    L.lbm_batch_destroy.restype = None
    L.lbm_batch_last_error.argtypes = [C.c_void_p]
    L.lbm_batch_last_error.restype = C.c_char_p
    _lib = L
    return L


def exported_symbols():
    """Names of the ``lbm_*`` entry points the loaded library resolves."""
    L = load()
    out = []
    for name in ("lbm_params_init", "lbm_params_check", "lbm_workspace_bytes", "lbm_omega_nu", "lbm_create",
                 "lbm_create_p", "lbm_create_ex", "lbm_set_stream", "lbm_destroy", "lbm_last_error",
                 "lbm_step", "lbm_run", "lbm_residual", "lbm_mass", "lbm_info", "lbm_sync", "lbm_fields",
                 "lbm_init_fields", "lbm_set_populations", "lbm_get_populations", "lbm_save_bytes",
                 "lbm_save", "lbm_load", "lbm_variant_count", "lbm_variant_info",
                 "lbm_get_variant",
                 "lbm_set_variant", "lbm_autotune", "lbm_step_noalloc", "lbm_batch_create",
                 "lbm_batch_destroy", "lbm_batch_last_error", "lbm_batch_instance_bytes", "lbm_batch_add",
                 "lbm_batch_remove", "lbm_batch_set_stall", "lbm_batch_set_wait_limit",
                 "lbm_batch_set_ctas_per_sm", "lbm_batch_get_ctas_per_sm", "lbm_batch_set_body",
                 "lbm_batch_get_body", "lbm_batch_autotune", "lbm_batch_launch", "lbm_batch_wait", "lbm_batch_run",
                 "lbm_batch_query",
                 "lbm_batch_fields", "lbm_batch_set_populations", "lbm_batch_get_populations",
                 "lbm_batch_mass", "lbm_batch_set_mass", "lbm_set_mass"):
        if hasattr(L, name):
            out.append(name)
    return out


def _check(status, h=None):
    if status != OK:
        msg = load().lbm_last_error(h)
        raise LbmError(status, msg.decode() if msg else "")
    return status


# ---------------------------------------------------------------------------
# C-named functions

def lbm_params_init(nx, ny, r, gamma, nu, u_lid, dtype=F32, bc=BC_CAVITY, drho=DRHO_CURRENT,
                    omega_xi=1.0, fx=0.0, fy=0.0, model=MODEL_PRC) -> lbm_params:
    p = lbm_params()
    _check(load().lbm_params_init(C.byref(p), nx, ny, r, gamma, nu, u_lid, dtype))
    p.bc, p.drho, p.omega_xi, p.fx, p.fy, p.model = bc, drho, omega_xi, fx, fy, model
    return p


def lbm_params_check(p: lbm_params):
    return _check(load().lbm_params_check(C.byref(p)))


def lbm_workspace_bytes(p: lbm_params) -> int:
    n = C.c_size_t()
    _check(load().lbm_workspace_bytes(C.byref(p), C.byref(n)))
    return n.value


def lbm_omega_nu(p: lbm_params) -> float:
    w = C.c_double()
    _check(load().lbm_omega_nu(C.byref(p), C.byref(w)))
    return w.value


def lbm_create(nx, ny, r, gamma, nu, u_lid, dtype=F32):
    h = _H()
    _check(load().lbm_create(nx, ny, r, gamma, nu, u_lid, dtype, C.byref(h)))
    return h


def lbm_create_p(p: lbm_params):
    h = _H()
    _check(load().lbm_create_p(C.byref(p), C.byref(h)))
    return h


def lbm_create_ex(p: lbm_params, workspace_ptr: int, workspace_bytes: int, stream_ptr: int):
    h = _H()
    _check(load().lbm_create_ex(C.byref(p), C.c_void_p(workspace_ptr), workspace_bytes,
                                C.c_void_p(stream_ptr), C.byref(h)))
    return h


def lbm_destroy(h):
    load().lbm_destroy(h)


def lbm_step(h, n):
    _check(load().lbm_step(h, int(n)), h)


def lbm_run(h, tol, max_steps):
    """Returns (status, steps_done); raises only on errors other than
    ENOTCONVERGED."""
    done = C.c_long()
    s = load().lbm_run(h, float(tol), int(max_steps), C.byref(done))
    if s not in (OK, ENOTCONVERGED):
        _check(s, h)
    return s, done.value


def lbm_residual(h) -> float:
    v = C.c_double()
    _check(load().lbm_residual(h, C.byref(v)), h)
    return v.value


def lbm_mass(h) -> float:
    v = C.c_double()
    _check(load().lbm_mass(h, C.byref(v)), h)
    return v.value


def lbm_set_mass(h, mass: float):
    _check(load().lbm_set_mass(h, float(mass)), h)


def lbm_info(h) -> lbm_info_t:
    info = lbm_info_t()
    _check(load().lbm_info(h, C.byref(info)), h)
    return info


def lbm_sync(h):
    _check(load().lbm_sync(h), h)


def _host_ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.c_void_p)


def lbm_fields(h, ny, nx):
    rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
    _check(load().lbm_fields(h, _host_ptr(rho), _host_ptr(ux), _host_ptr(uy), 0), h)
    return rho, ux, uy


def lbm_fields_device(h, rho_ptr, ux_ptr, uy_ptr):
    _check(load().lbm_fields(h, C.c_void_p(rho_ptr), C.c_void_p(ux_ptr), C.c_void_p(uy_ptr), 1), h)


def lbm_init_fields(h, rho, ux, uy):
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (rho, ux, uy)]
    _check(load().lbm_init_fields(h, *[_host_ptr(v) for v in a], 0), h)


def lbm_set_populations(h, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(load().lbm_set_populations(h, _host_ptr(f), 0), h)


def lbm_get_populations(h, ny, nx):
    f = np.empty((9, ny, nx))
    _check(load().lbm_get_populations(h, _host_ptr(f), 0), h)
    return f


def lbm_variant_count(dtype) -> int:
    n = C.c_int()
    _check(load().lbm_variant_count(dtype, C.byref(n)))
    return n.value


def lbm_variant_info(dtype, variant):
    """(tile_w, tile_h, threads, ctas_per_sm) of an interior-kernel variant."""
    v = [C.c_int() for _ in range(4)]
    _check(load().lbm_variant_info(dtype, variant, *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


def lbm_get_variant(h) -> int:
    v = C.c_int()
    _check(load().lbm_get_variant(h, C.byref(v)), h)
    return v.value


def lbm_set_variant(h, variant):
    _check(load().lbm_set_variant(h, int(variant)), h)


def lbm_autotune(h, dtype, steps=20):
    """Time every candidate on the handle's grid; selects the fastest.
    Returns (best, [ms per step of each interior variant, then of the
    cluster engine (-1 when it does not fit), then of the general kernel])."""
    n = lbm_variant_count(dtype)
    ms = (C.c_double * (n + 2))()
    best = C.c_int()
    _check(load().lbm_autotune(h, int(steps), C.byref(best), ms), h)
    return best.value, [ms[i] for i in range(n + 2)]


def lbm_step_noalloc(p: lbm_params, src_ptr: int, dst_ptr: int, snap_ptr: int, with_residual: bool,
                     out_ptr: int, stream_ptr: int):
    """One step on caller-owned device buffers, no device allocation (see
    the header for the buffer layout and the shared-scratch rules)."""
    _check(load().lbm_step_noalloc(C.byref(p), C.c_void_p(src_ptr), C.c_void_p(dst_ptr), C.c_void_p(snap_ptr),
                                   1 if with_residual else 0, C.c_void_p(out_ptr), C.c_void_p(stream_ptr)))


def lbm_save(h) -> bytes:
    n = C.c_size_t()
    _check(load().lbm_save_bytes(h, C.byref(n)), h)
    buf = (C.c_char * n.value)()
    _check(load().lbm_save(h, buf, n.value), h)
    return bytes(buf)


def lbm_load(h, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().lbm_load(h, buf, len(blob)), h)


# ---------------------------------------------------------------------------
# convenience wrapper

class Lbm:
    """One PRC-LBM instance on the current CUDA device.

    ``Lbm(params)`` lets the library own its memory and stream;
    ``Lbm(params, torch_workspace=True)`` places every buffer in one PyTorch
    uint8 tensor and enqueues on PyTorch's current stream.
    """

    def __init__(self, params: lbm_params, torch_workspace: bool = False):
        self.p = params
        self._ws = None
        if torch_workspace:
            import torch
            nbytes = lbm_workspace_bytes(params)
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            base = (base + 255) // 256 * 256
            self.h = lbm_create_ex(params, base, nbytes, torch.cuda.current_stream().cuda_stream)
        else:
            self.h = lbm_create_p(params)

    @classmethod
    def cavity(cls, cav, bc=BC_CAVITY, drho=DRHO_CURRENT, **kw):
        """From a ``inputs.Cavity`` workload description."""
        p = lbm_params_init(cav.nx, cav.ny, cav.r, cav.gamma, cav.nu, cav.u_lid, DTYPE_CODES[cav.dtype],
                            bc=bc, drho=drho)
        return cls(p, **kw)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.p.ny, self.p.nx)

    def step(self, n=1):
        lbm_step(self.h, n)

    def run(self, tol, max_steps):
        return lbm_run(self.h, tol, max_steps)

    def residual(self):
        return lbm_residual(self.h)

    def mass(self):
        return lbm_mass(self.h)

    def info(self):
        return lbm_info(self.h)

    def set_mass(self, mass: float):
        lbm_set_mass(self.h, mass)

    def sync(self):
        lbm_sync(self.h)

    def fields(self):
        return lbm_fields(self.h, self.p.ny, self.p.nx)

    def init_fields(self, rho, ux, uy):
        shape = self.shape
        lbm_init_fields(self.h, *[np.broadcast_to(v, shape) for v in (rho, ux, uy)])

    def set_populations(self, f):
        lbm_set_populations(self.h, np.reshape(f, (9,) + self.shape))

    def populations(self):
        return lbm_get_populations(self.h, self.p.ny, self.p.nx)

    @property
    def variant(self) -> int:
        return lbm_get_variant(self.h)

    @variant.setter
    def variant(self, v):
        lbm_set_variant(self.h, v)

    def autotune(self, steps=20):
        return lbm_autotune(self.h, self.p.dtype, steps)

    def save(self) -> bytes:
        return lbm_save(self.h)

    def load(self, blob: bytes):
        lbm_load(self.h, blob)


# ---------------------------------------------------------------------------
# batched engine

SLOT_ACTIVE, SLOT_CONVERGED, SLOT_DIVERGED, SLOT_MAXSTEPS, SLOT_EMPTY, SLOT_STALLED = range(6)
BATCH_BODY_AUTO, BATCH_BODY_GENERAL = 0, 1
SLOT_NAMES = ["ACTIVE", "CONVERGED", "DIVERGED", "MAXSTEPS", "EMPTY", "STALLED"]


def _bcheck(status, b):
    if status != OK:
        msg = load().lbm_batch_last_error(b)
        raise LbmError(status, msg.decode() if msg else "")
    return status


def lbm_batch_instance_bytes(p: lbm_params) -> int:
    n = C.c_size_t()
    _check(load().lbm_batch_instance_bytes(C.byref(p), C.byref(n)))
    return n.value


class Batch:
    """Wrapper of an lbm_batch_t: independent instances in one persistent
    launch (see include/prc_lbm.h)."""

    def __init__(self, capacity: int, dtype: int, stream_ptr: int = 0):
        self.dtype = dtype
        self.b = C.c_void_p()
        _bcheck(load().lbm_batch_create(capacity, dtype, C.c_void_p(stream_ptr), C.byref(self.b)), None)
        self.shapes = {}

    def close(self):
        if getattr(self, "b", None):
            load().lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, p: lbm_params, tol: float, max_steps: int) -> int:
        s = C.c_int()
        _bcheck(load().lbm_batch_add(self.b, C.byref(p), float(tol), int(max_steps), C.byref(s)), self.b)
        self.shapes[s.value] = (p.ny, p.nx)
        return s.value

    def remove(self, slot: int):
        _bcheck(load().lbm_batch_remove(self.b, slot), self.b)
        self.shapes.pop(slot, None)

    def set_stall(self, slot: int, window: int, ratio: float):
        """Retire the slot as STALLED when its residual stops falling (see
        lbm_batch_set_stall); window = 0 turns the test off."""
        _bcheck(load().lbm_batch_set_stall(self.b, slot, int(window), float(ratio)), self.b)

    def set_wait_limit(self, cycles: int, hold: bool = False):
        """For the next launch only: the grid-barrier wait limit in SM cycles
        (0: the default) and, with hold, a withheld arrival that makes the
        waits run out (lbm_batch_set_wait_limit)."""
        _bcheck(load().lbm_batch_set_wait_limit(self.b, int(cycles), 1 if hold else 0), self.b)

    @property
    def ctas_per_sm(self) -> int:
        """Resident CTAs per SM of the persistent grid (lbm_batch_get_ctas_per_sm)."""
        c = C.c_int()
        _bcheck(load().lbm_batch_get_ctas_per_sm(self.b, C.byref(c), None), self.b)
        return c.value

    @ctas_per_sm.setter
    def ctas_per_sm(self, value: int):
        _bcheck(load().lbm_batch_set_ctas_per_sm(self.b, int(value)), self.b)

    def set_body(self, body: int):
        """BATCH_BODY_AUTO (TMA-staged interior tiles when the launch allows
        them) or BATCH_BODY_GENERAL (lbm_batch_set_body)."""
        _bcheck(load().lbm_batch_set_body(self.b, int(body)), self.b)

    @property
    def tma_body(self) -> bool:
        """The next launch takes the TMA-staged body (lbm_batch_get_body)."""
        t = C.c_int()
        _bcheck(load().lbm_batch_get_body(self.b, C.byref(t)), self.b)
        return bool(t.value)

    @property
    def max_ctas_per_sm(self) -> int:
        m = C.c_int()
        _bcheck(load().lbm_batch_get_ctas_per_sm(self.b, None, C.byref(m)), self.b)
        return m.value

    def autotune(self, steps: int = 20):
        """Time every persistent-grid size on the active slots, restore their
        state and keep the fastest (lbm_batch_autotune).  Returns (best
        ctas_per_sm, milliseconds per step for ctas_per_sm = 1, 2, ...)."""
        n = self.max_ctas_per_sm
        best = C.c_int()
        ms = (C.c_double * n)(*([-1.0] * n))
        _bcheck(load().lbm_batch_autotune(self.b, int(steps), C.byref(best), ms), self.b)
        return best.value, list(ms)

    def launch(self, steps: int, use_graph: bool = True):
        _bcheck(load().lbm_batch_launch(self.b, int(steps), 1 if use_graph else 0), self.b)

    def wait(self) -> int:
        n = C.c_int()
        _bcheck(load().lbm_batch_wait(self.b, C.byref(n)), self.b)
        return n.value

    def run(self, steps: int, use_graph: bool = True) -> int:
        self.launch(steps, use_graph)
        return self.wait()

    def query(self, slot: int):
        info, st = lbm_info_t(), C.c_int()
        _bcheck(load().lbm_batch_query(self.b, slot, C.byref(info), C.byref(st)), self.b)
        return info, st.value

    def fields(self, slot: int):
        ny, nx = self.shapes[slot]
        rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
        _bcheck(load().lbm_batch_fields(self.b, slot, _host_ptr(rho), _host_ptr(ux), _host_ptr(uy), 0), self.b)
        return rho, ux, uy

    def set_populations(self, slot: int, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        _bcheck(load().lbm_batch_set_populations(self.b, slot, _host_ptr(f), 0), self.b)

    def populations(self, slot: int):
        ny, nx = self.shapes[slot]
        f = np.empty((9, ny, nx))
        _bcheck(load().lbm_batch_get_populations(self.b, slot, _host_ptr(f), 0), self.b)
        return f

    def mass(self, slot: int) -> float:
        m = C.c_double()
        _bcheck(load().lbm_batch_mass(self.b, slot, C.byref(m)), self.b)
        return m.value

    def set_mass(self, slot: int, mass: float):
        """Uniform density shift of a slot to the given total mass (see lbm_set_mass)."""
        _bcheck(load().lbm_batch_set_mass(self.b, slot, float(mass)), self.b)

    def populations_to_device(self, slot: int, f_ptr: int):
        """Full FP64 populations of a slot into a device buffer of 9 ny nx doubles."""
        _bcheck(load().lbm_batch_get_populations(self.b, slot, C.c_void_p(f_ptr), 1), self.b)

    def set_populations_from_device(self, slot: int, f_ptr: int):
        """Set a slot from a device buffer of 9 ny nx FP64 full populations."""
        _bcheck(load().lbm_batch_set_populations(self.b, slot, C.c_void_p(f_ptr), 1), self.b)
