"""ctypes front end of the FP64 oracle ``prc_oracle.c`` (oracle-A).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The oracle follows the step list of Appendix A of arXiv:2208.03562 in FP64; its
state is the post-collision population set f~[9][ny][nx] (x fastest).
"""
import ctypes as C
from dataclasses import dataclass, asdict

import numpy as np

from . import build as _build

BC_CAVITY, BC_CHANNEL, BC_PERIODIC = 0, 1, 2


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("r", C.c_double), ("gamma", C.c_double), ("nu", C.c_double), ("u_lid", C.c_double),
        ("omega_xi", C.c_double), ("omega_1", C.c_double), ("omega_21", C.c_double),
        ("omega_12", C.c_double), ("omega_22", C.c_double),
        ("fx", C.c_double), ("fy", C.c_double),
        ("bc", C.c_int), ("drho_off", C.c_int), ("corrections", C.c_int), ("model", C.c_int),
        ("appendix_literal", C.c_int), ("storage_f32", C.c_int),
    ]


@dataclass
class OracleParams:
    """Run parameters in lattice units (dx = dt = 1, dy = r)."""
    nx: int
    ny: int
    r: float = 1.0
    gamma: float = 1.0
    nu: float = 0.1
    u_lid: float = 0.0
    omega_xi: float = 1.0
    omega_1: float = 1.0
    omega_21: float = 1.0
    omega_12: float = 1.0
    omega_22: float = 1.0
    fx: float = 0.0
    fy: float = 0.0
    bc: int = BC_CAVITY
    drho_off: int = 0
    corrections: int = 1
    model: int = 0  # 0: PRC-LBM (central moments); 1: PRNR-LBM (raw moments)
    appendix_literal: int = 0  # 1: App. A's strain-rate residuals as printed (reading A4 not applied)
    storage_f32: int = 0  # 1: stored populations rounded to float32 deviations from w_i(r) every step

    def c(self) -> _Params:
        d = asdict(self)
        return _Params(**d)


_lib = None

_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER(_Params)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [P]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.c_long]
        L.orc_set_populations.argtypes = [C.c_void_p, _D]
        L.orc_get_populations.argtypes = [C.c_void_p, _D]
        L.orc_init_fields.argtypes = [C.c_void_p, _D, _D, _D]
        L.orc_fields.argtypes = [C.c_void_p, _D, _D, _D]
        L.orc_set_rho.argtypes = [C.c_void_p, _D]
        L.orc_density_gradient.argtypes = [C.c_void_p, C.c_int, C.c_int, _D, _D]
        L.orc_residual_update.restype = C.c_double
        L.orc_residual_update.argtypes = [C.c_void_p]
        L.orc_run.restype = C.c_double
        L.orc_run.argtypes = [C.c_void_p, C.c_double, C.c_long, C.POINTER(C.c_long)]
        L.orc_total_mass.restype = C.c_double
        L.orc_total_mass.argtypes = [C.c_void_p]
        L.orc_time.restype = C.c_long
        L.orc_time.argtypes = [C.c_void_p]
        L.orc_collide_node.argtypes = [P, _D, C.c_double, C.c_double, _D, _D]
        L.orc_rest_weights.argtypes = [P, _D]
        L.orc_equilibrium.argtypes = [P, C.c_double, C.c_double, C.c_double, _D]
        L.orc_omega_nu.restype = C.c_double
        L.orc_omega_nu.argtypes = [P]
        L.orc_num_threads.restype = C.c_int
        L.orc_num_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def num_threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return lib().orc_num_threads(n)


def rest_weights(p: OracleParams) -> np.ndarray:
    w = np.zeros(9)
    lib().orc_rest_weights(C.byref(p.c()), _ptr(w))
    return w


def equilibrium(p: OracleParams, rho: float, ux: float, uy: float) -> np.ndarray:
    f = np.zeros(9)
    lib().orc_equilibrium(C.byref(p.c()), rho, ux, uy, _ptr(f))
    return f


def omega_nu(p: OracleParams) -> float:
    return lib().orc_omega_nu(C.byref(p.c()))


def collide_node(p: OracleParams, f, dxrho=0.0, dyrho=0.0):
    """One node's App. A collision. Returns (f~[9], diag) with
    diag = (rho, u_x, u_y, d_x u_x, d_y u_y)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    ft = np.zeros(9)
    diag = np.zeros(5)
    lib().orc_collide_node(C.byref(p.c()), _ptr(f), float(dxrho), float(dyrho), _ptr(ft), _ptr(diag))
    return ft, diag


class Oracle:
    """A whole-grid FP64 run (state: post-collision populations)."""

    def __init__(self, p: OracleParams):
        self.p = p
        self._cp = p.c()
        self._h = lib().orc_create(C.byref(self._cp))
        if not self._h:
            raise MemoryError("oracle allocation failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def shape(self):
        return (self.p.ny, self.p.nx)

    def set_populations(self, ft: np.ndarray):
        ft = np.ascontiguousarray(ft, dtype=np.float64).reshape(9, self.p.ny, self.p.nx)
        lib().orc_set_populations(self._h, _ptr(ft))

    def populations(self) -> np.ndarray:
        ft = np.zeros((9, self.p.ny, self.p.nx))
        lib().orc_get_populations(self._h, _ptr(ft))
        return ft

    def init_fields(self, rho, ux, uy):
        a = [np.ascontiguousarray(np.broadcast_to(v, self.shape), dtype=np.float64) for v in (rho, ux, uy)]
        lib().orc_init_fields(self._h, *[_ptr(v) for v in a])

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def fields(self):
        rho, ux, uy = (np.zeros(self.shape) for _ in range(3))
        lib().orc_fields(self._h, _ptr(rho), _ptr(ux), _ptr(uy))
        return rho, ux, uy

    def residual_update(self) -> float:
        return lib().orc_residual_update(self._h)

    def run(self, tol: float, max_steps: int):
        """Run in blocks of 20 steps to residual < tol; returns (steps, residual)."""
        done = C.c_long(0)
        res = lib().orc_run(self._h, tol, int(max_steps), C.byref(done))
        return done.value, res

    def total_mass(self) -> float:
        return lib().orc_total_mass(self._h)

    @property
    def t(self) -> int:
        return lib().orc_time(self._h)

    # test hooks for the density-gradient stencil
    def set_rho(self, rho):
        rho = np.ascontiguousarray(np.broadcast_to(rho, self.shape), dtype=np.float64)
        lib().orc_set_rho(self._h, _ptr(rho))

    def density_gradient(self, x: int, y: int):
        a, b = C.c_double(), C.c_double()
        lib().orc_density_gradient(self._h, x, y, C.byref(a), C.byref(b))
        return a.value, b.value
