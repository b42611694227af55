"""Seeded synthetic inputs and workload definitions.

This module is shared by the tests, the oracle runs and the CUDA path.  It holds
no arithmetic of the lattice Boltzmann method itself: only random numbers,
smooth initial fields, and the parameters of the cavity workloads (grid, aspect
ratio r, preconditioning gamma, Reynolds and Mach numbers).

Conventions (lattice units, dx = dt = 1, dy = r): node (i, j) sits at
x = i + 1/2, y = (j + 1/2) r; a cavity has length L = nx and height H = ny r, so
its geometric aspect ratio is AR = H / L = ny r / nx (Sec. 5.2: r = AR Nx / Ny).
"""
from dataclasses import dataclass, asdict
import math

import numpy as np

CS_STAR = 1.0 / math.sqrt(3.0)  # Eq. 1, square-lattice sound speed


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# random states

def noise(seed: int, shape, amp: float) -> np.ndarray:
    """Gaussian noise N(0, amp^2) of the given shape (FP64)."""
    return amp * rng(seed).standard_normal(shape)


def random_fields(seed: int, nx: int, ny: int, drho: float = 1e-2, u: float = 0.05):
    """Smooth-free random fields rho = 1 + drho N, u ~ u N (FP64, [ny][nx])."""
    g = rng(seed)
    rho = 1.0 + drho * g.standard_normal((ny, nx))
    ux = u * g.standard_normal((ny, nx))
    uy = u * g.standard_normal((ny, nx))
    return rho, ux, uy


def sample_nodes(seed: int, k: int, nx: int, ny: int) -> np.ndarray:
    """k distinct flat node indexes (y * nx + x) drawn without replacement."""
    return np.sort(rng(seed).choice(nx * ny, size=min(k, nx * ny), replace=False))


def projection_signs(seed: int, k: int, nx: int, ny: int) -> np.ndarray:
    """k random +-1 fields of shape (k, 2, ny, nx): weights of k random
    projections of a velocity field (u_x, u_y).  For a difference field d,
    the mean of (sum w d)^2 over the projections is an unbiased estimate of
    ||d||_2^2, so a few stored projections let a test estimate the L2
    distance to a field it does not hold."""
    return np.where(rng(seed).standard_normal((k, 2, ny, nx)) >= 0.0, 1.0, -1.0)


def node_coords(nx: int, ny: int, r: float):
    """Physical node centres x = i + 1/2, y = (j + 1/2) r as [ny][nx] arrays."""
    x = np.arange(nx) + 0.5
    y = (np.arange(ny) + 0.5) * r
    return np.meshgrid(x, y)


def shear_wave(nx: int, ny: int, r: float, amp: float, along: str = "y"):
    """u_x = amp sin(2 pi y / H) (along='y') or u_y = amp sin(2 pi x / L)."""
    X, Y = node_coords(nx, ny, r)
    rho = np.ones((ny, nx))
    if along == "y":
        return rho, amp * np.sin(2 * np.pi * Y / (ny * r)), np.zeros((ny, nx))
    return rho, np.zeros((ny, nx)), amp * np.sin(2 * np.pi * X / nx)


def taylor_green(nx: int, ny: int, r: float, amp: float, u0: float = 0.0):
    """Divergence-free vortex array on the periodic box L = nx, H = ny r,
    u = amp (ky/k sin(kx x) cos(ky y), -kx/k cos(kx x) sin(ky y)) + (u0, 0)."""
    X, Y = node_coords(nx, ny, r)
    kx, ky = 2 * np.pi / nx, 2 * np.pi / (ny * r)
    k = math.hypot(kx, ky)
    ux = u0 + amp * (ky / k) * np.sin(kx * X) * np.cos(ky * Y)
    uy = -amp * (kx / k) * np.cos(kx * X) * np.sin(ky * Y)
    return np.ones((ny, nx)), ux, uy


# --------------------------------------------------------------------------
# cavity workloads

DTYPES = ("f64", "f32", "f16")


@dataclass
class Cavity:
    """A lid-driven cavity: nx x ny nodes, aspect ratio r, preconditioning
    gamma, Reynolds number Re = U H / nu with H = ny r, lid speed u_lid."""
    nx: int
    ny: int
    r: float
    gamma: float
    re: float
    u_lid: float
    dtype: str = "f32"
    tol: float = 1e-7
    max_steps: int = 2_000_000

    @property
    def height(self) -> float:
        return self.ny * self.r

    @property
    def nu(self) -> float:
        return self.u_lid * self.height / self.re

    @property
    def mach(self) -> float:
        """Ma = U / c_s with c_s = min(1, r) c_s* (Eq. 2)."""
        return self.u_lid / (min(1.0, self.r) * CS_STAR)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def asdict(self):
        return asdict(self)


def lid_speed_for_mach(r: float, mach: float, cap: float = 0.05) -> float:
    """U = Ma c_s with c_s = min(1, r) c_s* (Eq. 2), capped."""
    return min(cap, mach * min(1.0, r) * CS_STAR)


def sweep_mach(gamma: float) -> float:
    """Lid Mach number of the synthetic sweeps: 0.1, lowered to gamma / 2 for
    strong preconditioning. The paper notes that the smallest usable gamma
    grows with the Mach number (Sec. 5.2). Its own stable runs keep
    Ma / gamma <= 0.75."""
    return min(0.1, 0.5 * gamma)


def square_cavity_64() -> Cavity:
    """64 x 64 square lattice, r = gamma = 1, Re = 100, U = 0.1, FP64,
    to residual 1e-8 or 20000 steps."""
    return Cavity(64, 64, 1.0, 1.0, 100.0, 0.1, "f64", 1e-8, 20000)


def deep_cavity_128(gamma: float = 0.1, dtype: str = "f32", u_lid: float = None) -> Cavity:
    """128 x 128 nodes, r = 2 (H/L = 2), Re = 1000, to residual 1e-7.

    The lid speed defaults to Ma = 0.06 (U = 0.06 c_s*, the Mach number of the
    paper's deep-cavity runs at Re = 1000, Sec. 5.2).  With U = 0.05 and
    gamma = 0.1 (Ma = 0.087, U / gamma = 0.5) the corrected scheme diverges
    within ~200 steps from an impulsive start: ``deep_cavity_128_as_stated``."""
    if u_lid is None:
        u_lid = 0.06 * CS_STAR
    return Cavity(128, 128, 2.0, gamma, 1000.0, u_lid, dtype, 1e-7, 5_000_000)


def deep_cavity_128_as_stated(gamma: float = 0.1, dtype: str = "f32") -> Cavity:
    """The same cavity with U = 0.05 (unstable at gamma = 0.1)."""
    return Cavity(128, 128, 2.0, gamma, 1000.0, 0.05, dtype, 1e-7, 5_000_000)


def shallow_cavity_8192x2048(dtype: str = "f32") -> Cavity:
    """8192 x 2048 nodes, r = 0.5 (H/L = 0.125), gamma = 0.25, Re = 5000,
    U = 0.05, fixed 2000 steps."""
    return Cavity(8192, 2048, 0.5, 0.25, 5000.0, 0.05, dtype, 0.0, 2000)


def batched_sweep(seed: int = 0, n: int = 256, dtype: str = "f32"):
    """n independent cavities: nx ~ U{64..1024}, ny ~ U{32..512},
    r in {0.25, 0.5, 1, 2}, gamma log-uniform [0.05, 1], Re log-uniform
    [100, 5000], Ma = min(0.1, gamma / 2) (lid speed capped at 0.05),
    residual 1e-7."""
    g = rng(seed)
    out = []
    for _ in range(n):
        nx = int(g.integers(64, 1025))
        ny = int(g.integers(32, 513))
        r = float(g.choice([0.25, 0.5, 1.0, 2.0]))
        gamma = float(math.exp(g.uniform(math.log(0.05), 0.0)))
        re = float(math.exp(g.uniform(math.log(100.0), math.log(5000.0))))
        out.append(Cavity(nx, ny, r, gamma, re, lid_speed_for_mach(r, sweep_mach(gamma)), dtype, 1e-7, 2_000_000))
    return out


@dataclass
class Request:
    arrival_s: float
    cavity: Cavity


def serving_requests(seed: int = 0, n: int = 256, rate_hz: float = 50.0, dtype: str = "f16", scale: int = 1):
    """Poisson arrivals (mean rate_hz) of steady-state cavity solves:
    nx ~ U{128..2048}, ny ~ U{64..1024}, r ~ U[0.25, 2], gamma log-uniform
    [0.05, 1], Re log-uniform [100, 1000], Ma = min(0.1, gamma / 2) (cap
    0.05), residual 1e-6. `scale` divides both grid dimensions (the same
    draws, a smaller mix)."""
    g = rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(g.exponential(1.0 / rate_hz))
        nx = max(3, int(g.integers(128, 2049)) // scale)
        ny = max(3, int(g.integers(64, 1025)) // scale)
        r = float(g.uniform(0.25, 2.0))
        gamma = float(math.exp(g.uniform(math.log(0.05), 0.0)))
        re = float(math.exp(g.uniform(math.log(100.0), math.log(1000.0))))
        out.append(Request(t, Cavity(nx, ny, r, gamma, re, lid_speed_for_mach(r, sweep_mach(gamma)), dtype, 1e-6,
                                     2_000_000)))
    return out
