"""The collision arithmetic of the CUDA path against the oracle, on the CPU.

``csrc/prc_device.cuh`` writes the collision once for double, float and
packed FP32x2, with the algebra of App. A rearranged:
- the strain-rate system of Eqs. 43-44 solved for rho (X + Y) and rho (X - Y);
- relaxation and corrections folded;
- deviation form.

The header compiles for the host as well, so nvcc builds
``tests/host_collide.cu``, which runs the header's ``collide<double>`` with
the library's own coefficient set-up, into a host shared library.  Its FP64
post-collision populations must equal those of the oracle's matrix form
(Eq. 10-equivalent-centralmoment; Eq. 10-equivalent for the raw-moment scheme)
to round-off (a bound that grows like 1 / gamma^2, as the gamma-scaled
coefficients do).  This covers random states, densities, velocities, density
gradients and forces, r in {0.25, 0.5, 1, 1.6, 2} and gamma in
{0.05, 0.1, 0.5, 1}.  The rest weights are compared too.

The FP64 GPU parity tests compare the same code on the device.  This one
needs no GPU and pins the algebra itself.  It is skipped without nvcc.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import matrix_form as MF
from oracle import stepper as S
from paper_2208_03562_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

R_SET = [0.25, 0.5, 1.0, 1.6, 2.0]
GAMMA_SET = [0.05, 0.1, 0.5, 1.0]


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if not nvcc:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("host_collide") / "libhost_collide.so")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "--expt-relaxed-constexpr",
           "-shared", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2208_03562_gb300", "csrc"), os.path.join(HERE, "host_collide.cu"),
           "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    h = C.CDLL(out)
    D = C.POINTER(C.c_double)
    h.host_collide.argtypes = [C.c_double] * 6 + [C.c_int, C.c_int, D, C.c_double, C.c_double, D, D, D]
    h.host_collide.restype = C.c_int
    return h


def host_collide(lib, p, model, drho, g, dx, dy):
    ptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    g = np.ascontiguousarray(g, dtype=np.float64)
    out, w, diag = np.empty(9), np.empty(9), np.empty(3)
    lib.host_collide(p.r, p.gamma, p.nu, p.omega_xi, p.fx, p.fy, 1 if drho else 0, model, ptr(g), dx, dy,
                     ptr(out), ptr(w), ptr(diag))
    return out, w, diag


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("gamma", GAMMA_SET)
@pytest.mark.parametrize("r", R_SET)
def test_device_collision_equals_matrix_form(lib, r, gamma, model):
    g = I.rng(5000 + int(100 * r) + int(1000 * gamma) + 7 * model)
    oracle_collide = MF.collide_raw if model == 1 else MF.collide
    for k in range(48):
        drho, force = k % 2 == 0, k % 3 == 0
        p = S.OracleParams(nx=1, ny=1, r=r, gamma=gamma, nu=g.uniform(1e-3, 0.1), omega_xi=g.uniform(0.5, 1.8),
                           fx=1e-4 * g.standard_normal() if force else 0.0,
                           fy=1e-4 * g.standard_normal() if force else 0.0)
        rho = g.uniform(0.95, 1.05)
        ux, uy = 0.03 * g.standard_normal(2)
        f = S.equilibrium(p, rho, ux, uy) + 1e-3 * g.standard_normal(9)
        dx, dy = (1e-3 * g.standard_normal(2)) if drho else (0.0, 0.0)
        w = S.rest_weights(p)
        gt, w_lib, diag = host_collide(lib, p, model, drho, f - w, dx, dy)
        # the same rest weights up to the rounding order of their sums: two
        # units in the last place of a weight below 1
        assert np.max(np.abs(w_lib - w)) <= 2.3e-16
        ft, (rho_o, ux_o, uy_o, _, _) = oracle_collide(f, r, gamma, S.omega_nu(p), dx, dy, p.fx, p.fy,
                                                     omega_3=p.omega_xi)
        # P_gamma and Q_gamma grow like 4 / gamma^2 and the round-off of both
        # forms with them: measured worst cases are 1e-15 .. 6e-15 / gamma^2
        scale = np.max(np.abs(ft))
        assert np.max(np.abs((gt + w) - ft)) <= 5e-14 / gamma ** 2 * scale, (k, drho, force)
        assert abs(diag[0] - ux_o) <= 1e-14 and abs(diag[1] - uy_o) <= 1e-14
        assert abs(diag[2] - (rho_o - 1.0)) <= 1e-14


def test_a_planted_slip_in_the_algebra_is_caught(lib):
    """The comparison has teeth: the oracle with its corrections switched off
    (the kind of term a rearrangement could drop) differs from the library's
    collision far beyond the tolerance above."""
    g = I.rng(77)
    p = S.OracleParams(nx=1, ny=1, r=2.0, gamma=0.1, nu=0.01)
    f = S.equilibrium(p, 1.0, 0.04, -0.02) + 1e-3 * g.standard_normal(9)
    dx, dy = 1e-3, -2e-3
    gt, _, _ = host_collide(lib, p, 0, True, f - S.rest_weights(p), dx, dy)
    ft, _ = MF.collide(f, 2.0, 0.1, S.omega_nu(p), dx, dy, corrections=False)
    assert np.max(np.abs((gt + S.rest_weights(p)) - ft)) > 1e-8


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("gamma", [0.1, 0.5, 1.0])
@pytest.mark.parametrize("r", [0.5, 1.0, 2.0])
def test_packed_lanes_equal_scalar_float_and_fp64(lib, r, gamma, model):
    """The FP32 / FP16 kernels collide two neighbouring nodes as the two lanes
    of one packed FP32x2 value.  Two different nodes packed together must come
    out lane for lane exactly as the float collision of each node alone (no
    lane mixing, same operations), and within FP32 round-off of the FP64
    collision."""
    D, F = C.POINTER(C.c_double), C.POINTER(C.c_float)
    lib.host_collide_f32_pair.argtypes = [C.c_double] * 4 + [C.c_int, D, D, D, F, F]
    g = I.rng(6000 + int(100 * r) + int(1000 * gamma) + 7 * model)
    p = S.OracleParams(nx=1, ny=1, r=r, gamma=gamma, nu=0.01, omega_xi=1.0)
    w = S.rest_weights(p)
    for _ in range(24):
        nodes = []
        for _n in range(2):
            rho = g.uniform(0.97, 1.03)
            ux, uy = 0.03 * g.standard_normal(2)
            nodes.append(S.equilibrium(p, rho, ux, uy) + 1e-4 * g.standard_normal(9) - w)
        gab = np.ascontiguousarray(np.concatenate(nodes))
        dx, dy = 1e-3 * g.standard_normal(2), 1e-3 * g.standard_normal(2)
        pair, single = np.empty(18, np.float32), np.empty(18, np.float32)
        ptr = lambda a, t: a.ctypes.data_as(t)
        lib.host_collide_f32_pair(r, gamma, p.nu, p.omega_xi, model, ptr(gab, D), ptr(dx, D), ptr(dy, D),
                                  ptr(pair, F), ptr(single, F))
        assert np.array_equal(pair, single)
        for n in range(2):
            g64, _, _ = host_collide(lib, p, model, True, gab[9 * n:9 * n + 9], dx[n], dy[n])
            scale = np.max(np.abs(g64 + w))
            # measured worst cases: 1.3e-8 (gamma = 1) .. 5.1e-7 (gamma = 0.1) relative
            assert np.max(np.abs(pair[9 * n:9 * n + 9] - g64)) <= 2e-7 / gamma ** 2 * scale
