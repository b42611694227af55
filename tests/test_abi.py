"""C-ABI checks that need no GPU: the library builds, loads, exports every
entry point declared in include/prc_lbm.h, and its host-side parameter logic
follows the paper's parameter relations."""
import math
import os
import re

import pytest

from paper_2208_03562_gb300 import lbm as L

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "prc_lbm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("lbm_create", "lbm_step", "lbm_residual", "lbm_fields", "lbm_run", "lbm_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = L.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def _p(**kw):
    base = dict(nx=64, ny=64, r=1.0, gamma=1.0, nu=0.064, u_lid=0.1, dtype=L.F64)
    extra = {k: kw.pop(k) for k in list(kw) if k not in base}
    base.update(kw)
    p = L.lbm_params_init(base["nx"], base["ny"], base["r"], base["gamma"], base["nu"], base["u_lid"],
                          base["dtype"])
    for k, v in extra.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw", [dict(nx=2), dict(ny=0), dict(r=0.0), dict(r=-1.0), dict(gamma=0.0),
                                dict(gamma=1.5), dict(nu=0.0), dict(nu=-1.0), dict(dtype=7),
                                dict(u_lid=0.6), dict(r=0.25, u_lid=0.15), dict(omega_xi=2.0),
                                dict(omega_xi=0.0), dict(bc=3), dict(drho=2), dict(fx=float('nan'))])
def test_invalid_parameters_rejected(kw):
    p = _p(**kw)
    with pytest.raises(L.LbmError) as e:
        L.lbm_params_check(p)
    assert e.value.status == L.EINVAL


def test_omega_nu_mapping():
    """nu = gamma q^2 c_s*^2 (1/omega_nu - 1/2), q = min(1, r), c_s*^2 = 1/3."""
    for r in (0.25, 0.5, 1.0, 2.0):
        for gamma in (0.05, 0.3, 1.0):
            nu = 0.01
            p = _p(r=r, gamma=gamma, nu=nu, u_lid=0.01)
            w = L.lbm_omega_nu(p)
            q = min(1.0, r)
            assert math.isclose(gamma * q * q / 3 * (1 / w - 0.5), nu, rel_tol=1e-14)


def test_workspace_bytes_grow_with_precision():
    sizes = [L.lbm_workspace_bytes(_p(nx=8192, ny=2048, r=0.5, gamma=0.25, nu=0.01024, u_lid=0.05, dtype=d))
             for d in (L.F16, L.F32, L.F64)]
    assert sizes[0] < sizes[1] < sizes[2]
    # two population sets dominate: 2 * 9 * N * elem
    n = 8192 * 2048
    assert sizes[1] >= 2 * 9 * n * 4 and sizes[1] < 2 * 9 * n * 4 * 1.2


def test_create_without_driver_fails_loudly():
    """On a machine without a usable GPU the library reports an error; it
    never falls back to a CPU path."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("GPU present")
    except ImportError:
        pass
    with pytest.raises(L.LbmError) as e:
        L.lbm_create_p(_p())
    assert e.value.status == L.ECUDA
