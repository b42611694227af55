"""Step-count, stability and grid-saving studies on the paper's cavity shapes.

The paper's Sec. 5.2-5.3 experiments are lid-driven cavities of geometric
aspect ratio AR = H/L on rectangular lattices (r = dy/dx). Each is run at a
Mach number Ma and several preconditioning levels gamma. This module runs
them on the GPU library and reports:

- steps and wall time to a residual ||u_x(t+20) - u_x(t)||_2 (Sec. 5.2), per
  gamma, and the reduction against gamma = 1. The paper quotes about x25 for
  the shallow cavity at Ma = 0.06 and about x51 at Ma = 0.01 (Sec. 5.2); these
  are kept for context;
- the largest Reynolds number that stays stable for a given gamma (Sec. 5.3),
  by bisection over Re;
- the rectangular-versus-square grid comparison of Sec. 5.2: the same shallow
  cavity on 100 x 125 nodes with r = 0.2 and on 400 x 100 nodes with r = 1.
  It reports the centre-line profiles, their difference and the time to
  solution of each.

Every solve is an independent ``lbm.Lbm`` handle on its own CUDA stream. These
grids are small enough for the cluster-resident engine, which is the handle's
default. Solves run concurrently from a thread pool: the library releases the
GIL, and one solve occupies one thread-block cluster. Lid speed, viscosity and
grid follow the paper's definitions:
- Ma = U / (q c_s*) with q = min(1, r) (Eqs. 1-2);
- Re = U H / nu with H = ny r (Sec. 5);
- cavity walls with the lid on top (Sec. 5.1).
"""
from __future__ import annotations

import concurrent.futures as cf
import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

CS_STAR = 1.0 / math.sqrt(3.0)


@dataclass
class Experiment:
    name: str
    where: str            # section of the paper
    ar: float             # H / L
    r: float              # dy / dx
    nx: int
    ny: int
    re: float
    mach: float
    gammas: Sequence[float]
    paper_steps: Dict[float, float] = field(default_factory=dict)  # context only (gamma -> steps)
    paper_ratio: Optional[float] = None                             # context only

    @property
    def u_lid(self) -> float:
        return self.mach * min(1.0, self.r) * CS_STAR

    @property
    def nu(self) -> float:
        return self.u_lid * self.ny * self.r / self.re


# The convergence-history experiments of Sec. 5.2 (grid, r, Re, Ma, gamma as printed).
PAPER_EXPERIMENTS = [
    Experiment("shallow_Ma0.06", "Sec. 5.2, convergence, shallow cavity", 0.25, 0.2, 100, 125, 100.0, 0.06,
               (1.0, 0.5, 0.1, 0.08), {1.0: 610_000, 0.08: 24_000}, 25.0),
    Experiment("shallow_Ma0.01", "Sec. 5.2, convergence, shallow cavity", 0.25, 0.2, 100, 125, 100.0, 0.01,
               (1.0, 0.5, 0.1, 0.05), {1.0: 5_000_000, 0.05: 97_000}, 51.0),
    Experiment("deep_Re100_Ma0.06", "Sec. 5.2, convergence, deep cavity", 2.0, 1.6, 100, 125, 100.0, 0.06,
               (1.0, 0.5, 0.1, 0.08), {}, 14.0),
    Experiment("deep_Re100_Ma0.02", "Sec. 5.2, convergence, deep cavity", 2.0, 1.6, 100, 125, 100.0, 0.02,
               (1.0, 0.5, 0.1, 0.05), {}, 23.0),
    Experiment("deep_Re1000_Ma0.06", "Sec. 5.2, convergence, deep cavity at Re = 1000 (figure caption grid)",
               2.0, 4.0 / 3.0, 100, 150, 1000.0, 0.06, (1.0, 0.75, 0.5, 0.1),
               {1.0: 11_154_000, 0.1: 583_000}, 19.0),
]


def _lib():
    from . import lbm as L
    L.load()
    return L


def solve(nx, ny, r, gamma, nu, u_lid, tol, max_steps, dtype="f32", want_fields=False, time_limit_s=None,
          model=0):
    """One steady-state solve from rest; returns a result dict. model 0 is
    the central-moment scheme (PRC-LBM), 1 the raw-moment one (PRNR-LBM)."""
    L = _lib()
    p = L.lbm_params_init(nx, ny, r, gamma, nu, u_lid, L.DTYPE_CODES[dtype], model=model)
    h = L.Lbm(p)
    t0 = time.perf_counter()
    steps, status = 0, None
    chunk = 200_000
    try:
        while steps < max_steps:
            st, n = h.run(tol, min(chunk, max_steps - steps))
            steps += n
            status = st
            if st == L.OK or (time_limit_s is not None and time.perf_counter() - t0 > time_limit_s):
                break
    except L.LbmError as e:
        status = e.status
    wall = time.perf_counter() - t0
    out = {"gamma": gamma, "model": model, "steps": steps, "wall_s": wall, "variant": h.variant,
           "status": {L.OK: "converged", L.EDIVERGED: "diverged"}.get(status, "not converged"),
           "residual": h.info().residual}
    if want_fields and out["status"] != "diverged":
        out["fields"] = h.fields()
    h.close()
    return out


def convergence_study(exp: Experiment, tol: float = 1e-6, max_steps: int = 20_000_000, dtype: str = "f32",
                      workers: int = 8, want_fields: bool = False, time_limit_s: float = None,
                      model: int = 0) -> dict:
    """Steps to `tol` for every gamma of an experiment, solved concurrently."""
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {g: ex.submit(solve, exp.nx, exp.ny, exp.r, g, exp.nu, exp.u_lid, tol, max_steps, dtype,
                             want_fields, time_limit_s, model) for g in exp.gammas}
        runs = {g: f.result() for g, f in futs.items()}
    base = runs.get(1.0)
    for g, r in runs.items():
        if base and base["status"] == "converged" and r["status"] == "converged":
            r["step_reduction_vs_gamma1"] = base["steps"] / r["steps"]
    return {"experiment": exp.name, "model": model, "where": exp.where, "nx": exp.nx, "ny": exp.ny, "r": exp.r, "re": exp.re,
            "mach": exp.mach, "u_lid": exp.u_lid, "nu": exp.nu, "tol": tol, "dtype": dtype,
            "runs": [runs[g] for g in exp.gammas],
            "paper_context": {"steps": exp.paper_steps, "reduction": exp.paper_ratio}}


def max_stable_re(nx, ny, r, gamma, u_lid, re_lo=50.0, re_hi=1e5, steps=200_000, iters=8, dtype="f32",
                  tol=1e-9, model=0) -> dict:
    """Largest Re (bisection in log Re) for which a run from rest stays finite
    for `steps` steps (or converges before), Sec. 5.3."""
    def stable(re):
        nu = u_lid * ny * r / re
        # the shear rate must stay in (0, 2) for the run to be defined at all
        q = min(1.0, r)
        w = 1.0 / (nu / (gamma * q * q / 3.0) + 0.5)
        if not (0.0 < w < 2.0):
            return False
        return solve(nx, ny, r, gamma, nu, u_lid, tol, steps, dtype, model=model)["status"] != "diverged"
    lo, hi = re_lo, re_hi
    if not stable(lo):
        return {"gamma": gamma, "model": model, "max_stable_re": None, "note": "unstable at the lower bracket"}
    if stable(hi):
        return {"gamma": gamma, "model": model, "max_stable_re": hi, "note": "stable at the upper bracket"}
    for _ in range(iters):
        mid = math.sqrt(lo * hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return {"gamma": gamma, "model": model, "max_stable_re": lo, "bracket": [lo, hi], "steps": steps}


def stability_study(gammas=(1.0, 0.5, 0.2), nx=100, ny=100, r=0.25, u_lid=0.02, steps=200_000, workers=6,
                    dtype="f32", models=(0, 1)) -> dict:
    """Sec. 5.3: AR = 0.25 cavity, r = 0.25, U = 0.02; max stable Re per
    gamma, for the central-moment (0) and raw-moment (1) schemes."""
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(max_stable_re, nx, ny, r, g, u_lid, steps=steps, dtype=dtype, model=m)
                for m in models for g in gammas]
        res = [f.result() for f in futs]
    return {"where": "Sec. 5.3, stability", "nx": nx, "ny": ny, "r": r, "u_lid": u_lid, "steps": steps,
            "runs": res}


def centreline_profiles(fields, nx, ny, r):
    """u along the vertical centre line and v along the horizontal one, with
    their coordinates normalised by L = nx and H = ny r (node centres)."""
    import numpy as np
    _, ux, uy = fields
    ys = (np.arange(ny) + 0.5) / ny
    xs = (np.arange(nx) + 0.5) / nx
    if nx % 2:
        u_c = ux[:, nx // 2]
    else:
        u_c = 0.5 * (ux[:, nx // 2 - 1] + ux[:, nx // 2])
    if ny % 2:
        v_c = uy[ny // 2, :]
    else:
        v_c = 0.5 * (uy[ny // 2 - 1, :] + uy[ny // 2, :])
    return ys, u_c, xs, v_c


def grid_saving_study(re=100.0, mach=0.06, gamma=1.0, tol=1e-7, dtype="f32", max_steps=20_000_000) -> dict:
    """Sec. 5.2: shallow cavity AR = 0.25, rectangular 100 x 125 (r = 0.2)
    against square 400 x 100 (r = 1), same Re and Ma. Profiles are compared
    on the rectangular grid's centre-line points (linear interpolation of
    the square-grid profile), normalised by the lid speed."""
    import numpy as np
    cases = {"rect_r0.2_100x125": (100, 125, 0.2), "square_r1_400x100": (400, 100, 1.0)}
    out = {}
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        futs = {}
        for name, (nx, ny, r) in cases.items():
            u = mach * min(1.0, r) * CS_STAR
            nu = u * ny * r / re
            futs[name] = (ex.submit(solve, nx, ny, r, gamma, nu, u, tol, max_steps, dtype, True), u)
        for name, (f, u) in futs.items():
            out[name] = dict(f.result(), u_lid=u)
    prof = {}
    for name, (nx, ny, r) in cases.items():
        ys, u_c, xs, v_c = centreline_profiles(out[name].pop("fields"), nx, ny, r)
        prof[name] = (ys, u_c / out[name]["u_lid"], xs, v_c / out[name]["u_lid"])
    a, b = prof["rect_r0.2_100x125"], prof["square_r1_400x100"]
    du = np.max(np.abs(a[1] - np.interp(a[0], b[0], b[1])))
    dv = np.max(np.abs(a[3] - np.interp(a[2], b[2], b[3])))
    return {"where": "Sec. 5.2, rectangular vs square lattice", "re": re, "mach": mach, "gamma": gamma, "tol": tol,
            "runs": out, "nodes": {k: v[0] * v[1] for k, v in cases.items()},
            "max_abs_diff_u_centreline_over_U": float(du), "max_abs_diff_v_centreline_over_U": float(dv)}
