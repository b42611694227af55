"""Writes study_oracle.json: FP64 oracle runs of the studies built on the hot
path, the stand-ins for the convergence and grid-saving experiments of
Sec. 5.2 of arXiv:2208.03562 (lid-driven cavities, lid on top, from rest):

* the shallow cavity of the convergence study, AR = 0.25 on 100 x 125 nodes,
  r = 0.2, Re = 100, Ma = 0.06, at gamma = 1 and gamma = 0.1, each to the
  residual 1e-8 (Sec. 5.2 residual, blocks of 20 steps);
* the grid-saving comparison, the same cavity on the rectangular 100 x 125
  grid (r = 0.2) and on the square 400 x 100 grid (r = 1), gamma = 1, each to
  the residual 1e-7.

Calls only the oracle (oracle/stepper.py).  Each record keeps the steps, the
residual, ||u_x||_2, ||u_y||_2, 8 random projections of (u_x, u_y)
(inputs.projection_signs(6000 + k, ...)) and the centre-line profiles that
the study compares (u on the vertical centre line, v on the horizontal one,
the mean of the two middle lines for an even count).

  python tests/golden/make_study_oracle.py

About ten minutes on four host cores (one oracle thread per run).
"""
import json
import math
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "study_oracle.json")
N_PROJ = 8
CS_STAR = 1.0 / math.sqrt(3.0)


def cavity(nx, ny, r, re, mach):
    u = mach * min(1.0, r) * CS_STAR          # Ma = U / (q c_s*), q = min(1, r)
    return dict(nx=nx, ny=ny, r=r, u_lid=u, nu=u * ny * r / re)  # Re = U H / nu, H = ny r


# name -> (cavity, gamma, residual, projection seed)
RUNS = {
    "shallow_gamma1": (cavity(100, 125, 0.2, 100.0, 0.06), 1.0, 1e-8, 6001),
    "shallow_gamma0.1": (cavity(100, 125, 0.2, 100.0, 0.06), 0.1, 1e-8, 6002),
    "rect_r0.2_100x125": (cavity(100, 125, 0.2, 100.0, 0.06), 1.0, 1e-7, 6003),
    "square_r1_400x100": (cavity(400, 100, 1.0, 100.0, 0.06), 1.0, 1e-7, 6004),
}


def _g(v):
    return float("%.15e" % v)


def centre(a, axis):
    """The middle line of a 2-D array along an axis (mean of the two middle
    ones for an even count)."""
    n = a.shape[axis]
    take = (lambda k: a[:, k]) if axis == 1 else (lambda k: a[k, :])
    return take(n // 2) if n % 2 else 0.5 * (take(n // 2 - 1) + take(n // 2))


def job(name):
    import numpy as np
    from oracle import stepper as S
    from paper_2208_03562_gb300 import inputs as I
    cav, gamma, tol, seed = RUNS[name]
    S.num_threads(1)
    o = S.Oracle(S.OracleParams(nx=cav["nx"], ny=cav["ny"], r=cav["r"], gamma=gamma, nu=cav["nu"],
                                u_lid=cav["u_lid"]))
    t = time.perf_counter()
    steps, res = o.run(tol, 5_000_000)
    _, ux, uy = o.fields()
    w = I.projection_signs(seed, N_PROJ, cav["nx"], cav["ny"])
    rec = dict(cav, gamma=gamma, tol=tol, status="converged" if res < tol else "not converged", steps=int(steps),
               residual=_g(res), norm_ux=_g(math.sqrt(math.fsum((ux * ux).ravel()))),
               norm_uy=_g(math.sqrt(math.fsum((uy * uy).ravel()))),
               proj=[_g(math.fsum((w[k, 0] * ux).ravel()) + math.fsum((w[k, 1] * uy).ravel()))
                     for k in range(N_PROJ)], proj_seed=seed,
               u_centre=[_g(v) for v in centre(ux, 1)], v_centre=[_g(v) for v in centre(uy, 0)],
               oracle_s=round(time.perf_counter() - t, 1))
    return name, rec


def main():
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(len(RUNS)) as pool:
        recs = dict(pool.map(job, list(RUNS)))
    out = {"source": __doc__.strip().splitlines()[0], "n_proj": N_PROJ, "runs": recs}
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote %s in %.0f s" % (OUT, time.perf_counter() - t0))


if __name__ == "__main__":
    main()
