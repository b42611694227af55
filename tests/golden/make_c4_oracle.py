"""Writes c4_oracle.json: FP64 oracle results on the batched-sweep workload
(256 uneven lid-driven cavities, seed 0; nx 64..1024, ny 32..512, r in
{0.25, 0.5, 1, 2}, gamma log-uniform 0.05..1, Re log-uniform 100..5000), the
stand-in for the paper's parameter sweeps over gamma, r and Re (Sec. 5.2-5.3).

Calls only the oracle (oracle/stepper.py) and the seeded input generators.
For every cavity, from rest, 1000 steps in blocks of 20 with the Sec. 5.2
residual after each block (a non-finite residual ends the run: diverged);
for the eight smallest cavities, also the run to the residual 1e-7 (the
sweep's tolerance) or divergence.  Each cavity also runs from a rest state
perturbed by relative noise of 1e-7 per population (the rounding level of
FP32 storage; inputs.noise(8000 + i, ...)); the relative L2 distance of its
velocity from the unperturbed run at step 1000 is the oracle's own
sensitivity to perturbations of that size ("sensitivity"; infinite when
either run diverged).  A cavity whose flow is unstable or chaotic amplifies
such perturbations, so its step-1000 state is not fixed to the FP32 parity
bar by the parameters alone.  Each record keeps the status, the steps,
the residual, ||u_x||_2, ||u_y||_2 and the total mass, (u_x, u_y) at 16
sampled nodes (inputs.sample_nodes(9000 + i, ...)) and 8 random projections
of (u_x, u_y) (inputs.projection_signs(7000 + i, ...)), from which a test
estimates the L2 distance of another field to the oracle's without holding
it.

  python tests/golden/make_c4_oracle.py [--workers N]

Takes about three quarters of an hour on 8 host cores (one oracle thread per
cavity, cavities in parallel).
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_oracle.json")
N_SAMPLES, N_PROJ = 16, 8
STEPS = 1000
TOL = 1e-7
MAX_STEPS = 2_000_000


def _g(v):
    return float("%.13e" % v)


def _record(o, i, cav, status, steps, res):
    import numpy as np
    from paper_2208_03562_gb300 import inputs as I
    rho, ux, uy = o.fields()
    rec = {"status": status, "steps": int(steps), "residual": _g(res) if math.isfinite(res) else str(res)}
    if status == "diverged":
        return rec
    idx = I.sample_nodes(9000 + i, N_SAMPLES, cav.nx, cav.ny)
    w = I.projection_signs(7000 + i, N_PROJ, cav.nx, cav.ny)
    rec.update({
        "norm_ux": _g(math.sqrt(math.fsum((ux * ux).ravel()))),
        "norm_uy": _g(math.sqrt(math.fsum((uy * uy).ravel()))),
        "mass": _g(o.total_mass()),
        "ux": [_g(v) for v in ux.ravel()[idx]],
        "uy": [_g(v) for v in uy.ravel()[idx]],
        "proj": [_g(math.fsum((w[k, 0] * ux).ravel()) + math.fsum((w[k, 1] * uy).ravel())) for k in range(N_PROJ)],
    })
    return rec


PERTURB = 1e-7


def job(args):
    i, kind = args
    from oracle import stepper as S
    from paper_2208_03562_gb300 import inputs as I
    S.num_threads(1)
    cav = I.batched_sweep(seed=0, n=256)[i]
    par = S.OracleParams(nx=cav.nx, ny=cav.ny, r=cav.r, gamma=cav.gamma, nu=cav.nu, u_lid=cav.u_lid)
    o = S.Oracle(par)
    t = time.perf_counter()
    if kind == "step1000":
        steps, res = o.run(0.0, STEPS)
        status = "diverged" if not math.isfinite(res) else "finite"
        # the same run from a perturbed rest state
        p = S.Oracle(par)
        w = S.rest_weights(par)
        p.set_populations(w[:, None, None] * (1.0 + I.noise(8000 + i, (9, cav.ny, cav.nx), PERTURB)))
        _, res_p = p.run(0.0, STEPS)
        if status == "finite" and math.isfinite(res_p):
            _, ux, uy = o.fields()
            _, px, py = p.fields()
            num = math.fsum(((px - ux) ** 2 + (py - uy) ** 2).ravel())
            den = math.fsum((ux * ux + uy * uy).ravel())
            sens = math.sqrt(num / den)
        else:
            sens = math.inf
    else:
        steps, res = o.run(TOL, MAX_STEPS)
        status = "diverged" if not math.isfinite(res) else ("converged" if res < TOL else "maxsteps")
    rec = _record(o, i, cav, status, steps, res)
    if kind == "step1000":
        rec["sensitivity"] = _g(sens) if math.isfinite(sens) else "inf"
    rec["oracle_s"] = round(time.perf_counter() - t, 1)
    return i, kind, rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=len(os.sched_getaffinity(0)))
    a = ap.parse_args()
    from paper_2208_03562_gb300 import inputs as I
    mix = I.batched_sweep(seed=0, n=256)
    smallest = sorted(range(len(mix)), key=lambda i: (mix[i].nodes, i))[:8]
    jobs = [(i, "converge") for i in smallest] + \
        sorted([(i, "step1000") for i in range(len(mix))], key=lambda j: -mix[j[0]].nodes)
    out = {"source": __doc__.strip().splitlines()[0],
           "workload": "inputs.batched_sweep(seed=0, n=256), FP64 oracle from rest",
           "n_samples": N_SAMPLES, "n_proj": N_PROJ, "steps": STEPS, "tol": TOL, "max_steps": MAX_STEPS,
           "perturbation": PERTURB,
           "step1000": {}, "converge": {}}
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(a.workers) as pool:
        for n, (i, kind, rec) in enumerate(pool.imap_unordered(job, jobs)):
            out[kind][str(i)] = rec
            if n % 16 == 0:
                print("%d/%d done, %.0f s" % (n + 1, len(jobs), time.perf_counter() - t0), flush=True)
    for kind in ("step1000", "converge"):
        out[kind] = {k: out[kind][k] for k in sorted(out[kind], key=int)}
    with open(OUT, "w") as fh:
        fh.write("{\n")
        keys = list(out)
        for n, k in enumerate(keys):
            if isinstance(out[k], dict) and k in ("step1000", "converge"):
                fh.write(' "%s": {\n' % k)
                items = list(out[k].items())
                for m, (kk, v) in enumerate(items):
                    fh.write('  "%s": %s%s\n' % (kk, json.dumps(v), "," if m + 1 < len(items) else ""))
                fh.write(" }%s\n" % ("," if n + 1 < len(keys) else ""))
            else:
                fh.write(' "%s": %s%s\n' % (k, json.dumps(out[k]), "," if n + 1 < len(keys) else ""))
        fh.write("}\n")
    print("wrote %s in %.0f s" % (OUT, time.perf_counter() - t0))


if __name__ == "__main__":
    main()
