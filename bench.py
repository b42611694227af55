#!/usr/bin/env python
"""Throughput of the fused PRC-LBM step (arXiv:2208.03562) on GB300.

Workload: shallow shear-driven cavity, H/L = 0.125, 8192 x 2048 nodes, r = 0.5,
gamma = 0.25, Re = 5000, u_lid = 0.05, started from rest; one bench step = one
time step of the whole hot path (pull-stream + walls, collision with the
preconditioned corrections and local strain rates, store; every 20th step the
FP64 residual and mass reduction).  Primary line: FP32 shifted storage; FP16
shifted storage is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank runs its own replica (weak scaling, no collective on the
data path); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & time-to-steady-state (FP32/FP16 vs FP64 plain), % of HBM roofline"
FALLBACK_HBM_GBS = 6800.0
BYTES_PER_NODE = {"f64": 144, "f32": 72, "f16": 36}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip every leg but the primary one")
    ap.add_argument("--skip", default="", help="comma-separated legs to skip: time_to_steady_state, "
                                               "batched_sweep, serving")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16", "f64"], help="storage of the primary leg")
    ap.add_argument("--variant", type=int, default=None,
                    help="profiling only: use this interior-kernel variant instead of autotuning")
    ap.add_argument("--nx", type=int, default=0, help="profiling only: override the grid width")
    ap.add_argument("--ny", type=int, default=0, help="profiling only: override the grid height")
    ap.add_argument("--profile-case", default="", choices=["", "batch", "cluster"],
                    help="profiling only: run one small fixed case of the batch engine or the cluster engine "
                         "(for an ncu capture of k_batch / k_cluster) and exit")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
            return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# The sources the step kernel k_step_tma is compiled from (its body, the
# collision, the edge-strip tile body, the reductions, the arithmetic types)
# and the variant lists: a DRAM-traffic figure stays valid while these are
# unchanged, whatever else in the library changes.
STEP_KERNEL_SOURCES = ("prc_tma.cuh", "prc_kernels.cuh", "prc_device.cuh", "prc_reduce.cuh", "prc_vec.cuh",
                       "ops_f32.cu", "ops_f16.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    for name in STEP_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2208_03562_gb300", "csrc", name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """DRAM bytes per launch of the kernel from the committed ncu summary,
    only if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d[kernel_key]
        if e.get("csrc_sha") == kernel_source_hash():
            return float(e["bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


GRID_OVERRIDE = {}
FORCE_VARIANT = {}


def workload(dtype):
    from paper_2208_03562_gb300 import inputs as I
    cav = I.shallow_cavity_8192x2048(dtype)
    if GRID_OVERRIDE:
        cav.nx = GRID_OVERRIDE.get("nx") or cav.nx
        cav.ny = GRID_OVERRIDE.get("ny") or cav.ny
    return cav


def config_of(cav):
    return {"workload": "shallow lid-driven cavity 8192x2048, H/L=0.125, r=0.5, gamma=0.25, Re=5000, "
                        "u_lid=0.05, from rest",
            "nx": cav.nx, "ny": cav.ny, "r": cav.r, "gamma": cav.gamma, "Re": cav.re, "u_lid": cav.u_lid,
            "storage": "shifted f_i - w_i rho0, A/B planes", "residual_every": 20,
            "l2": "inputs larger than L2: every step streams both population sets (>129 MB)"}


# ---------------------------------------------------------------------------

def gpu_leg(cav_dtype, steps, warmup, torch, L, dist=None, clocks_index=None):
    cav = workload(cav_dtype)
    p = L.lbm_params_init(cav.nx, cav.ny, cav.r, cav.gamma, cav.nu, cav.u_lid, L.DTYPE_CODES[cav_dtype])
    g = L.Lbm(p, torch_workspace=True)
    from paper_2208_03562_gb300 import autotune
    if FORCE_VARIANT and cav_dtype in FORCE_VARIANT:
        g.variant = FORCE_VARIANT[cav_dtype]
        tuned = {"variant": g.variant, "forced": True}
    else:
        tuned = autotune.tune(g, steps=20)
    tuned["shapes"] = [L.lbm_variant_info(p.dtype, i) for i in range(L.lbm_variant_count(p.dtype))]
    stream = torch.cuda.current_stream()
    g.step(warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(clocks_index) if clocks_index is not None else None
    if sampler:
        sampler.__enter__()
        time.sleep(0.4)
    regions = timed_regions(g, steps, stream, torch, dist)
    if sampler:
        sampler.__exit__()
    ms = sorted(regions)[len(regions) // 2]
    info = g.info()
    launch = launch_times(g, min(steps, 200), torch)
    g.close()
    tuned["regions_ms"] = {"n": len(regions), "median": ms, "min": min(regions), "max": max(regions)}
    return cav, ms, info, (sampler.summary() if sampler else None), tuned, launch


def timed_regions(g, steps, stream, torch, dist, min_total_s=0.5, max_regions=200):
    """Time regions of exactly `steps` steps, each bracketed by a barrier (under
    torchrun) and a device synchronisation on both sides and timed with CUDA
    events on the stream the step kernel is launched on, until at least
    min_total_s of device time has been measured (at least three regions).
    Every region is the max over ranks.  The caller reports the median."""
    out, total = [], 0.0
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while len(out) < 3 or (total < min_total_s * 1e3 and len(out) < max_regions):
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0.record(stream)
        g.step(steps)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        if dist:
            ms = max_over_ranks(ms, dist, torch, "cuda")
            dist.barrier()
        out.append(ms)
        total += ms
    return out


def max_over_ranks(value, dist, torch, device):
    """The largest of every rank's `value` (a time), on every rank."""
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def launch_times(g, n, torch):
    """Duration of each step launch, from CUDA events recorded on the stream
    the step kernel is launched on (the handle enqueues on PyTorch's current
    stream), one step per lbm_step call (no graph).  A step is one launch of
    the fused step kernel; every 20th step also launches the residual
    finalisation, so those are reported apart."""
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    t_first = g.info().step
    for a, b in ev:
        a.record(stream)
        g.step(1)
        b.record(stream)
    torch.cuda.synchronize()
    plain, epi = [], []
    for k, (a, b) in enumerate(ev):
        ((epi if (t_first + k + 1) % 20 == 0 else plain)).append(a.elapsed_time(b))
    mean = lambda xs: sum(xs) / len(xs) if xs else None
    return {"launches": n, "ms_step_kernel": mean(plain), "ms_residual_step": mean(epi),
            "n_plain": len(plain), "n_residual": len(epi)}


def kernel_timing(ms_step, isolated):
    """The step kernel's average launch duration inside the timed region:
    the region's event time over its step launches (one launch of the fused
    step kernel per step).  The residual finalisation launched every 20th
    step is included, so this bounds the kernel's duration from above.  The
    isolated per-launch figures (an event pair around each single step,
    outside any graph) ride along for comparison."""
    return {"ms_step_kernel": ms_step, "source": "timed region / step launches",
            "isolated_launches": isolated}


def e2e_leg(steps, torch, L):
    """Same workload through the public C ABI with host buffers: upload the
    initial fields from pinned host memory, run, read the fields back."""
    cav = workload("f32")
    h = L.lbm_create(cav.nx, cav.ny, cav.r, cav.gamma, cav.nu, cav.u_lid, L.F32)
    shape = (cav.ny, cav.nx)
    rho = torch.ones(shape, dtype=torch.float64).pin_memory().numpy()
    ux = torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()
    uy = torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()
    outs = [torch.empty(shape, dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
    import ctypes as C

    def once():
        L._check(L.load().lbm_init_fields(h, *[a.ctypes.data_as(C.c_void_p) for a in (rho, ux, uy)], 0), h)
        L.lbm_step(h, steps)
        L._check(L.load().lbm_fields(h, *[a.ctypes.data_as(C.c_void_p) for a in outs], 0), h)

    once()  # warm (graph build, allocator)
    t = time.perf_counter()
    once()
    dt = time.perf_counter() - t
    L.lbm_destroy(h)
    n = cav.nodes
    return {"value": n * steps / dt / 1e9, "unit": "GLUPS",
            "h2d_bytes_per_step": 3 * 8 * n / steps, "d2h_bytes_per_step": 3 * 8 * n / steps,
            "wall_s": dt, "what": "lbm_init_fields(host, pinned) + lbm_step(%d) + lbm_fields(host, pinned); "
                                  "bytes per step are the per-solve transfers divided by the steps" % steps}


# ---------------------------------------------------------------------------
# time to steady state, with the error of every result against the FP64 oracle

def deep_cavity_100x150(gamma, dtype):
    """The paper's deep cavity at Re = 1000 (Sec. 5.2): AR = 2 on 100 x 150
    nodes, r = 4/3, Ma = 0.06, to residual 1e-6."""
    from paper_2208_03562_gb300 import inputs as I
    return I.Cavity(100, 150, 4.0 / 3.0, gamma, 1000.0, 0.06 * I.CS_STAR, dtype, 1e-6, 5_000_000)


def oracle_solve(job):
    """Runs in a spawned worker process: the FP64 oracle from rest to each
    tolerance of `tols` in turn (blocks of 20 steps, Sec. 5.2 residual).
    Returns {tol: (status, steps, residual, u_x, u_y, seconds)}."""
    from oracle import stepper as S
    cav, tols, max_steps, threads = job
    S.num_threads(threads)
    o = S.Oracle(S.OracleParams(nx=cav["nx"], ny=cav["ny"], r=cav["r"], gamma=cav["gamma"], nu=cav["nu"],
                                u_lid=cav["u_lid"]))
    out, done, t0 = {}, 0, time.perf_counter()
    for tol in tols:
        n, res = o.run(tol, max_steps - done)
        done += n
        _, ux, uy = o.fields()
        st = "converged" if res < tol else ("diverged" if res != res or res == float("inf") else "maxsteps")
        out[tol] = (st, done, res, ux, uy, time.perf_counter() - t0)
        if st != "converged":
            break
    return out


class OracleJobs:
    """FP64 oracle runs on the host cores, in spawned worker processes, while
    the GPU legs run; each GPU result is compared with its oracle result when
    both are in."""

    def __init__(self, jobs, workers=3):
        import concurrent.futures as cf
        import multiprocessing as mp
        cores = len(os.sched_getaffinity(0))
        self.threads = max(1, (cores - 4) // workers)
        self.ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
        self.fut = {}
        for name, cav, tols, max_steps in jobs:
            d = {"nx": cav.nx, "ny": cav.ny, "r": cav.r, "gamma": cav.gamma, "nu": cav.nu, "u_lid": cav.u_lid}
            self.fut[name] = self.ex.submit(oracle_solve, (d, tols, max_steps, self.threads))

    def result(self, name, tol, timeout):
        try:
            return self.fut[name].result(timeout=timeout).get(tol)
        except Exception:
            return None

    def close(self):
        """Stop every worker (a run still going is abandoned), so that nothing
        else loads the host cores afterwards."""
        for f in self.fut.values():
            f.cancel()
        procs = list(getattr(self.ex, "_processes", {}).values())
        self.ex.shutdown(wait=False, cancel_futures=True)
        for pr in procs:
            if pr.is_alive():
                pr.terminate()
            pr.join(timeout=10)


def rel_l2(a, b):
    """||(u_x, u_y)_a - (u_x, u_y)_b||_2 / ||(u_x, u_y)_b||_2."""
    import numpy as np
    num = np.sum((a[0] - b[0]) ** 2 + (a[1] - b[1]) ** 2)
    den = np.sum(b[0] ** 2 + b[1] ** 2)
    return float(np.sqrt(num / den))


PENDING = []


def with_oracle(entry, fields, oj, name, tol, timeout):
    """Queue the comparison of a GPU result with the FP64 oracle's run to the
    same residual; resolve_oracle() adds the oracle's steps and the relative
    L2 error of (u_x, u_y) once the oracle has finished."""
    PENDING.append((entry, fields, oj, name, tol, timeout))
    return entry


def resolve_oracle():
    t0 = time.perf_counter()
    for entry, fields, oj, name, tol, timeout in PENDING:
        r = oj.result(name, tol, max(1.0, timeout - (time.perf_counter() - t0))) if oj else None
        if r is None:
            entry["oracle"] = "unavailable (not finished within %.0f s)" % timeout
            continue
        st, steps, res, ux, uy, secs = r
        entry["oracle_steps"] = steps
        entry["oracle_status"] = st
        if fields is not None and st == "converged":
            entry["oracle_rel_l2"] = rel_l2((fields[1], fields[2]), (ux, uy))
    PENDING.clear()


def gpu_solve(L, cav, dtype, tol, budget_s, tune=False):
    """One steady-state solve from rest on a single-instance handle: wall time
    from the first step to the launch that met the residual, residual checks
    included.  With tune, the library's autotuner first picks the engine
    (interior variants, cluster engine, general kernel; the state is restored
    and the tuning is not in the time)."""
    p = L.lbm_params_init(cav.nx, cav.ny, cav.r, cav.gamma, cav.nu, cav.u_lid, dtype)
    g = L.Lbm(p)
    tuned = g.autotune(200) if tune else None
    t0 = time.perf_counter()
    steps, st = 0, None
    while time.perf_counter() - t0 < budget_s:
        st, n = g.run(tol, 100000)
        steps += n
        if st == L.OK:
            break
    dts = time.perf_counter() - t0
    out = {"status": "converged" if st == L.OK else "unfinished", "steps": steps, "s": dts,
           "residual": g.residual(), "us_per_step": 1e6 * dts / max(steps, 1), "engine": g.variant}
    if tuned:
        out["autotune_ms_per_step"] = tuned[1]
    fields = g.fields() if st == L.OK else None
    g.close()
    return out, fields


def promoted_solve(cav, tol):
    """The FP16 -> FP32 precision schedule on single-instance handles."""
    from paper_2208_03562_gb300 import serve as SV
    t0 = time.perf_counter()
    r = SV.solve_promoted(cav.nx, cav.ny, cav.r, cav.gamma, cav.nu, cav.u_lid, tol, 20_000_000)
    out = {"status": r["status"], "steps": r["steps"], "steps_by_stage": r["steps_by_stage"],
           "s": time.perf_counter() - t0, "residual": r.get("residual")}
    return out, r.get("fields")


def ttss_leg(L, oj, c2_f64_budget_s=20.0, budget_s=30.0):
    """Time to steady state (Sec. 5.2), each result with its error against the
    FP64 oracle run from rest to the same residual:
    - deep cavity 100 x 150 (AR = 2, r = 4/3, Re = 1000, Ma = 0.06), residual
      1e-6: the plain FP64 path at gamma = 1 against the preconditioned FP32
      path (gamma = 0.1) and the FP16 -> FP32 schedule (gamma = 0.1), with the
      step and time ratios;
    - deep cavity 128 x 128 (r = 2, Re = 1000, Ma = 0.06): FP32 gamma = 0.1 to
      1e-6 and to 1e-7, the FP16 -> FP32 schedule on the batch engine (the
      solve server) and on single-instance handles, and the plain FP64 gamma = 1
      path for at most c2_f64_budget_s seconds (it does not settle on this
      grid: a lower bound);
    - the square cavity 64 x 64 (r = gamma = 1, Re = 100, U = 0.1) in FP64 to
      1e-8."""
    from paper_2208_03562_gb300 import inputs as I
    from paper_2208_03562_gb300 import serve as SV
    out = {}
    # deep cavity 100 x 150
    d = {"workload": "deep lid-driven cavity 100x150, AR=2, r=4/3, Re=1000, Ma=0.06, from rest (Sec. 5.2)",
         "tol": 1e-6}
    c1 = deep_cavity_100x150(1.0, "f64")
    r, f = gpu_solve(L, c1, L.F64, 1e-6, 4 * budget_s, tune=True)
    d["f64_plain_gamma1"] = with_oracle(r, f, oj, "deep100_g1", 1e-6, 240)
    c01 = deep_cavity_100x150(0.1, "f32")
    r, f = gpu_solve(L, c01, L.F32, 1e-6, budget_s)
    d["f32_gamma0.1"] = with_oracle(r, f, oj, "deep100_g0.1", 1e-6, 120)
    r, f = gpu_solve(L, deep_cavity_100x150(1.0, "f32"), L.F32, 1e-6, budget_s)
    d["f32_gamma1"] = with_oracle(r, f, oj, "deep100_g1", 1e-6, 240)
    r, f = promoted_solve(c01, 1e-6)
    d["f16_to_f32_gamma0.1"] = with_oracle(r, f, oj, "deep100_g0.1", 1e-6, 120)
    a, b, c = d["f32_gamma0.1"], d["f64_plain_gamma1"], d["f16_to_f32_gamma0.1"]
    if a["status"] == "converged" and b["status"] == "converged":
        d["speedup_f32_vs_f64_plain"] = b["s"] / a["s"]
        d["step_ratio_f64_gamma1_over_f32_gamma0.1"] = b["steps"] / a["steps"]
    if c["status"] == "converged" and b["status"] == "converged":
        d["speedup_f16_to_f32_vs_f64_plain"] = b["s"] / c["s"]
    out["deep_100x150"] = d
    # deep cavity 128 x 128
    e = {"workload": "deep lid-driven cavity 128x128, r=2 (H/L=2), Re=1000, Ma=0.06, from rest", "tol": 1e-6}
    cav = I.deep_cavity_128(0.1)
    r, f = gpu_solve(L, cav, L.F32, 1e-6, budget_s)
    e["f32_gamma0.1"] = with_oracle(r, f, oj, "deep128_g0.1", 1e-6, 120)
    r, f = gpu_solve(L, cav, L.F32, 1e-7, budget_s)
    e["f32_gamma0.1_tol1e-7"] = with_oracle(r, f, oj, "deep128_g0.1", 1e-7, 120)
    t0 = time.perf_counter()
    srv = SV.gpu_server(SV.fp16_schedule(2000), capacity=2, reserve_bytes=0, budget_bytes=1 << 30,
                        keep_fields=True)
    p = L.lbm_params_init(cav.nx, cav.ny, cav.r, cav.gamma, cav.nu, cav.u_lid, L.F16)
    res = srv.serve([SV.SolveRequest(0, 0.0, p, 1e-6, 20_000_000)], time_limit_s=budget_s)
    srv.close()
    if res:
        r = {"status": res[0].status, "steps": res[0].steps, "steps_by_stage": res[0].steps_by_stage,
             "s": time.perf_counter() - t0, "residual": res[0].residual, "engine": "batch"}
        e["f16_to_f32_gamma0.1"] = with_oracle(r, res[0].fields, oj, "deep128_g0.1", 1e-6, 120)
    r, f = promoted_solve(cav, 1e-6)
    e["f16_to_f32_gamma0.1_single"] = with_oracle(r, f, oj, "deep128_g0.1", 1e-6, 120)
    c64 = I.deep_cavity_128(1.0, "f64")
    r, _ = gpu_solve(L, c64, L.F64, 1e-6, c2_f64_budget_s, tune=True)
    r["note"] = "lower bound: stopped at the time budget (omega_nu = 1.90 at gamma = 1; no oracle run)"
    e["f64_plain_gamma1"] = r
    out["deep_128x128"] = e
    # square cavity 64 x 64, FP64
    q = I.square_cavity_64()
    r, f = gpu_solve(L, q, L.F64, 1e-8, budget_s, tune=True)
    out["square_64x64_f64"] = with_oracle(r, f, oj, "square64", 1e-8, 60)
    out["square_64x64_f64"]["workload"] = "square cavity 64x64, r=gamma=1, Re=100, U=0.1, FP64, residual 1e-8"
    return out


def ttss_oracle_jobs():
    """The FP64 oracle runs that the time-to-steady-state results are
    compared with (name, cavity, tolerances, step limit)."""
    from paper_2208_03562_gb300 import inputs as I
    return [("deep100_g1", deep_cavity_100x150(1.0, "f64"), [1e-6], 2_000_000),
            ("deep128_g0.1", I.deep_cavity_128(0.1, "f64"), [1e-6, 1e-7], 2_000_000),
            ("deep100_g0.1", deep_cavity_100x150(0.1, "f64"), [1e-6], 2_000_000),
            ("square64", I.square_cavity_64(), [1e-8], 20000)]


def run_batch(L, cavs, budget_s):
    """One batch of the given cavities (FP32), persistent launches of 2000
    steps until every slot retired or the time budget ran out.  Returns
    per-cavity (state, steps, residual, projected remaining steps or None)
    and the launch record."""
    import math
    b = L.Batch(max(1, len(cavs)), L.F32)
    slots = []
    for c in cavs:
        p = L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid, L.F32)
        slots.append((b.add(p, c.tol, c.max_steps), c))
    best, ms = b.autotune(20) if cavs else (None, [])  # persistent-grid size; slot state restored
    t0 = time.perf_counter()
    launches, active = 0, len(cavs)
    hist = {s: [] for s, _ in slots}
    while active and time.perf_counter() - t0 < budget_s:
        active = b.run(2000)
        launches += 1
        for s, _ in slots:
            info, st = b.query(s)
            if st == L.SLOT_ACTIVE:
                hist[s] = (hist[s] + [(info.step, info.residual)])[-4:]
    dt = time.perf_counter() - t0
    per = []
    for s, c in slots:
        info, st = b.query(s)
        left = None
        if st == L.SLOT_ACTIVE:
            h = hist[s]
            if len(h) >= 2 and 0 < h[-1][1] < h[0][1]:
                rate = math.log(h[0][1] / h[-1][1]) / (h[-1][0] - h[0][0])
                left = max(0.0, min(math.log(h[-1][1] / c.tol) / rate, c.max_steps - info.step))
        per.append((L.SLOT_NAMES[st], int(info.step), float(info.residual), left))
    b.close()
    return per, {"wall_s": dt, "launches": launches, "autotune": {"ctas_per_sm": best, "ms_per_step": ms}}


def batch_summary(cavs, per, wall_s):
    n = len(cavs)
    ns = sum(step * c.nodes for (_, step, _, _), c in zip(per, cavs))
    states = {}
    for st, _, _, _ in per:
        states[st] = states.get(st, 0) + 1
    agg = ns / wall_s / 1e9
    peak, kind = peak_hbm()
    out = {"workload": "%d cavities, nx 64..1024, ny 32..512, r in {0.25,0.5,1,2}, gamma 0.05..1, Re 100..5000, "
                       "FP32, residual 1e-7 (seed 0)" % n,
           "aggregate_glups": agg,
           "hbm_frac": {"value": agg * BYTES_PER_NODE["f32"] / peak, "peak_gbs": peak, "peak_kind": kind,
                        "what": "aggregate node updates x 72 B (FP32 algorithmic bytes) / HBM copy bandwidth"},
           "wall_s": wall_s, "states": states,
           "retired_fraction": (n - states.get("ACTIVE", 0)) / n}
    if states.get("ACTIVE", 0):
        rem = sum(left * c.nodes for (st, _, _, left), c in zip(per, cavs) if st == "ACTIVE" and left is not None)
        stuck = sum(1 for st, _, _, left in per if st == "ACTIVE" and left is None)
        out["projected_wall_s_to_retire_all"] = wall_s + rem / (agg * 1e9)
        out["projection"] = ("active slots: remaining steps from the residual decay over their last launches "
                             "(capped at the step limit), remaining node-steps at the measured aggregate rate; "
                             "%d active slots whose residual did not fall are not in it" % stuck)
    return out


def batch_leg(L, budget_s=30.0, n=256):
    """The batched sweep: n uneven cavities (seed 0) in one batch, persistent
    launches until every slot retired or the time budget ran out; aggregate
    GLUPS over the slots' own steps, the fraction retired, and a projection of
    the wall time to retire the whole mix: each active slot's remaining steps
    from the decay of its residual over the last launches, and the remaining
    node-steps at the measured aggregate rate."""
    from paper_2208_03562_gb300 import inputs as I
    cavs = I.batched_sweep(seed=0, n=n, dtype="f32")
    per, rec = run_batch(L, cavs, budget_s)
    out = batch_summary(cavs, per, rec["wall_s"])
    out["launches"] = rec["launches"]
    out["autotune"] = rec["autotune"]
    return out


def batch_leg_sharded(L, dist, rank, world, torch, budget_s=30.0, n=256):
    """The batched sweep on `world` GPUs: whole cavities placed on ranks by
    the greedy bytes x expected-steps balance (shard.py), one batch per rank,
    no collective on the data path; per-cavity results gathered on rank 0.
    The wall time is the slowest rank's."""
    from paper_2208_03562_gb300 import inputs as I
    from paper_2208_03562_gb300 import shard as SH
    cavs = I.batched_sweep(seed=0, n=n, dtype="f32")
    rec = {}

    def solve(mine):
        per, r = run_batch(L, mine, budget_s)
        rec.update(r)
        return per

    torch.cuda.synchronize()
    dist.barrier()
    per = SH.run_sharded(cavs, [SH.cost(c) for c in cavs], solve, rank, world, dist)
    wall = max_over_ranks(rec["wall_s"], dist, torch, "cuda")
    if rank != 0:
        return None
    out = batch_summary(cavs, per, wall)
    out["placement"] = "greedy longest-first over bytes x expected steps, %d ranks" % world
    return out


def serve_leg(L, budget_s=60.0, n=256, scale=1, capacity=16):
    """The serving workload: Poisson arrivals (50/s, seed 0) of steady-state
    solves, FP16 storage until the residual stalls, then FP32 to 1e-6, for at
    most budget_s seconds; the requests still running or waiting then are
    counted as unfinished.  At most `capacity` solves share the device at a
    time (first come, first served, and within device memory): the offered
    load is far above what the device completes, and with every request
    admitted at once none would finish within the budget."""
    from paper_2208_03562_gb300 import inputs as I
    from paper_2208_03562_gb300 import serve as SV
    reqs = []
    for i, rq in enumerate(I.serving_requests(seed=0, n=n, scale=scale)):
        c = rq.cavity
        reqs.append(SV.SolveRequest(i, rq.arrival_s, L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid,
                                                                        L.F16), c.tol, c.max_steps))
    srv = SV.gpu_server(SV.fp16_schedule(2000), capacity=capacity, keep_fields=False)
    res = srv.serve(reqs, time_limit_s=budget_s)
    sm = SV.summary(srv, res)
    srv.close()
    sm["unfinished"] = n - len(res)
    sm["workload"] = ("%d requests of the serving mix (Poisson 50/s, nx 128..2048, ny 64..1024, r 0.25..2, "
                      "gamma 0.05..1, Re 100..1000, seed 0)%s; FP16->FP32, residual 1e-6, %.0f s budget, "
                      "at most %d solves on the device at a time"
                      % (n, "" if scale == 1 else " with both grid dimensions divided by %d" % scale, budget_s,
                         capacity))
    sm["note"] = "time-bounded: percentiles are over the requests that finished within the budget"
    return sm


def oracle_sample_rate(nx, ny, steps_budget_s=12.0, max_steps=200, threads=0):
    """The FP64 oracle on a slab of the workload, on `threads` host cores
    (0: every core this process may use)."""
    from oracle import stepper as S
    from paper_2208_03562_gb300 import inputs as I
    cav = I.shallow_cavity_8192x2048("f64")
    threads = S.num_threads(threads if threads > 0 else len(os.sched_getaffinity(0)))
    o = S.Oracle(S.OracleParams(nx=nx, ny=ny, r=cav.r, gamma=cav.gamma, nu=cav.nu, u_lid=cav.u_lid))
    t = time.perf_counter()
    o.step(1)
    one = max(time.perf_counter() - t, 1e-6)
    steps = int(max(2, min(max_steps, steps_budget_s / one)))
    t = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t
    return nx * ny * steps / dt / 1e9, threads, steps, dt


def reference_main(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import stepper as S
    from paper_2208_03562_gb300 import inputs as I
    cav = I.shallow_cavity_8192x2048("f64")
    nx, ny = cav.nx, 64  # slab: full width, 64 rows of the workload per step
    threads = S.num_threads(len(os.sched_getaffinity(0)))
    o = S.Oracle(S.OracleParams(nx=nx, ny=ny, r=cav.r, gamma=cav.gamma, nu=cav.nu, u_lid=cav.u_lid))
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    v = nx * ny * args.steps / dt / 1e9
    sample = "FP64 oracle (plain C, OpenMP over rows) on a %dx%d slab of the 8192x2048 workload, %d steps" % (
        nx, ny, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(cav),
            "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def profile_case(name):
    """Profiling only: a small fixed workload of one engine, two launches, for
    an ncu capture of the second (`-k regex:k_batch` or `regex:k_cluster`,
    `-s 1 -c 1`).
    batch: the first 24 cavities of the batched-sweep mix (FP32, 4.3 M
    nodes, both population sets 311 MB > L2), launches of 20 and 60 steps.
    cluster: the 128 x 128 deep cavity (r = 2, gamma = 0.1, FP32), launches of
    200 and 2000 steps."""
    import torch
    torch.cuda.set_device(0)
    from paper_2208_03562_gb300 import lbm as L, inputs as I
    L.load()
    if name == "batch":
        mix = I.batched_sweep(seed=0, n=256, dtype="f32")[:24]
        b = L.Batch(len(mix), L.F32)
        for c in mix:
            b.add(L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid, L.F32), 1e-30, 10 ** 6)
        b.run(20)
        b.run(60)
        b.close()
        out = {"profile_case": name, "slots": len(mix), "nodes": sum(c.nodes for c in mix), "steps": [20, 60]}
    else:
        cav = I.deep_cavity_128(0.1)
        h = L.Lbm(L.lbm_params_init(cav.nx, cav.ny, cav.r, 0.1, cav.nu, cav.u_lid, L.F32))
        if h.variant != L.VARIANT_CLUSTER:
            raise RuntimeError("the 128 x 128 cavity did not select the cluster engine")
        h.step(200)
        h.step(2000)
        h.sync()
        out = {"profile_case": name, "nodes": cav.nodes, "steps": [200, 2000], "step_after": h.info().step}
        h.close()
    print(json.dumps(out))


def main():
    args = parse()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.nx or args.ny:
        GRID_OVERRIDE.update(nx=args.nx, ny=args.ny)
    if args.variant is not None:
        FORCE_VARIANT[args.dtype] = args.variant
    if args.impl == "reference":
        return reference_main(args)
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    from paper_2208_03562_gb300 import lbm as L
    L.load()
    dev_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local

    cav, ms, info, clocks, tuned, launch = gpu_leg(args.dtype, args.steps, args.warmup, torch, L, dist, dev_index)
    nodes = cav.nodes
    ms_step = ms / args.steps
    glups = world * nodes * args.steps / (ms / 1e3) / 1e9
    peak, peak_kind = peak_hbm()
    bpn = BYTES_PER_NODE[args.dtype]
    achieved = bpn * nodes / (ms_step / 1e3) / 1e9
    line = {"metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic", "config": config_of(cav),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": ncu_traffic("k_step_" + args.dtype),
                         "peak_kind": peak_kind, "bytes_per_node": bpn, "nodes_per_launch": nodes,
                         "kernel": "k_step_tma (interior tiles + edge strips, one launch per step)",
                         "timing": kernel_timing(ms_step, launch)},
            "gpu_launches": args.steps + args.steps // 20,
            "clocks": clocks,
            "residual_at_end": info.residual,
            "autotune": tuned}
    extras = {}
    if not args.no_extras and args.dtype == "f32":
        cav16, ms16, _, _, tuned16, launch16 = gpu_leg("f16", args.steps, args.warmup, torch, L, dist, None)
        s16 = ms16 / args.steps
        a16 = BYTES_PER_NODE["f16"] * nodes / (s16 / 1e3) / 1e9
        extras["fp16"] = {"value": world * nodes * args.steps / (ms16 / 1e3) / 1e9, "unit": "GLUPS",
                          "ms_per_step": s16,
                          "roofline": {"bound": "hbm", "achieved": a16, "peak": peak, "unit": "GB/s",
                                       "frac": a16 / peak, "bytes_per_node": 36,
                                       "traffic": ncu_traffic("k_step_f16")},
                          "variant": tuned16.get("variant"), "regions_ms": tuned16.get("regions_ms"),
                          "what": "FP16 shifted storage, FP32 collision, same workload and timing"}
        cav64, ms64, _, _, _, launch64 = gpu_leg("f64", max(20, args.steps // 10), args.warmup, torch, L, dist,
                                                 None)
        st64 = max(20, args.steps // 10)
        extras["fp64"] = {"value": world * nodes * st64 / (ms64 / 1e3) / 1e9, "unit": "GLUPS",
                          "ms_per_step": ms64 / st64, "steps": st64,
                          "hbm_frac": 144 * nodes / (ms64 / st64 / 1e3) / 1e9 / peak,
                          "what": "plain FP64 path (general kernel, FP64 collision): bound by FP64 ALU throughput"}
    if world > 1 and not args.no_extras and "batched_sweep" not in args.skip:
        try:
            r = batch_leg_sharded(L, dist, rank, world, torch)
        except Exception as e:  # reported, not hidden
            r = {"error": repr(e)}
        if rank == 0:
            extras["batched_sweep"] = r
    if rank == 0 and not args.no_extras:
        try:
            line["e2e"] = e2e_leg(args.steps, torch, L)
        except Exception as e:  # reported, not hidden
            line["e2e"] = {"error": repr(e)}
        oj = None
        if "time_to_steady_state" not in args.skip:
            oj = OracleJobs(ttss_oracle_jobs())
        for key, fn in (("time_to_steady_state", lambda L: ttss_leg(L, oj)), ("batched_sweep", batch_leg),
                        ("serving", serve_leg)):
            if key in args.skip or key in extras:
                continue
            try:
                extras[key] = fn(L)
            except Exception as e:  # reported, not hidden
                extras[key] = {"error": repr(e)}
        if oj:
            resolve_oracle()
            extras["time_to_steady_state"]["oracle_cores"] = {"workers": 3, "threads_each": oj.threads}
            oj.close()
        v1, _, steps1, dt1 = oracle_sample_rate(8192, 8, steps_budget_s=3.0, max_steps=100, threads=1)
        v, threads, steps, dt = oracle_sample_rate(8192, 64)
        line["cpu_baseline"] = {"value": v, "unit": "GLUPS", "cores": threads, "kind": "oracle",
                                "sample": "FP64 oracle on an 8192x64 slab of the workload, %d steps, %.1f s"
                                          % (steps, dt),
                                "single_core": {"value": v1, "unit": "GLUPS", "cores": 1,
                                                "sample": "FP64 oracle on an 8192x8 slab, %d steps, %.1f s"
                                                          % (steps1, dt1)}}
    # the large objects first, the compact FP64 / FP16 summaries last
    for key in ("time_to_steady_state", "batched_sweep", "serving", "fp64", "fp16"):
        if key in extras:
            line[key] = extras[key]
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
