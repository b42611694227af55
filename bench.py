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
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(clocks_index) if clocks_index is not None else None
    if sampler:
        sampler.__enter__()
        time.sleep(0.4)
    t0.record(stream)
    g.step(steps)
    t1.record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.__exit__()
    ms = t0.elapsed_time(t1)
    if dist:
        ms = max_over_ranks(ms, dist, torch, "cuda")
        dist.barrier()
    info = g.info()
    launch = launch_times(g, min(steps, 200), torch)
    g.close()
    return cav, ms, info, (sampler.summary() if sampler else None), tuned, launch


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


def ttss_leg(L, budget_s=60.0):
    """Time to steady state on the deep cavity (128 x 128, r = 2, Re = 1000,
    Ma = 0.06), to residual 1e-6 (Sec. 5.2), wall time from the first step to
    the step that met the residual, with the residual checks included:
    - the preconditioned FP32 path (gamma = 0.1), a single-instance handle,
      also to residual 1e-7;
    - the FP16 -> FP32 precision schedule (gamma = 0.1) through the solve
      server (batch engine, stall test on the device) and on single-instance
      handles (stall test on the host between launches);
    - the plain FP64 path (gamma = 1, no preconditioning), for at most
      budget_s seconds: on this grid it does not settle (its shear rate is
      close to the stability limit), so the figure is a lower bound."""
    from paper_2208_03562_gb300 import inputs as I
    import time as _t
    out = {"workload": "deep lid-driven cavity 128x128, r=2 (H/L=2), Re=1000, Ma=0.06, from rest",
           "tol": 1e-6}
    for name, dt, gamma, bud, tol in (("f32_gamma0.1", L.F32, 0.1, budget_s / 3, 1e-6),
                                      ("f32_gamma0.1_tol1e-7", L.F32, 0.1, budget_s / 3, 1e-7),
                                      ("f16_to_f32_gamma0.1", None, 0.1, budget_s / 3, 1e-6),
                                      ("f16_to_f32_gamma0.1_single", "single", 0.1, budget_s / 3, 1e-6),
                                      ("f64_plain_gamma1", L.F64, 1.0, budget_s, 1e-6)):
        cav = I.deep_cavity_128(gamma)
        t0 = _t.perf_counter()
        steps, st = 0, None
        if dt == "single":  # the same schedule on single-instance handles (cluster engine)
            from paper_2208_03562_gb300 import serve as SV
            r = SV.solve_promoted(cav.nx, cav.ny, cav.r, gamma, cav.nu, cav.u_lid, 1e-6, 20_000_000)
            out[name] = {"status": r["status"], "steps": r["steps"], "steps_by_stage": r["steps_by_stage"],
                         "s": _t.perf_counter() - t0, "residual": r.get("residual")}
            continue
        if dt is None:  # FP16 storage until the residual stalls, then FP32
            from paper_2208_03562_gb300 import serve as SV
            srv = SV.gpu_server(SV.fp16_schedule(2000), capacity=2, reserve_bytes=0, budget_bytes=1 << 30,
                                keep_fields=False)
            p = L.lbm_params_init(cav.nx, cav.ny, cav.r, gamma, cav.nu, cav.u_lid, L.F16)
            r = srv.serve([SV.SolveRequest(0, 0.0, p, 1e-6, 20_000_000)], time_limit_s=bud)
            srv.close()
            dts = _t.perf_counter() - t0
            if r:
                out[name] = {"status": r[0].status, "steps": r[0].steps, "steps_by_stage": r[0].steps_by_stage,
                             "s": dts, "residual": r[0].residual}
            else:
                out[name] = {"status": "unfinished", "s": dts}
            continue
        p = L.lbm_params_init(cav.nx, cav.ny, cav.r, gamma, cav.nu, cav.u_lid, dt)
        g = L.Lbm(p)
        while _t.perf_counter() - t0 < bud:
            st, n = g.run(tol, 100000)
            steps += n
            if st == L.OK:
                break
        dts = _t.perf_counter() - t0
        out[name] = {"status": "converged" if st == L.OK else "unfinished", "steps": steps, "s": dts,
                     "residual": g.residual(), "us_per_step": 1e6 * dts / max(steps, 1), "tol": tol}
        g.close()
    a, b = out.get("f32_gamma0.1", {}), out.get("f64_plain_gamma1", {})
    if a.get("status") == "converged" and b.get("status") == "converged":
        out["speedup_f32_vs_f64_plain"] = b["s"] / a["s"]
        out["step_ratio_gamma1_over_gamma0.1"] = b["steps"] / a["steps"]
    return out


def batch_leg(L, budget_s=30.0, n=256):
    """The batched sweep: n uneven cavities (seed 0) in one batch, persistent
    launches until every slot retired or the time budget ran out; aggregate
    GLUPS over the slots' own steps."""
    from paper_2208_03562_gb300 import inputs as I
    import time as _t
    cavs = I.batched_sweep(seed=0, n=n, dtype="f32")
    b = L.Batch(n, L.F32)
    slots = []
    for c in cavs:
        p = L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid, L.F32)
        slots.append((b.add(p, c.tol, c.max_steps), c.nodes))
    best, ms = b.autotune(20)  # persistent-grid size; the slots' state is restored
    t0 = _t.perf_counter()
    launches, active = 0, n
    while active and _t.perf_counter() - t0 < budget_s:
        active = b.run(2000)
        launches += 1
    dt = _t.perf_counter() - t0
    ns, states = 0, {}
    for s, nodes in slots:
        info, st = b.query(s)
        ns += info.step * nodes
        states[L.SLOT_NAMES[st]] = states.get(L.SLOT_NAMES[st], 0) + 1
    b.close()
    return {"workload": "%d cavities, nx 64..1024, ny 32..512, r in {0.25,0.5,1,2}, gamma 0.05..1, Re 100..5000, "
                        "FP32, residual 1e-7 (seed 0)" % n,
            "aggregate_glups": ns / dt / 1e9, "wall_s": dt, "launches": launches, "states": states,
            "autotune": {"ctas_per_sm": best, "ms_per_step": ms},
            "note": "time-bounded: slots still ACTIVE had not reached 1e-7 when the budget ran out"}


def serve_leg(L, budget_s=60.0, n=64, scale=4):
    """The serving workload: Poisson arrivals (50/s, seed 0) of steady-state
    solves, FP16 storage until the residual stalls, then FP32 to 1e-6. The
    bench runs the first n requests with both grid dimensions divided by
    `scale`. The full mix (256 requests up to 2048 x 1024, ~1e5-1e6 steps
    each) takes tens of GPU-minutes."""
    from paper_2208_03562_gb300 import inputs as I
    from paper_2208_03562_gb300 import serve as SV
    reqs = []
    for i, rq in enumerate(I.serving_requests(seed=0, n=n, scale=scale)):
        c = rq.cavity
        reqs.append(SV.SolveRequest(i, rq.arrival_s, L.lbm_params_init(c.nx, c.ny, c.r, c.gamma, c.nu, c.u_lid,
                                                                        L.F16), c.tol, c.max_steps))
    srv = SV.gpu_server(SV.fp16_schedule(2000), capacity=n, keep_fields=False)
    res = srv.serve(reqs, time_limit_s=budget_s)
    sm = SV.summary(srv, res)
    srv.close()
    sm["unfinished"] = n - len(res)
    sm["workload"] = ("first %d requests of the serving mix (Poisson 50/s, nx 128..2048, ny 64..1024, r 0.25..2, "
                      "gamma 0.05..1, Re 100..1000, seed 0) with both grid dimensions divided by %d; "
                      "FP16->FP32, residual 1e-6" % (n, scale))
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
    if not args.no_extras and args.dtype == "f32":
        cav16, ms16, _, _, tuned16, launch16 = gpu_leg("f16", args.steps, args.warmup, torch, L, dist, None)
        s16 = ms16 / args.steps
        a16 = BYTES_PER_NODE["f16"] * nodes / (s16 / 1e3) / 1e9
        line["fp16"] = {"value": world * nodes * args.steps / (ms16 / 1e3) / 1e9, "unit": "GLUPS",
                        "ms_per_step": s16, "roofline": {"achieved": a16, "peak": peak, "frac": a16 / peak,
                                                         "bytes_per_node": 36,
                                                         "traffic": ncu_traffic("k_step_f16"),
                                                         "timing": kernel_timing(s16, launch16)},
                        "autotune": tuned16}
    if not args.no_extras and args.dtype == "f32":
        cav64, ms64, _, _, _, launch64 = gpu_leg("f64", max(20, args.steps // 10), args.warmup, torch, L, dist, None)
        st64 = max(20, args.steps // 10)
        line["fp64"] = {"value": world * nodes * st64 / (ms64 / 1e3) / 1e9, "unit": "GLUPS",
                        "ms_per_step": ms64 / st64, "steps": st64,
                        "roofline_hbm": {"achieved": 144 * nodes / (ms64 / st64 / 1e3) / 1e9,
                                         "peak": peak, "bytes_per_node": 144,
                                         "timing": kernel_timing(ms64 / st64, launch64)},
                        "note": "plain FP64 path (general kernel, FP64 collision): bound by FP64 ALU throughput"}
    if rank == 0 and not args.no_extras:
        try:
            line["e2e"] = e2e_leg(args.steps, torch, L)
        except Exception as e:  # reported, not hidden
            line["e2e"] = {"error": repr(e)}
        for key, fn in (("time_to_steady_state", ttss_leg), ("batched_sweep", batch_leg), ("serving", serve_leg)):
            if key in args.skip:
                continue
            try:
                line[key] = fn(L)
            except Exception as e:  # reported, not hidden
                line[key] = {"error": repr(e)}
        v1, _, steps1, dt1 = oracle_sample_rate(8192, 8, steps_budget_s=3.0, max_steps=100, threads=1)
        v, threads, steps, dt = oracle_sample_rate(8192, 64)
        line["cpu_baseline"] = {"value": v, "unit": "GLUPS", "cores": threads, "kind": "oracle",
                                "sample": "FP64 oracle on an 8192x64 slab of the workload, %d steps, %.1f s"
                                          % (steps, dt),
                                "single_core": {"value": v1, "unit": "GLUPS", "cores": 1,
                                                "sample": "FP64 oracle on an 8192x8 slab, %d steps, %.1f s"
                                                          % (steps1, dt1)}}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
