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
import glob
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
    ap.add_argument("--no-extras", action="store_true", help="skip FP16, e2e and CPU-baseline legs")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16", "f64"], help="storage of the primary leg")
    ap.add_argument("--nx", type=int, default=0, help="profiling only: override the grid width")
    ap.add_argument("--ny", type=int, default=0, help="profiling only: override the grid height")
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


def kernel_source_hash():
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2208_03562_gb300", "csrc", "*"))):
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
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
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    info = g.info()
    g.close()
    return cav, ms, info, (sampler.summary() if sampler else None), tuned


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


def oracle_sample_rate(nx, ny, steps_budget_s=12.0, max_steps=200):
    """The FP64 oracle on the host cores on a slab of the workload."""
    from oracle import stepper as S
    from paper_2208_03562_gb300 import inputs as I
    cav = I.shallow_cavity_8192x2048("f64")
    threads = S.num_threads(len(os.sched_getaffinity(0)))
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


def main():
    args = parse()
    if args.nx or args.ny:
        GRID_OVERRIDE.update(nx=args.nx, ny=args.ny)
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

    cav, ms, info, clocks, tuned = gpu_leg(args.dtype, args.steps, args.warmup, torch, L, dist, dev_index)
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
                         "peak_kind": peak_kind, "bytes_per_node": bpn,
                         "kernel": "k_step (+ 1 finalize per 20 steps in the timed region)"},
            "gpu_launches": 1 + args.steps + args.steps // 20,
            "clocks": clocks,
            "residual_at_end": info.residual,
            "autotune": tuned}
    if not args.no_extras and args.dtype == "f32":
        cav16, ms16, _, _, tuned16 = gpu_leg("f16", args.steps, args.warmup, torch, L, dist, None)
        s16 = ms16 / args.steps
        a16 = BYTES_PER_NODE["f16"] * nodes / (s16 / 1e3) / 1e9
        line["fp16"] = {"value": world * nodes * args.steps / (ms16 / 1e3) / 1e9, "unit": "GLUPS",
                        "ms_per_step": s16, "roofline": {"achieved": a16, "peak": peak, "frac": a16 / peak,
                                                         "bytes_per_node": 36,
                                                         "traffic": ncu_traffic("k_step_f16")},
                        "autotune": tuned16}
    if rank == 0 and not args.no_extras:
        try:
            line["e2e"] = e2e_leg(args.steps, torch, L)
        except Exception as e:  # reported, not hidden
            line["e2e"] = {"error": repr(e)}
        v, threads, steps, dt = oracle_sample_rate(8192, 64)
        line["cpu_baseline"] = {"value": v, "unit": "GLUPS", "cores": threads, "kind": "oracle",
                                "sample": "FP64 oracle on an 8192x64 slab of the workload, %d steps, %.1f s"
                                          % (steps, dt)}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
