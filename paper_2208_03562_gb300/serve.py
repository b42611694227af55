"""Continuous-batching server of steady-state cavity solves.

Requests arrive over time. Each one is a lid-driven cavity: grid, r, gamma,
nu, lid speed, residual tolerance and step limit. The server holds every
admitted solve on the device as a slot of a batched engine (``lbm.Batch``).
One persistent launch advances all slots at once. Between launches the server:

- admits waiting requests, first come first served, while a slot and device
  memory are free;
- collects each solve whose FP64 residual ||u_x(t) - u_x(t-20)||_2 (Sec. 5.2)
  has fallen below its tolerance, with its fields.

Requests that arrive while others are on the GPU join the next launch, so
their work overlaps. A slot retires on the device at the step where it
converges, so its result does not depend on when the host looks or on the
other slots of the mix.

Admission is by device memory. The server takes a byte budget (by default the
free device memory at start minus a reserve) and admits a request only if its
slot fits into what the resident solves leave. A request that could never fit
is rejected at once instead of blocking the queue.

Precision schedule. Storage stages run from narrow to wide, e.g. FP16 then
FP32, both with FP32 collision and FP64 residuals. A solve starts in the first
stage. When its residual stops falling there, it moves to the next stage. The
batch's stall test detects this on the device: the residual is compared with
the one `stall_window` steps earlier. In FP16 the stall is the rounding floor,
since half precision keeps 11 significant bits. The move reads the slot's
populations into a device staging buffer, releases the slot, fills a slot of
the next stage from the buffer, and goes on with the remaining step budget.
The state never leaves the device. The last stage has no stall test.

No counterpart in the paper: this is how many independent steady-state
solves of the method share one GPU.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

# slot states of the batched engine (include/prc_lbm.h, lbm_slot_state)
SLOT_ACTIVE, SLOT_CONVERGED, SLOT_DIVERGED, SLOT_MAXSTEPS, SLOT_EMPTY, SLOT_STALLED = range(6)


@dataclass
class Stage:
    """One storage precision of the schedule.  stall_window = 0: no stall test
    (a solve stays in this stage until it converges, diverges or runs out of
    steps)."""
    dtype: int
    stall_window: int = 0
    stall_ratio: float = 0.9


@dataclass
class SolveRequest:
    rid: int
    arrival_s: float
    params: object          # lbm_params; the dtype field is set per stage
    tol: float
    max_steps: int
    mass0: float = None     # total mass of the initial state (default: rest, nx ny rho0)

    def __post_init__(self):
        if self.mass0 is None:
            self.mass0 = float(self.nodes)

    @property
    def nodes(self) -> int:
        return int(self.params.nx) * int(self.params.ny)


@dataclass
class SolveResult:
    rid: int
    status: str                       # converged | diverged | maxsteps | stalled | rejected
    steps: int                        # time steps over all stages
    steps_by_stage: List[int]
    residual: float
    arrival_s: float
    admit_s: float
    done_s: float
    nodes: int
    fields: Optional[tuple] = None    # (rho, ux, uy) host arrays of the final state

    @property
    def latency_s(self) -> float:
        """Time to steady state seen by the client: arrival to result."""
        return self.done_s - self.arrival_s

    @property
    def queue_s(self) -> float:
        return self.admit_s - self.arrival_s

    @property
    def service_s(self) -> float:
        return self.done_s - self.admit_s


@dataclass
class _Live:
    req: SolveRequest
    stage: int
    slot: int
    bytes: int
    admit_s: float
    steps_done: List[int] = field(default_factory=list)  # finished stages
    waiting_promotion: bool = False


class SolveServer:
    """Continuous batching of steady-state solves over one batch per stage.

    make_batch(capacity, dtype) -> Batch-like object (lbm.Batch on a GPU);
    instance_bytes(params, dtype) -> device bytes of one slot;
    staging(n_doubles) -> device pointer of a scratch buffer of at least
    n_doubles FP64 values (the promotion buffer; reused, grown on demand).
    Every batch must enqueue on the same stream so that the persistent
    launches of the stages run one after another.
    """

    def __init__(self, stages: Sequence[Stage], capacity: int, budget_bytes: int,
                 make_batch: Callable, instance_bytes: Callable, staging: Optional[Callable] = None,
                 chunk_node_steps: float = 4e9, max_chunk: int = 20000, keep_fields: bool = True,
                 clock: Callable[[], float] = time.monotonic, sleep: Callable[[float], None] = time.sleep):
        if not stages:
            raise ValueError("at least one stage")
        self.stages = list(stages)
        self.capacity = int(capacity)
        self.budget = int(budget_bytes)
        self.instance_bytes = instance_bytes
        self.staging = staging
        self.chunk_node_steps = float(chunk_node_steps)
        self.max_chunk = int(max_chunk)
        self.keep_fields = keep_fields
        self.clock, self.sleep = clock, sleep
        self.batches = [make_batch(self.capacity, st.dtype) for st in self.stages]
        self.used = 0
        self.staging_bytes = 0
        self.live = {}            # (stage, slot) -> _Live
        self.results = []
        self.launches = 0
        self.node_steps = 0

    # ------------------------------------------------------------------ sizes
    def _bytes(self, req: SolveRequest, stage: int) -> int:
        return int(self.instance_bytes(self._params(req, stage), self.stages[stage].dtype))

    def _params(self, req: SolveRequest, stage: int):
        p = type(req.params)()
        for name, _ in req.params._fields_:
            setattr(p, name, getattr(req.params, name))
        p.dtype = self.stages[stage].dtype
        return p

    def _staging_need(self, req: SolveRequest) -> int:
        return 9 * req.nodes * 8 if len(self.stages) > 1 else 0

    def _fits_ever(self, req: SolveRequest) -> bool:
        need = max(self._bytes(req, s) for s in range(len(self.stages)))
        return need + max(self.staging_bytes, self._staging_need(req)) <= self.budget

    def _free_slots(self, stage: int) -> int:
        return self.capacity - sum(1 for (s, _) in self.live if s == stage)

    # -------------------------------------------------------------- transitions
    def _add(self, req: SolveRequest, stage: int, steps_left: int) -> int:
        st = self.stages[stage]
        b = self.batches[stage]
        slot = b.add(self._params(req, stage), req.tol, steps_left)
        if st.stall_window > 0 and stage + 1 < len(self.stages):
            b.set_stall(slot, st.stall_window, st.stall_ratio)
        return slot

    def _admit(self, req: SolveRequest, now: float) -> bool:
        nb = self._bytes(req, 0)
        grow = max(0, self._staging_need(req) - self.staging_bytes)
        if self._free_slots(0) < 1 or self.used + nb + grow > self.budget:
            return False
        self.staging_bytes += grow
        self.used += grow
        slot = self._add(req, 0, req.max_steps)
        self.used += nb
        self.live[(0, slot)] = _Live(req, 0, slot, nb, now)
        return True

    def _promote(self, lv: _Live, steps_in_stage: int) -> bool:
        """Move a stalled solve to the next stage, on the device."""
        nxt = lv.stage + 1
        nb = self._bytes(lv.req, nxt)
        if self._free_slots(nxt) < 1 or self.used - lv.bytes + nb > self.budget:
            return False
        src = self.batches[lv.stage]
        ptr = self.staging(9 * lv.req.nodes)
        src.populations_to_device(lv.slot, ptr)
        src.remove(lv.slot)
        del self.live[(lv.stage, lv.slot)]
        self.used -= lv.bytes
        lv.steps_done.append(steps_in_stage)
        left = lv.req.max_steps - sum(lv.steps_done)
        slot = self._add(lv.req, nxt, max(1, left))
        self.batches[nxt].set_populations_from_device(slot, ptr)
        # narrow storage rounds every population and so lets the total mass
        # drift; a closed cavity conserves it exactly, and its steady state
        # depends on it: restore the request's initial mass
        self.batches[nxt].set_mass(slot, lv.req.mass0)
        self.used += nb
        lv.stage, lv.slot, lv.bytes, lv.waiting_promotion = nxt, slot, nb, False
        self.live[(nxt, slot)] = lv
        return True

    def _finish(self, lv: _Live, status: str, steps_in_stage: int, residual: float, now: float):
        b = self.batches[lv.stage]
        flds = b.fields(lv.slot) if self.keep_fields else None
        b.remove(lv.slot)
        del self.live[(lv.stage, lv.slot)]
        self.used -= lv.bytes
        steps = lv.steps_done + [steps_in_stage]
        self.results.append(SolveResult(lv.req.rid, status, sum(steps), steps, residual, lv.req.arrival_s,
                                        lv.admit_s, now, lv.req.nodes, flds))

    def _reject(self, req: SolveRequest, now: float):
        self.results.append(SolveResult(req.rid, "rejected", 0, [], math.inf, req.arrival_s, now, now, req.nodes))

    # ------------------------------------------------------------------- loop
    def _harvest(self, now: float):
        """Collect the slots that retired during the last launch."""
        for key in sorted(self.live):
            lv = self.live.get(key)
            if lv is None:
                continue
            b = self.batches[lv.stage]
            info, state = b.query(lv.slot)
            if state == SLOT_ACTIVE:
                continue
            last = lv.stage + 1 == len(self.stages)
            if state == SLOT_CONVERGED:
                self._finish(lv, "converged", int(info.step), float(info.residual), now)
            elif state == SLOT_DIVERGED:
                self._finish(lv, "diverged", int(info.step), float(info.residual), now)
            elif state == SLOT_MAXSTEPS:
                self._finish(lv, "maxsteps", int(info.step), float(info.residual), now)
            elif state == SLOT_STALLED and last:
                self._finish(lv, "stalled", int(info.step), float(info.residual), now)
            elif state == SLOT_STALLED:
                lv.waiting_promotion = True

    def _promotions(self):
        for key in sorted(self.live):
            lv = self.live.get(key)
            if lv is not None and lv.waiting_promotion:
                info, _ = self.batches[lv.stage].query(lv.slot)
                self._promote(lv, int(info.step))

    def _active_nodes(self) -> int:
        return sum(lv.req.nodes for lv in self.live.values() if not lv.waiting_promotion)

    def chunk_steps(self) -> int:
        n = max(1, self._active_nodes())
        k = int(self.chunk_node_steps / n)
        k = max(20, min(self.max_chunk, k))
        return (k + 19) // 20 * 20

    def serve(self, requests: Sequence[SolveRequest], time_limit_s: float = math.inf) -> List[SolveResult]:
        """Run until every request has a result (or time_limit_s passed: the
        solves still queued or resident are then reported unfinished)."""
        pending = deque(sorted(requests, key=lambda r: (r.arrival_s, r.rid)))
        t0 = self.clock()
        now = 0.0
        while pending or self.live:
            now = self.clock() - t0
            if now > time_limit_s:
                break
            self._promotions()
            while pending and pending[0].arrival_s <= now:
                req = pending[0]
                if not self._fits_ever(req):
                    pending.popleft()
                    self._reject(req, now)
                    continue
                if not self._admit(req, now):
                    break
                pending.popleft()
            running = [s for s in range(len(self.stages))
                       if any(k[0] == s and not lv.waiting_promotion for k, lv in self.live.items())]
            if not running:
                if pending:
                    self.sleep(max(0.0, pending[0].arrival_s - (self.clock() - t0)))
                    continue
                if self.live:  # only solves waiting for promotion: memory or slots are short
                    raise RuntimeError("promotion cannot proceed: budget or capacity too small")
                break
            k = self.chunk_steps()
            nodes = {s: sum(lv.req.nodes for key, lv in self.live.items() if key[0] == s and not lv.waiting_promotion)
                     for s in running}
            before = {key: self.batches[key[0]].query(key[1])[0].step for key, lv in self.live.items()
                      if not lv.waiting_promotion}
            for s in running:
                self.batches[s].launch(k)
            for s in running:
                self.batches[s].wait()
            self.launches += len(running)
            for key, t_before in before.items():
                info, _ = self.batches[key[0]].query(key[1])
                self.node_steps += (int(info.step) - int(t_before)) * self.live[key].req.nodes
            self._harvest(self.clock() - t0)
        self.wall_s = self.clock() - t0
        return self.results

    def close(self):
        for b in self.batches:
            b.close()


def percentile(xs: Sequence[float], q: float) -> float:
    """Nearest-rank percentile (q in [0, 100])."""
    if not xs:
        return math.nan
    s = sorted(xs)
    k = max(1, int(math.ceil(q / 100.0 * len(s))))
    return s[k - 1]


def summary(server: SolveServer, results: Sequence[SolveResult]) -> dict:
    done = [r for r in results if r.status != "rejected"]
    conv = [r for r in results if r.status == "converged"]
    lat = [r.latency_s for r in conv]
    return {
        "requests": len(results), "converged": len(conv),
        "by_status": {s: sum(1 for r in results if r.status == s)
                      for s in sorted(set(r.status for r in results))},
        "p50_time_to_steady_state_s": percentile(lat, 50), "p99_time_to_steady_state_s": percentile(lat, 99),
        "p50_service_s": percentile([r.service_s for r in conv], 50),
        "p99_service_s": percentile([r.service_s for r in conv], 99),
        "p50_queue_s": percentile([r.queue_s for r in done], 50),
        "aggregate_glups": server.node_steps / max(server.wall_s, 1e-12) / 1e9,
        "wall_s": server.wall_s, "launches": server.launches,
        "steps_p50": percentile([r.steps for r in conv], 50),
    }


class _TorchStaging:
    """Device FP64 promotion buffer from PyTorch's allocator, grown on demand."""

    def __init__(self):
        self.buf = None

    def __call__(self, n: int) -> int:
        import torch
        if self.buf is None or self.buf.numel() < n:
            self.buf = None
            self.buf = torch.empty(int(n), dtype=torch.float64, device="cuda")
        return self.buf.data_ptr()


def gpu_server(stages: Sequence[Stage], capacity: int = 256, budget_bytes: Optional[int] = None,
               reserve_bytes: int = 2 << 30, **kw) -> SolveServer:
    """A server on the current CUDA device: one lbm.Batch per stage, all on one
    PyTorch stream, memory budget = free device memory minus reserve_bytes
    unless budget_bytes is given."""
    import torch

    from . import lbm as L
    L.load()
    stream = torch.cuda.Stream()
    if budget_bytes is None:
        free, _ = torch.cuda.mem_get_info()
        budget_bytes = max(0, free - reserve_bytes)

    def make_batch(cap, dtype):
        return L.Batch(cap, dtype, stream.cuda_stream)

    def instance_bytes(p, dtype):
        p.dtype = dtype
        return L.lbm_batch_instance_bytes(p)

    srv = SolveServer(stages, capacity, budget_bytes, make_batch, instance_bytes, _TorchStaging(), **kw)
    srv.stream = stream
    return srv


def fp16_schedule(stall_window: int = 2000, stall_ratio: float = 0.9) -> List[Stage]:
    """FP16 shifted storage until the residual stalls, then FP32 to the tolerance."""
    return [Stage(2, stall_window, stall_ratio), Stage(1)]


def solve_promoted(nx: int, ny: int, r: float, gamma: float, nu: float, u_lid: float, tol: float,
                   max_steps: int, stall_window: int = 2000, stall_ratio: float = 0.9) -> dict:
    """One steady-state solve with the FP16 -> FP32 precision schedule on
    single-instance handles (the cluster engine for small grids): FP16
    storage until the residual stalls -- at a check `stall_window` steps
    after the previous one the residual is above `stall_ratio` times that
    one's -- then the state moves to an FP32 handle with the initial mass
    restored, which runs to `tol`.  The same rule as the batch's stall test,
    applied on the host between launches."""
    from . import lbm as L
    L.load()
    g = L.Lbm(L.lbm_params_init(nx, ny, r, gamma, nu, u_lid, L.F16))
    mass0 = float(nx * ny)  # the rest start
    steps16, prev, status = 0, None, None
    try:
        while steps16 < max_steps:
            st, n = g.run(tol, min(stall_window, max_steps - steps16))
            steps16 += n
            status = st
            if st == L.OK:
                break
            res = g.residual()
            if prev is not None and res > stall_ratio * prev:
                break  # stalled at the FP16 floor
            prev = res
    except L.LbmError as e:
        g.close()
        return {"status": "diverged" if e.status == L.EDIVERGED else "error", "steps": steps16,
                "steps_by_stage": [steps16, 0]}
    if status == L.OK:
        res = g.residual()
        g.close()
        return {"status": "converged", "steps": steps16, "steps_by_stage": [steps16, 0], "residual": res}
    f = g.populations()
    g.close()
    h = L.Lbm(L.lbm_params_init(nx, ny, r, gamma, nu, u_lid, L.F32))
    h.set_populations(f)
    h.set_mass(mass0)
    try:
        st, n = h.run(tol, max_steps - steps16)
    except L.LbmError as e:
        h.close()
        return {"status": "diverged" if e.status == L.EDIVERGED else "error", "steps": steps16,
                "steps_by_stage": [steps16, 0]}
    out = {"status": "converged" if st == L.OK else "not converged", "steps": steps16 + n,
           "steps_by_stage": [steps16, n], "residual": h.residual(), "fields": h.fields()}
    h.close()
    return out
