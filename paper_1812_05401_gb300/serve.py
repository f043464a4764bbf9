"""Continuous-batching serving loop over grouped VP-LBM launches.

Requests (inputs.Request: an arrival time and a workload) are admitted while
both a slot and device memory (vplbm_footprint_bytes against a budget) are
free, first come first served. Admitted solves stay resident on the device
and advance together: each round is one vplbm_group_step call in which every
active solve runs min(remaining, round_steps) steps, one grouped launch per
time step and storage/collision class. Requests that arrive while rounds are
on the GPU join at the next round boundary, so their work overlaps with the
solves already running. A finished solve's force series is read back and its
memory released once the GPU has completed its last round (CUDA event), which
is the request's completion time; latency = completion - arrival.

A request may carry a deadline (seconds after its arrival), and any thread may
cancel one (Server.cancel). A withdrawn request that is still waiting is
dropped; a running one stops at the next round boundary and is reported as
failed, with the force series of the steps it ran. run(log=...) writes one
JSON line per request: its result, or why it was rejected or dropped.

All solves share one CUDA stream (grouped launches require it). The host never
waits for the GPU except for the oldest round in flight: solver memory is
allocated and released stream-ordered, the initial field is generated on the
device, and a finished solve's force series is copied asynchronously into
page-locked memory behind its last round. Results do not depend on the mix:
the grouped kernel is the same code as the single-solver step, with
deterministic fixed-order reductions.
"""
from __future__ import annotations

import json
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import vplbm as V

SERVE_TILE_ROWS = 32


@dataclass
class Result:
    rid: int
    name: str
    arrival: float
    admitted: float
    finished: float
    steps: int               # steps run (fewer than requested for a solve stopped early)
    nodes: int
    storage: str
    collision: str
    fx: np.ndarray = field(repr=False, default=None)
    fy: np.ndarray = field(repr=False, default=None)
    populations: np.ndarray | None = field(repr=False, default=None)
    error: str | None = None  # set if the solve diverged or was stopped (results not valid)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Active:
    req: object
    solver: V.Solver
    remaining: int
    admitted: float
    footprint: int
    records: object = None  # pinned [steps][3] float64 tensor, filled behind the last round
    n_records: int = 0
    stopped: str | None = None  # why the solve was stopped before its last step


class Server:
    def __init__(self, budget_bytes: int, max_active: int = 256, round_steps: int = 500,
                 stream=None, keep_populations: bool = False, on_admit=None, clock=None):
        """on_admit(request, solver): optional hook called right after a solve is
        created (before its first step). clock: the time source (seconds),
        time.perf_counter by default."""
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.round_steps = int(round_steps)
        self.stream = stream or torch.cuda.Stream()
        self.keep_populations = keep_populations
        self.on_admit = on_admit
        self.clock = clock or time.perf_counter
        self.rejected = []
        self.errors = {}
        self.dropped = {}  # rid -> why a request was withdrawn before it ran
        self._cancelled = set()
        self._lock = threading.Lock()

    def cancel(self, rid: int):
        """Withdraws a request (from any thread): one still waiting is dropped,
        one running stops at the next round boundary and is reported as
        failed with the force series of the steps it ran."""
        with self._lock:
            self._cancelled.add(rid)

    def _create(self, w):
        # full-height tiles: a grouped launch of many solves already fills the
        # GPU, and taller tiles run the per-tile reduction less often
        cfg, bodies = V.config_from_workload(w, ring_len=max(1, w.steps), stream=self.stream,
                                             reduce_mass=False, tile_rows=SERVE_TILE_ROWS)
        u0 = (w.u_ref, 0.0) if w.bc == "channel" else (0.0, 0.0)
        s = V.Solver(cfg, bodies, perturbation=(u0[0], u0[1], w.perturbation, w.seed))
        return s, V.vplbm_footprint_bytes(cfg)

    def run(self, requests, realtime: bool = True, log=None):
        """Serves the requests; returns (results, report). With realtime=False
        every request counts as arrived at time 0. log: a text stream that
        gets one JSON line per request (its result, or why it was rejected or
        dropped)."""
        torch = self.torch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        active: list[_Active] = []
        inflight = deque()  # (event, [finished or stopped _Active])
        results = []
        used = 0
        t0 = self.clock()

        def now():
            return self.clock() - t0

        def arrived(req):
            return req.arrival if realtime else 0.0

        def withdrawn(req, t):
            with self._lock:
                if req.rid in self._cancelled:
                    return "cancelled"
            if req.deadline is not None and t - arrived(req) > req.deadline:
                return "deadline"
            return None

        def emit(rec):
            if log is not None:
                log.write(json.dumps(rec) + "\n")

        def read_back(a):
            """Copies the solve's force series behind its last queued round."""
            n = max(1, a.req.workload.steps - a.remaining)
            a.records = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
            a.n_records = V.vplbm_forces_async(a.solver.h, a.records.numpy())

        def retire(block: bool):
            nonlocal used
            while inflight and (block or inflight[0][0].query() or len(inflight) > 2):
                ev, fin = inflight.popleft()
                ev.synchronize()
                for a in fin:
                    rec = a.records.numpy()[:a.n_records]
                    fx, fy = rec[:, 0].copy(), rec[:, 1].copy()
                    pops = a.solver.populations() if self.keep_populations else None
                    err = None
                    try:  # the stream is past this solve's last round: no wait
                        a.solver.synchronize()
                    except V.VplbmError as e:  # this solve diverged; the others are unaffected
                        err = str(e)
                    w = a.req.workload
                    ran = w.steps - a.remaining
                    if a.stopped:
                        err = f"{a.stopped}: stopped after {ran} of {w.steps} steps" + (
                            f"; {err}" if err else "")
                    t_done = now()
                    r = Result(a.req.rid, w.name, arrived(a.req), a.admitted, t_done, ran,
                               w.nx * w.ny, w.storage, w.collision, fx, fy, pops, err)
                    results.append(r)
                    emit({"rid": r.rid, "name": r.name, "arrival": r.arrival,
                          "admitted": r.admitted, "finished": r.finished, "latency": r.latency,
                          "steps": r.steps, "nodes": r.nodes, "storage": r.storage,
                          "collision": r.collision, "error": r.error})
                    a.solver.close()
                    used -= a.footprint
                if not block and not inflight:
                    break

        while pending or active or inflight:
            t = now()
            # withdrawn solves stop at this round boundary, behind their queued rounds
            stop = []
            for a in active:
                a.stopped = withdrawn(a.req, t)
                if a.stopped:
                    read_back(a)
                    stop.append(a)
            if stop:
                ev = torch.cuda.Event()
                ev.record(self.stream)
                inflight.append((ev, stop))
                active = [a for a in active if not a.stopped]
            # admission: FIFO while a slot and memory are free
            while pending and (not realtime or pending[0].arrival <= t) and len(active) < self.max_active:
                req = pending[0]
                why = withdrawn(req, t)
                if why:
                    self.dropped[req.rid] = why
                    pending.popleft()
                    emit({"rid": req.rid, "name": req.workload.name, "arrival": arrived(req),
                          "dropped": why, "at": t})
                    continue
                cfg, _ = V.config_from_workload(req.workload, ring_len=max(1, req.workload.steps),
                                                tile_rows=SERVE_TILE_ROWS)
                fp = V.vplbm_footprint_bytes(cfg)
                if fp > self.budget:
                    self.rejected.append(req.rid)
                    pending.popleft()
                    emit({"rid": req.rid, "name": req.workload.name, "arrival": arrived(req),
                          "rejected": f"footprint {fp} bytes over the budget"})
                    continue
                if used + fp > self.budget:
                    break
                pending.popleft()
                try:
                    s, fp = self._create(req.workload)
                except V.VplbmError as e:  # e.g. out of device memory: refuse this request only
                    self.rejected.append(req.rid)
                    self.errors[req.rid] = str(e)
                    emit({"rid": req.rid, "name": req.workload.name, "arrival": arrived(req),
                          "rejected": str(e)})
                    continue
                if self.on_admit:
                    self.on_admit(req, s)
                used += fp
                active.append(_Active(req, s, req.workload.steps, now(), fp))
            if not active:
                if inflight:
                    retire(block=True)
                    continue
                if pending and realtime:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now())))
                continue
            steps = [min(a.remaining, self.round_steps) for a in active]
            V.vplbm_group_step([a.solver.h for a in active], steps)
            for a, k in zip(active, steps):
                a.remaining -= k
            done = [a for a in active if a.remaining == 0]
            for a in done:  # force series copied behind the solve's last round
                read_back(a)
            ev = torch.cuda.Event()
            ev.record(self.stream)
            active = [a for a in active if a.remaining > 0]
            inflight.append((ev, done))
            retire(block=False)
        retire(block=True)
        t_end = now()
        rep = self.report(results, t_end)
        rep["dropped"] = len(self.dropped)
        rep["stopped"] = sum(1 for r in results if r.error and r.error.startswith(
            ("deadline:", "cancelled:")))
        return results, rep

    @staticmethod
    def report(results, makespan: float):
        """Throughput and latency of the served solves: those that finished
        without an error. A solve that diverged or was stopped is counted in
        `failed` and in the GPU work figure `mlups_all`, but not in
        solves_per_s, the latency percentiles or `mlups`."""
        ok = [r for r in results if not r.error]
        lat = np.array([r.latency for r in ok]) if ok else np.full(1, np.nan)
        updates = float(sum(r.nodes * r.steps for r in ok))
        updates_all = float(sum(r.nodes * r.steps for r in results))
        return {
            "completed": len(results),
            "served": len(ok),
            "failed": len(results) - len(ok),
            "makespan_s": round(makespan, 3),
            "solves_per_s": round(len(ok) / makespan, 3) if makespan > 0 else None,
            "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
            "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
            "mlups": round(updates / makespan / 1e6, 1) if makespan > 0 else None,
            "mlups_all": round(updates_all / makespan / 1e6, 1) if makespan > 0 else None,
        }
