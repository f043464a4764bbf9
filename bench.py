"""Benchmark of the VP-LBM hot path on GB300.

Workload (default): the moving-cylinder channel, 16384 x 4096 D2Q9 MRT with
FP32 populations (67.1M nodes): a cylinder of D = 256 translating as
y(t) = y0 + 0.5 D sin(2 pi t / 20000), inlet u = 0.05, Re = 2000, free-slip
walls, zero-gradient outlet. One step = the mask/solid-velocity update over
the swept region plus the fused pull-penalize-collide-reduce kernel over every
node, i.e. every row of the hot path. The two population buffers (4.8 GB) are
far larger than L2, so no flush is needed between steps.

Output: one JSON line (rank 0). `value` is MLUPS (million node updates per
second) over all ranks; `e2e` repeats the measurement through the public API
with a host read of each step's force record; `roofline` relates the fused
kernel's algorithmic bytes (73 B per node update: 9 x 4 B read, 9 x 4 B
written, 1 B mask) to its CUDA-event duration; `cpu_baseline` times the FP64
oracle on a bounded sample of the same workload. `--impl reference` times only
the oracle (the reference arm).

Multi-GPU: the grid is not split (no halo exchange is built); every rank runs
its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CPU_WARMUP, CPU_STEPS = 5, 20  # the cpu_baseline leg's oracle sample (full grid)
ALGO_BYTES = {"f32": 73.0, "f16": 37.0, "bf16": 37.0, "f64": 145.0}  # per node update, u8 mask
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["paper_1812_05401_gb300/csrc/vplbm_device.cuh", "paper_1812_05401_gb300/csrc/vplbm_params.h",
                  "paper_1812_05401_gb300/csrc/vplbm_kernels_impl.cuh"]


def _code_only(text: str) -> str:
    """Kernel source without its comments and with runs of blank space made
    one space: an edit to a comment leaves the compiled kernel, and so its
    hash, unchanged. (No string literal in these sources holds // or /*.)"""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash() -> str:
    """Identifies the fused kernel's code (its comments aside); DRAM counters
    taken on another code are not reported as this kernel's traffic."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(_code_only(open(os.path.join(ROOT, f)).read()).encode())
    return h.hexdigest()[:16]


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        for k in ("hbm_gbs", "hbm_GBs", "copy_gbs"):
            if k in d and d[k]:
                return float(d[k]), "measured"
        if "hbm" in d and isinstance(d["hbm"], dict):
            for k in ("gbs", "GB/s", "value"):
                if k in d["hbm"]:
                    return float(d["hbm"][k]), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


def traffic_per_launch(workload: str, storage: str, streaming: str = "ab"):
    """DRAM bytes per fused launch from the committed ncu summary, if it was
    taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "fused_step_dram_moving_cylinder_16384x4096.json")
    try:
        d = json.load(open(p))
        e = d.get(f"{workload}:{storage}" + ("" if streaming == "ab" else f":{streaming}"))
        if e and e.get("kernel_hash") == kernel_hash():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def clocks_rejected(clk):
    """Why a timed region's clock record disqualifies it, else None: a
    hardware or thermal slowdown, or SM clocks well below their maximum with
    no reason reported (a clock lock left on the GPU). A power cap keeps the
    number (the record's reasons note it)."""
    if not clk:
        return None
    bad = [r for r in clk.get("reasons", [])
           if r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")]
    if bad:
        return "+".join(bad)
    if not clk.get("reasons") and clk["sm_mhz"] < 0.85 * clk["sm_max_mhz"]:
        return "SM clocks below 85% of their maximum with no reason reported"
    return None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_totals(units: float, ms: float, device=None):
    """Whole-job totals of independent replicas: the units all ranks processed
    (sum) and the slowest rank's time (max). Works on any initialised process
    group (NCCL with CUDA tensors, gloo with CPU tensors); without one it
    returns its inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(units), float(ms)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    m = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(u.item()), float(m.item())


def make_workload(name: str, storage: str):
    from paper_1812_05401_gb300 import inputs as I
    makers = {"moving-cylinder": I.c5_moving_cylinder, "cylinder-re1000": I.c3_cylinder_re1000,
              "cylinder-re100": I.c2_cylinder_re100, "circular-couette": I.c1_circular_couette}
    if name not in makers:
        raise ValueError(name)
    w = makers[name]()
    w.storage = storage
    return w


# -----------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the workload
# -----------------------------------------------------------------------------

def oracle_rates(budget_s: float = 8.0):
    """The FP64 oracle's rate on the host cores for each configuration at its
    full grid size (C1 Couette, C2 and C3 cylinders, C5 moving cylinder), with
    one thread and with every core: after one untimed step (which also sizes
    the sample), the steps that fit in about budget_s seconds, timed as one
    call (as the cpu_baseline leg and the reference arm time it). Prints one
    JSON line."""
    import oracle as O
    from paper_1812_05401_gb300 import inputs as I
    out = {"kind": "oracle", "nproc": os.cpu_count(), "budget_s_per_rate": budget_s, "configs": {}}
    for name, w in (("C1", I.c1_circular_couette()), ("C2", I.c2_cylinder_re100()),
                    ("C3", I.c3_cylinder_re1000("f32")), ("C5", I.c5_moving_cylinder("f32"))):
        cfg = oracle_config(w)
        f = O.init_equilibrium(cfg, 1.0, None)
        rates = {}
        for threads in (1, 0):
            O.set_num_threads(threads)
            t0 = time.perf_counter()
            O.run(cfg, f, 1)
            steps = max(2, int(budget_s / max(time.perf_counter() - t0, 1e-6)))
            t0 = time.perf_counter()
            O.run(cfg, f, steps, t0=1)
            dt = time.perf_counter() - t0
            rates["1_thread" if threads == 1 else f"{O.num_threads()}_threads"] = {
                "mlups": round(w.nx * w.ny * steps / dt / 1e6, 3), "steps": steps,
                "seconds": round(dt, 2)}
        O.set_num_threads(0)
        out["configs"][name] = {"workload": w.name, "nodes": w.nx * w.ny, **rates}
        del f
    print(json.dumps(out), flush=True)


def oracle_config(w):
    """The oracle's configuration of a workload (full grid, same physics)."""
    import oracle as O
    tau = O.tau_from_reynolds(w.u_ref, w.l_ref, w.re) if w.re else w.tau
    chan = w.bc == "channel"
    return O.Config(nx=w.nx, ny=w.ny, collision=O.MRT if w.collision == "mrt" else O.SRT, tau=tau,
                    lam=w.lam, bc_x=O.BC_INLET_OUTLET if chan else O.BC_PERIODIC,
                    bc_y=O.BC_FREE_SLIP if chan else O.BC_PERIODIC,
                    u_in=(w.u_ref, 0.0) if chan else (0.0, 0.0),
                    bodies=[O.Body(b.cx, b.cy, b.radius, b.amp_x, b.amp_y, b.period, b.omega,
                                   b.outside) for b in w.bodies])


def oracle_full(w, warmup: int, steps: int):
    """Times the FP64 oracle on the workload's full grid, on every host core:
    `warmup` untimed steps, then `steps` timed steps in one call. Returns
    (MLUPS, steps, seconds, threads)."""
    import oracle as O
    cfg = oracle_config(w)
    f = O.init_equilibrium(cfg, 1.0, w.initial_velocity())
    if warmup:
        O.run(cfg, f, warmup)
    t0 = time.perf_counter()
    O.run(cfg, f, steps, t0=warmup)
    dt = time.perf_counter() - t0
    return w.nx * w.ny * steps / dt / 1e6, steps, dt, O.num_threads()


def device_l2_bytes() -> int:
    """L2 size of GPU 0 from its device properties (0 without a GPU)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(getattr(torch.cuda.get_device_properties(0), "L2_cache_size", 0))
    except Exception:
        pass
    return 0


def l2_residency(nodes: int, storage: str, streaming: str, l2_bytes: int):
    """(cache_resident, note): whether the population buffers fit in L2, and
    the line's statement of it (inputs larger than L2 need no flush)."""
    esize = {"f32": 4, "f16": 2, "bf16": 2, "f64": 8}[storage]
    pop_bytes = (2 if streaming == "ab" else 1) * 9 * nodes * esize
    if pop_bytes < l2_bytes:
        return True, ("inputs fit in L2 (%.0f MB): population buffers of %.1f MB, cache-resident, "
                      "so the roofline fraction is not a DRAM figure" % (l2_bytes / 1e6, pop_bytes / 1e6))
    return False, "inputs larger than L2 (%.0f MB): %s population buffer%s of %.2f GB" % (
        l2_bytes / 1e6, "two" if streaming == "ab" else "one in-place",
        "s" if streaming == "ab" else "", 9 * nodes * esize / 1e9)


def workload_config(w, storage: str, streaming: str, world: int, l2_note: str | None = None):
    """The `config` object of the JSON line (both arms)."""
    return {"workload": w.name + f" {w.collision.upper()} {storage.upper()}",
            "nx": w.nx, "ny": w.ny, "nodes": w.nx * w.ny, "storage": storage,
            "collision": w.collision, "re": w.re, "u_in": w.u_ref,
            "step": "mask update of the moving body + fused pull/penalize/collide/reduce kernel",
            "streaming": streaming,
            **({"l2": l2_note} if l2_note else {}),
            "parallelism": f"replicas x{world}"}


# -----------------------------------------------------------------------------
# GPU arm
# -----------------------------------------------------------------------------

def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1812_05401_gb300 import vplbm as V

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return replica_totals(0.0, x, dev)[1]

    w = make_workload(args.workload, args.storage)
    nodes = w.nx * w.ny
    s = V.Solver.from_workload(w, stream=stream, ring_len=max(4096, args.steps + 16),
                               streaming=args.streaming)
    try:
        # warm-up
        s.step(args.warmup)
        s.synchronize()
        s.forces()

        # ---- device-resident timed region ------------------------------------
        def timed_region():
            V.vplbm_enable_timing(s.h, True)
            V.vplbm_fused_timing(s.h)  # reset
            clocks = ClockSampler(local)
            clocks.start()
            time.sleep(0.3)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            barrier()
            torch.cuda.synchronize()
            l0 = s.launches
            with torch.cuda.stream(stream):
                e0.record(stream)
            s.step(args.steps)
            with torch.cuda.stream(stream):
                e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            launches = s.launches - l0
            ms = e0.elapsed_time(e1)
            clk = clocks.stop()
            s.synchronize()  # raises if the run diverged
            fused_ms, fused_n = V.vplbm_fused_timing(s.h)
            V.vplbm_enable_timing(s.h, False)
            return ms, launches, clk, fused_ms, fused_n

        ms, launches, clk, fused_ms, fused_n = timed_region()
        why = clocks_rejected(clk)
        if max_over_ranks(1.0 if why else 0.0) > 0:  # every rank re-measures, once
            first = clk
            ms, launches, clk, fused_ms, fused_n = timed_region()
            if clk is not None:
                clk = dict(clk, remeasured=why or "another rank's clocks", first_run=first)
        units, ms = replica_totals(nodes * args.steps, ms, dev)
        value = units / (ms / 1e3) / 1e6

        # ---- end to end through the public API: each step's force record is
        # read back to the host (synchronizing), the body state goes in as the
        # launch parameters of the step.
        s.forces()
        e_steps = max(3, args.steps // 2)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            s.step(1)
            fx, fy, ms_ = s.forces(cap=1)
        torch.cuda.synchronize()
        barrier()
        e_units, e_ms = replica_totals(nodes * e_steps, (time.perf_counter() - t0) * 1e3, dev)
        e2e = e_units / (e_ms / 1e3) / 1e6
    finally:
        s.close()

    # ---- the same workload in another storage or streaming scheme (side
    # measurements: FP16-offset store, in-place AA streaming)
    def side_run(storage, streaming):
        ws = make_workload(args.workload, storage)
        s2 = V.Solver.from_workload(ws, stream=stream, ring_len=4096, streaming=streaming)
        try:
            s2.step(args.warmup)
            s2.synchronize()
            V.vplbm_enable_timing(s2.h, True)
            V.vplbm_fused_timing(s2.h)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                a0.record(stream)
            s2.step(args.steps)
            with torch.cuda.stream(stream):
                a1.record(stream)
            torch.cuda.synchronize()
            s2.synchronize()
            ms2 = max_over_ranks(a0.elapsed_time(a1))
            k2, n2 = V.vplbm_fused_timing(s2.h)
            cfg2, _ = V.config_from_workload(ws, streaming=streaming)
            foot = V.vplbm_footprint_bytes(cfg2)
        finally:
            s2.close()
        peak, _ = hbm_peak()
        kms2 = k2 / max(n2, 1)
        ach = ALGO_BYTES[storage] * nodes / (kms2 / 1e3) / 1e9
        return {"value": round(world * nodes * args.steps / (ms2 / 1e3) / 1e6, 1),
                "unit": "MLUPS", "fused_kernel_ms": round(kms2, 4),
                "achieved_gbs": round(ach, 1), "frac": round(ach / peak, 4),
                "algo_bytes_per_node": ALGO_BYTES[storage], "footprint_gb": round(foot / 1e9, 3)}

    extra = {}
    if args.compare_f16 and args.storage == "f32":
        extra["f16_offset_store"] = side_run("f16", args.streaming)
        extra["bf16_offset_store"] = side_run("bf16", args.streaming)
    if args.precision:
        extra["precision_vs_oracle"] = precision_record()
    if args.compare_aa and args.storage == "f32" and args.streaming == "ab":
        extra["aa_inplace"] = side_run("f32", "aa")

    if args.serve_in_bench:
        rep = run_serving(args, n_requests=args.serve_requests, rate=args.serve_rate_bench,
                          quiet=True)
        extra["serving"] = rep
        # the FP16-offset store against the plain FP32 store on the same
        # requests: closed-loop capacity, then latency under Poisson arrivals,
        # and each cylinder request's mean drag coefficient in the two forms
        served = {}
        for st in ("f32", "f16"):
            cap = run_serving(args, n_requests=args.serve_requests_storage, rate=0.0, storage=st,
                              quiet=True)
            rep, res = run_serving(args, n_requests=args.serve_requests_storage,
                                   rate=args.serve_rate_bench, storage=st, quiet=True,
                                   want_results=True)
            served[st] = res
            extra[f"serving_{st}"] = {**rep, "capacity_solves_per_s": cap["solves_per_s"],
                                      "capacity_mlups": cap["mlups"]}
        extra["serving_f16_vs_f32_drag"] = drag_agreement(
            args, served["f32"], served["f16"], n_requests=args.serve_requests_storage)

    peak, peak_src = hbm_peak()
    l2_bytes = device_l2_bytes()
    resident, l2_note = l2_residency(nodes, args.storage, args.streaming, l2_bytes)
    kms = fused_ms / max(fused_n, 1)
    achieved = ALGO_BYTES[args.storage] * nodes / (kms / 1e3) / 1e9
    traffic = traffic_per_launch(args.workload, args.storage, args.streaming)
    result = {
        "metric": "VP-LBM MLUPS (node updates per second / 1e6)",
        "value": round(value, 1),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.storage != "f64" else "f64",
        "data": "synthetic",
        "config": workload_config(w, args.storage, args.streaming, world, l2_note),
        "e2e": {"value": round(e2e, 1), "unit": "MLUPS", "h2d_bytes_per_step": 704,
                "d2h_bytes_per_step": 24,
                "note": "public API per step: vplbm_step(1) then vplbm_forces (synchronizing read of F_x, F_y, mass)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": f"{peak_src} copy bandwidth",
                     "kernel": f"fused_step_kernel<{args.storage.upper()},{w.collision.upper()}>" + (
                         "" if args.streaming == "ab" else " (in place: push and local steps)"),
                     "kernel_ms": round(kms, 4), "algo_bytes_per_node": ALGO_BYTES[args.storage],
                     "algo_bytes_per_launch": ALGO_BYTES[args.storage] * nodes,
                     "cache_resident": resident},
        "gpu_launches": launches,
        "clocks": clk,
    }
    result.update(extra)
    if rank == 0 and not args.no_cpu_baseline:
        # the reference arm's sample at the driver's --steps 20 --warmup 5
        mlups, n, dt, cores = oracle_full(w, warmup=CPU_WARMUP, steps=CPU_STEPS)
        result["cpu_baseline"] = {
            "value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle on the full {w.nx}x{w.ny} grid of this workload, {n} timed "
                      f"steps after {CPU_WARMUP}, {dt:.1f} s, {cores} threads of {os.cpu_count()} "
                      f"processors"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def precision_record():
    """Wake statistics of each storage form against the FP64 oracle's (the
    Re = 100 cylinder channel, 1024 x 256, MRT; the oracle's values are the
    stored ones its own run wrote, tests/golden/c2_wake_statistics.json). The
    FP64 path develops the wake over the oracle's development steps; FP32 and
    the 16-bit offsets (stochastic rounding, four realizations: rounding seeds
    0..3) then record the oracle's window from that state. For each storage:
    the largest relative error of C_Dave, St and C_Lrms over its realizations,
    the relative error of the realizations' mean statistics, and whether every
    realization is within the 1e-3 bar on C_Dave and St."""
    import torch

    from paper_1812_05401_gb300 import diag
    from paper_1812_05401_gb300 import inputs as I
    from paper_1812_05401_gb300 import vplbm as V
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "c2_wake_statistics.json")))
    dev, meas = g["develop_steps"], g["measure_steps"]
    keys = ("C_D_ave", "C_L_rms", "St")
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    w = I.c2_cylinder_re100()
    w.storage = "f64"
    with V.Solver.from_workload(w, stream=stream, ring_len=16, reduce_mass=False) as s:
        s.step(dev)
        s.synchronize()
        f0 = s.populations()
    out = {"workload": w.name + " MRT", "window_steps": meas, "bar": 1e-3,
           "reference": "FP64 oracle statistics (stored)"}
    for st in ("f32", "f16", "bf16"):
        w.storage = st
        runs = []
        for seed in ((0,) if st == "f32" else (0, 1, 2, 3)):
            with V.Solver.from_workload(w, stream=stream, ring_len=meas, reduce_mass=False,
                                        with_initial_velocity=False, rounding_seed=seed) as s:
                s.set_populations(f0)
                s.step(meas)
                s.synchronize()
                fx, fy, _ = s.forces()
            runs.append(diag.wake_statistics(fx, fy, w.u_ref, w.l_ref, discard=0.0))
        worst = {k: max(abs(r[k] - g[k]) / abs(g[k]) for r in runs) for k in keys}
        mean = {k: (sum(r[k] for r in runs) / len(runs) - g[k]) / abs(g[k]) for k in keys}
        out[st] = {"realizations": len(runs),
                   "C_D_ave_rel_err": float(f"{worst['C_D_ave']:.3g}"),
                   "St_rel_err": float(f"{worst['St']:.3g}"),
                   "C_L_rms_rel_err": float(f"{worst['C_L_rms']:.3g}"),
                   "mean_C_D_ave_rel_err": float(f"{mean['C_D_ave']:.3g}"),
                   "mean_St_rel_err": float(f"{mean['St']:.3g}"),
                   "within_bar": bool(worst["C_D_ave"] < 1e-3 and worst["St"] < 1e-3)}
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


def run_serving_passes(args):
    """Closed-loop capacity, then Poisson arrivals at 0.8 x capacity, for the
    mixed storage and for all-FP32 and all-FP16 requests."""
    out, served = {}, {}
    for st in (None, "f32", "f16"):
        cap, res = run_serving(args, rate=0.0, storage=st, quiet=True, want_results=True)
        served[st] = res
        rate = round(0.8 * cap["solves_per_s"], 2)
        rep = run_serving(args, rate=rate, storage=st, quiet=True)
        out[st or "mixed"] = {"capacity_solves_per_s": cap["solves_per_s"], "capacity_mlups": cap["mlups"],
                              "at_0.8_capacity": rep}
    out["fp16_vs_fp32_drag"] = drag_agreement(args, served["f32"], served["f16"])
    print(json.dumps({"metric": "served solves/s and p50/p99 latency (VP-LBM serving mix)",
                      "serving": out}), flush=True)


def drag_agreement(args, res32, res16, n_requests=None):
    """Mean drag coefficient (second half of each run) of every cylinder
    request served with FP16-offset storage against the same request served
    with FP32 storage; requests that diverged in either pass are left out.
    Reported for all cylinder requests and for those below the onset of
    vortex shedding (Re < 47), which reach a steady drag: a short run above
    it averages over a wake whose shedding onset any perturbation -- rounding
    noise of either storage included -- moves."""
    import numpy as np

    from paper_1812_05401_gb300 import diag
    from paper_1812_05401_gb300 import inputs as I
    reqs = {r.rid: r.workload for r in I.serving_mix(n_requests or args.serve_requests, rate=1.0,
                                                        seed=1234)}
    a = {r.rid: r for r in res32 if not r.error}
    b = {r.rid: r for r in res16 if not r.error}
    rel, steady = [], []
    for rid in sorted(set(a) & set(b)):
        w = reqs[rid]
        if "cylinder" not in w.name:
            continue
        cd = []
        for r in (a[rid], b[rid]):
            c, _ = diag.coefficients(r.fx, r.fy, w.u_ref, w.l_ref)
            cd.append(float(np.mean(c[len(c) // 2:])))
        d = abs(cd[1] - cd[0]) / abs(cd[0])
        rel.append(d)
        if w.re < 47.0:
            steady.append(d)

    def summary(x):
        x = np.array(x)
        if x.size == 0:
            return {"requests": 0}
        return {"requests": int(x.size), "cd_rel_diff_median": float(np.median(x)),
                "cd_rel_diff_max": float(x.max()), "within_1e-3": int((x <= 1e-3).sum())}
    return {"steady_re_below_47": summary(steady), "all_cylinder_requests": summary(rel)}


def run_serving(args, n_requests=None, rate=None, storage=None, quiet=False, want_results=False):
    """The serving mix (Poisson arrivals; Couette or cylinder channel 50/50;
    side log-uniform in 64..1024; Re in 20..500; SRT/MRT 50/50; 2000..20000
    steps; FP32 or FP16-offset storage) through the continuous-batching
    server. rate = 0: every request arrives at t = 0 (closed loop, capacity)."""
    import torch

    from paper_1812_05401_gb300 import inputs as I
    from paper_1812_05401_gb300 import serve
    n = n_requests or args.serve_requests
    rate = args.serve_rate if rate is None else rate
    reqs = I.serving_mix(n, rate=rate if rate > 0 else 1.0, seed=1234, storage=storage)
    if rate <= 0:
        for r in reqs:
            r.arrival = 0.0
    free, total = torch.cuda.mem_get_info()
    srv = serve.Server(budget_bytes=int(0.5 * free), max_active=args.serve_slots,
                       round_steps=args.serve_round)
    torch.cuda.synchronize()
    log = open(args.serve_log, "a") if args.serve_log else None
    try:
        results, rep = srv.run(reqs, realtime=rate > 0, log=log)
    finally:
        if log:
            log.close()
    rep.update({"requests": n, "arrival_rate_per_s": rate if rate > 0 else "all at t=0",
                "storage": storage or "f32/f16 50-50", "budget_bytes": int(0.5 * free),
                "slots": args.serve_slots, "round_steps": args.serve_round,
                "rejected": len(srv.rejected)})
    if not quiet:
        print(json.dumps({"metric": "served solves/s (VP-LBM serving mix)", "serving": rep}), flush=True)
    return (rep, results) if want_results else rep


def run_grouped(args):
    """Grouped-launch throughput by grid size (the serving kernel): for each
    side s, a batch of k cylinder channels of 4s x s nodes (k s.t. the batch
    holds ~16M nodes; diameter 40 s / 256, Re 200, FP32, SRT and MRT
    alternating, the server's tile height) advanced by vplbm_group_step; CUDA
    events around `steps` grouped steps after 20 untimed ones. Prints one JSON
    line."""
    import torch

    from paper_1812_05401_gb300 import inputs as I
    from paper_1812_05401_gb300 import vplbm as V
    from paper_1812_05401_gb300.serve import SERVE_TILE_ROWS
    stream = torch.cuda.Stream()
    rows = []
    for side in args.grouped:
        nx, ny = 4 * side, side
        k = max(1, (16 << 20) // (nx * ny))
        solvers = []
        try:
            for i in range(k):
                w = I.cylinder_channel(nx, ny, max(4.0, round(40 * side / 256)), 0.05, 200.0, 0,
                                       storage="f32", seed=i + 1)
                w.collision = "mrt" if i % 2 else "srt"
                solvers.append(V.Solver.from_workload(w, stream=stream, ring_len=args.steps + 32,
                                                      tile_rows=SERVE_TILE_ROWS))
            hs = [x.h for x in solvers]
            V.vplbm_group_step(hs, [20] * k)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
            V.vplbm_group_step(hs, [args.steps] * k)
            with torch.cuda.stream(stream):
                e1.record(stream)
            torch.cuda.synchronize()
            for x in solvers:
                x.synchronize()  # raises if a solve diverged
            ms = e0.elapsed_time(e1)
            rows.append({"grid": f"{nx}x{ny}", "solves": k, "nodes": k * nx * ny,
                         "steps": args.steps, "ms_per_step": round(ms / args.steps, 4),
                         "mlups": round(k * nx * ny * args.steps / (ms / 1e3) / 1e6, 1)})
        finally:
            for x in solvers:
                x.close()
    print(json.dumps({"metric": "grouped-launch MLUPS by grid size (FP32 cylinder channels, "
                                "SRT/MRT alternating, ~16M nodes per batch)", "unit": "MLUPS",
                      "grouped": rows}), flush=True)


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, on the same workload
    at its full grid size. One step = one oracle step of the whole grid; W
    untimed steps, then K timed steps."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = make_workload(args.workload, args.storage)
    value, n, dt, cores = oracle_full(w, warmup=args.warmup, steps=args.steps)
    desc = (f"FP64 oracle on the full {w.nx}x{w.ny} grid of this workload, {n} timed steps "
            f"after {args.warmup}, {dt:.1f} s, {cores} threads of {os.cpu_count()} processors")
    out = {"impl": "reference", "metric": "VP-LBM MLUPS (node updates per second / 1e6)",
           "value": round(value, 3), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(dt / n * 1e3, 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": workload_config(w, args.storage, args.streaming, world, l2_residency(
               w.nx * w.ny, args.storage, args.streaming, device_l2_bytes())[1]),
           "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": cores,
                            "kind": "oracle", "sample": desc},
           "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="moving-cylinder",
                    choices=["moving-cylinder", "cylinder-re1000", "cylinder-re100",
                             "circular-couette"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "f64"])
    ap.add_argument("--no-compare-f16", dest="compare_f16", action="store_false")
    ap.add_argument("--no-compare-aa", dest="compare_aa", action="store_false",
                    help="skip the in-place (AA) streaming side measurement")
    ap.add_argument("--streaming", default="ab", choices=["ab", "aa"],
                    help="streaming scheme of the headline run (A/B buffers or in place)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", dest="precision", action="store_false",
                    help="skip the storage forms' wake statistics against the oracle's")
    ap.add_argument("--serving", action="store_true", help="run only the serving mix")
    ap.add_argument("--oracle-rates", action="store_true",
                    help="time the FP64 oracle (CPU baseline) on every configuration, 1 thread and all cores")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-requests-storage", type=int, default=128,
                    help="requests of each all-FP32 and all-FP16 serving pass in the default run")
    ap.add_argument("--serve-rate", type=float, default=0.0)
    ap.add_argument("--serve-slots", type=int, default=256)
    ap.add_argument("--no-serving", dest="serve_in_bench", action="store_false",
                    help="skip the serving measurement in the default run")
    ap.add_argument("--serve-rate-bench", type=float, default=8.2,
                    help="Poisson arrival rate of the serving measurement in the default run "
                         "(0.8 x the measured closed-loop capacity of 10.2 solves/s)")
    ap.add_argument("--serve-round", type=int, default=500)
    ap.add_argument("--serve-log", default=None, metavar="PATH",
                    help="append one JSON line per served request (result, rejection or drop)")
    ap.add_argument("--grouped", type=lambda v: [int(x) for x in v.split(",")], default=None,
                    metavar="S1,S2,...",
                    help="grouped-launch throughput for batches of 4S x S channels (serving "
                         "kernel), timed over --steps grouped steps (e.g. --steps 200)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.oracle_rates:
        oracle_rates()
    elif args.impl == "reference":
        run_reference(args)
    else:
        from paper_1812_05401_gb300 import build as B
        if not B.up_to_date():
            B.build()
        if args.serving:
            run_serving_passes(args)
        elif args.grouped:
            run_grouped(args)
        else:
            run_gpu(args)


if __name__ == "__main__":
    main()
