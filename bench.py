"""Benchmark of the GB300 flood-model step: Gcell-updates/s and HBM roofline.

Default workload: the 16384 x 16384 single-grid step (268 M cells, FP32
state h, qx, qy with DEM z and Manning n, ~5.4 GB resident, far larger than
the 129 MB L2), fractal terrain with a carved channel, two inflow sections and
an outflow edge, primed to ~30 % wet.  One benchmark "step" is one time step
of the whole grid: epoch bookkeeping (CFL dt, Eq. 6 inflow) when due, the
face update (Eq. 3), depth update (Eq. 4), boundary faces and ledgers.  The
default kernel is the temporal-blocking one (4 steps per launch, the
library's AUTO choice for this grid); the one-step stream kernel is timed
beside it (`one_step`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle (the
independent definition used by the tests) on the host cores over a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_CELL = 32          # read h, qx, qy, z, n (20 B) + write h, qx, qy (12 B), FP32
# DRAM bytes read + written per cell by one launch of a kernel on the 16384^2
# workload, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of a
# smaller case of the same workload (state > L2) in the same launch shape, scaled by
# the cell count; key (kernel, steps per launch).  Stream kernel: the 4096^2 case in
# the 4 warps x 32-row chunks of the 16384^2 launch.  Temporal-blocking kernel: the
# 8192^2 case with the 304-row (chunk, strip) items the 16384^2 launch takes from its
# counter (--tile 0,304).  Only kernels whose code has not changed since their capture
# are listed; the others report traffic null.
TRAFFIC_B_PER_CELL = {("stream", 1): 31.32, ("tiled", 4): 32.29}
# Warp instructions per cell-update of the temporal-blocking kernel (issue-bound), from the same
# capture (smsp__inst_executed.sum): the "alu" roofline beside the one-step HBM one.  The issue peak is
# 152 SMs x 4 warp-instructions per cycle x the sampled SM clock.
INST_PER_CELL_UPDATE = {("tiled", 4): 907034250 / (8192 * 8192 * 4)}
SMS, ISSUE_PER_SM_CYCLE = 152, 4
# the same two for the vector-norm friction option (theta = 1)
TRAFFIC_VEC_B_PER_CELL = {("tiled", 4): 32.27}
INST_VEC_PER_CELL_UPDATE = {("tiled", 4): 1117140607 / (8192 * 8192 * 4)}
METRIC = "Gcell-updates/s and % of HBM roofline (FP32, 1 GB300); adjoint/forward time ratio"
UNIT = "Gcell-updates/s"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload(name: str):
    import inputs
    if name == "c3":
        return inputs.c3_large(), "fractal_16384x16384_1m_two_inflows_fp32"
    if name == "c2":
        return inputs.c2_fractal(), "fractal_2048x2048_5m_fp32"
    if name.startswith("c3:"):
        n = int(name.split(":")[1])
        return inputs.c3_large(nx=n, ny=n), f"fractal_{n}x{n}_1m_two_inflows_fp32"
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, power, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int = 0):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_strip(prob, rows: int = 1024):
    """The FP64 oracle on a full-width strip of the workload's first `rows` rows
    (the x-side boundary sections re-expressed for the strip)."""
    import oracle
    from inputs import Problem, Section
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    rows = max(16, min(prob.ny, rows))
    sub = Problem(prob.name + "_strip", prob.nx, rows, prob.dx, prob.z[:rows].copy(), prob.n[:rows].copy(),
                  [s for s in prob.sections if s.side in (0, 1)], prob.opts,
                  h0=None if prob.h0 is None else prob.h0[:rows].copy())
    secs = []
    for s in sub.sections:
        a, b = int(np.floor(s.frac_start * prob.ny + 0.5)), int(np.floor(s.frac_end * prob.ny + 0.5))
        a, b = min(a, rows), min(b, rows)
        if b > a:
            secs.append(Section(s.side, a / rows, b / rows, s.kind, s.slope, s.t_s, s.q_m3s))
    sub.sections = secs
    return oracle.Oracle(sub), sub, threads


def _oracle_rate(o, sub, seconds: float, min_steps: int = 1, max_steps: int = 10 ** 9):
    """Gcell-updates/s of the oracle on `sub`: steps until `seconds` have passed."""
    o.run(1)                      # warm (page-in)
    steps, elapsed = 0, 0.0
    while (elapsed < seconds or steps < min_steps) and steps < max_steps:
        t0 = time.perf_counter()
        o.run(1)
        elapsed += time.perf_counter() - t0
        steps += 1
    return sub.nx * sub.ny * steps / elapsed / 1e9, steps, elapsed


def cpu_baseline(prob, seconds_target: float = 10.0):
    """The FP64 oracle on the host cores: all cores on a bounded sample of the
    workload (a full-width strip of the grid), beside it one core on the same
    strip, and the 2048^2 workload over 100 steps on all cores and on one core
    (the per-core figure the paper's CPU column reports, Table 1)."""
    import inputs
    import oracle
    o, sub, threads = oracle_strip(prob)
    v, steps, el = _oracle_rate(o, sub, seconds_target)
    out = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"FP64 C oracle, {sub.nx}x{sub.ny} full-width strip of the workload, {steps} steps, "
                     f"{el:.1f} s, OpenMP {threads} threads", "more": []}
    oracle.set_threads(1)
    o1, sub1, _ = oracle_strip(prob)
    oracle.set_threads(1)
    v1, steps1, el1 = _oracle_rate(o1, sub1, seconds_target / 3)
    out["more"].append({"workload": f"{sub1.nx}x{sub1.ny} strip", "threads": 1, "steps": steps1,
                        "seconds": round(el1, 2), "value": v1})
    c2 = inputs.c2_fractal()
    c2.h0 = inputs.wet_start(c2.z, c2.dx, 0.3)
    for t, cap in ((threads, 100), (1, 100)):
        oracle.set_threads(t)
        oc = oracle.Oracle(c2)
        vc, sc, ec = _oracle_rate(oc, c2, 0.0, min_steps=cap, max_steps=cap)
        out["more"].append({"workload": "fractal_2048x2048_5m (30 % wet)", "threads": t, "steps": sc,
                            "seconds": round(ec, 2), "value": vc})
    oracle.set_threads(threads)
    return out


def run_reference(args):
    """The oracle as the reference arm: W warm-up and K timed steps, each one time
    step of a 1024-row full-width strip of the same workload on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prob, wname = workload(args.workload)
    o, sub, threads = oracle_strip(prob)
    warm = max(3, args.warmup)
    o.run(warm)
    t0 = time.perf_counter()
    o.run(args.steps)
    elapsed = time.perf_counter() - t0
    cells = sub.nx * sub.ny
    value = cells * args.steps / elapsed / 1e9
    sample = (f"FP64 C oracle, {sub.nx}x{sub.ny} full-width strip of the workload per step, {warm} warm-up + "
              f"{args.steps} timed steps, {elapsed:.1f} s, OpenMP {threads} threads; ms_per_step scaled to the "
              f"{prob.nx}x{prob.ny} grid")
    cb = {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": warm, "ms_per_step": prob.nx * prob.ny / (value * 1e9) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "nx": prob.nx, "ny": prob.ny, "sample": sample},
            "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def max_over_ranks(ms: float, dist) -> float:
    """The slowest rank's time (all ranks get it); ms itself without a process group."""
    if not dist:
        return ms
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, cells: int, steps: int, ms: float) -> float:
    """Whole-job Gcell-updates/s of `world` replicas of `cells` cells over `steps` steps in ms."""
    return world * cells * steps / (ms * 1e-3) / 1e9


def timed_run(F, torch, prob, kernel_name, k, tile, graph, steps_req, warmup, local, dist, repeats=5):
    """Warm up, then time `repeats` runs of exactly steps_req steps of one kernel
    on `prob`, each bracketed by a barrier and a synchronize: CUDA events around
    every launch on the library's stream, nvidia-smi clocks sampled meanwhile.
    The runs continue one simulation (a run may start and end inside a CFL
    epoch; its epoch starts are timed with it).  total_ms is the median run."""
    kernel = {"rows": F.KERNEL_ROWS, "tiled": F.KERNEL_TILED, "reference": F.KERNEL_REFERENCE,
              "stream": F.KERNEL_STREAM, "tma": F.KERNEL_TMA, "auto": F.KERNEL_AUTO}[kernel_name]
    sim = F.Sim(prob, precision=F.F32, kernel=kernel, steps_per_launch=k, tile=tile, use_graph=graph)
    E = prob.opts.epoch_steps
    stream = torch.cuda.current_stream()
    # steps per launch: K for the temporal-blocked kernel, else 1 (a launch never crosses an epoch end)
    per_launch = (k or 4) if kernel_name in ("tiled", "auto") else 1
    # warm-up: at least one whole epoch
    warm = max(warmup, E)
    sim.step(warm)
    sim.sync()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    runs_ms, kern, launches = [], [], 0
    for _ in range(repeats):
        step0 = int(sim.ledger()["step"])
        # the launches of this run: up to per_launch steps each, cut at epoch ends
        plan, st = [], step0
        while st < step0 + steps_req:
            kk = min(per_launch, E - st % E, step0 + steps_req - st)
            plan.append((st % E == 0, kk))
            st += kk
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(plan) + 1)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev[0].record(stream)
        for j, (_, kk) in enumerate(plan):
            sim.step(kk)
            ev[j + 1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        runs_ms.append(ev[0].elapsed_time(ev[-1]))
        # launches that neither start an epoch nor are cut short run the step kernel alone
        kern += [ev[j].elapsed_time(ev[j + 1]) for j, (begin, kk) in enumerate(plan) if not begin and kk == per_launch]
        n_epochs = sum(1 for begin, _ in plan if begin)
        launches += len(plan) + n_epochs * (1 + (1 if sim_inflows(prob) else 0))
    clk = clocks.stop()
    sim.sync()
    total_ms = max_over_ranks(statistics.median(runs_ms), dist)
    kern_ms = statistics.mean(kern) if kern else total_ms / max(1, steps_req // per_launch)
    return {"sim": sim, "total_ms": total_ms, "kern_ms": kern_ms, "per_launch": per_launch, "steps": steps_req,
            "runs_ms": runs_ms, "clocks": clk, "launches": launches, "ledger": sim.ledger(), "warmup": warm}


def run_gpu(args):
    import torch
    import paper_2204_10323_gb300 as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    prob, wname = workload(args.workload)
    prob.opts.theta = args.theta
    prob.opts.friction = args.friction
    variant = args.theta != 1.0 or args.friction != 0
    ncell = prob.nx * prob.ny
    E = prob.opts.epoch_steps
    h0, qx0, qy0 = prob.initial_state(np.float32)
    stream = torch.cuda.current_stream()
    tile = tuple(int(v) for v in args.tile.split(",")) if args.tile else (0, 0)
    run = timed_run(F, torch, prob, args.kernel, args.k, tile, args.graph, args.steps, args.warmup, local, dist,
                    repeats=args.repeats)
    sim, total_ms, kern_ms, per_launch, steps = run["sim"], run["total_ms"], run["kern_ms"], run["per_launch"], \
        run["steps"]
    clk, launches, L = run["clocks"], run["launches"], run["ledger"]

    value = job_throughput(world, ncell, steps, total_ms)
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_CELL * ncell * per_launch / (kern_ms * 1e-3) / 1e9
    traffic = None
    if args.traffic_bytes:
        traffic = float(args.traffic_bytes)
    elif args.workload == "c3" and not variant and (args.kernel, per_launch) in TRAFFIC_B_PER_CELL:
        traffic = TRAFFIC_B_PER_CELL[(args.kernel, per_launch)] * ncell
    elif args.workload == "c3" and args.theta == 1.0 and args.friction == 1 and \
            (args.kernel, per_launch) in TRAFFIC_VEC_B_PER_CELL:
        traffic = TRAFFIC_VEC_B_PER_CELL[(args.kernel, per_launch)] * ncell

    # end to end through the C ABI with host buffers: upload state, K steps, read depth + ledger
    pin_h = torch.from_numpy(h0).pin_memory()
    pin_qx = torch.from_numpy(qx0).pin_memory()
    pin_qy = torch.from_numpy(qy0).pin_memory()
    out_h = torch.empty_like(pin_h).pin_memory()
    e2e_steps = args.steps
    # untimed first pass: the first copies out of freshly pinned host buffers cost
    # about 40 ms more than later ones (first use of the new pinned pages)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.write_state(pin_h.numpy(), pin_qx.numpy(), pin_qy.numpy())
    first_write_ms = (time.perf_counter() - t0) * 1e3
    F.flood_read(sim.h, F.FIELD_H, __import__("ctypes").c_void_p(out_h.data_ptr()), out_h.numel() * 4, 0)
    runs = []
    phases = {"write_state": [], "steps": [], "read_depth": [], "ledger": []}
    for _ in range(max(5, args.repeats)):   # median of the end-to-end runs, each phase timed on the host
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.write_state(pin_h.numpy(), pin_qx.numpy(), pin_qy.numpy())
        t1 = time.perf_counter()
        sim.step(e2e_steps)
        F.flood_sync(sim.h)
        t2 = time.perf_counter()
        F.flood_read(sim.h, F.FIELD_H, __import__("ctypes").c_void_p(out_h.data_ptr()), out_h.numel() * 4, 0)
        t3 = time.perf_counter()
        led = sim.ledger()
        t4 = time.perf_counter()
        runs.append(ncell * e2e_steps / (t4 - t0) / 1e9)
        for key, dt_s in zip(phases, (t1 - t0, t2 - t1, t3 - t2, t4 - t3)):
            phases[key].append(round(dt_s * 1e3, 3))
    h2d = (pin_h.numel() + pin_qx.numel() + pin_qy.numel()) * 4
    d2h = out_h.numel() * 4 + 9 * 8
    e2e = {"value": statistics.median(runs), "unit": UNIT, "runs": runs, "phases_ms": phases,
           "first_write_state_ms": round(first_write_ms, 3),
           "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
           "what": f"flood_write_state from pinned host (h, qx, qy), flood_step({e2e_steps}), "
                   f"flood_read(depth) + ledger to host; median of {len(runs)} runs"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "steps_requested": args.steps, "repeats": len(run["runs_ms"]),
            "repeat_ms": [round(x, 4) for x in run["runs_ms"]],
            "warmup": run["warmup"], "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wname, "nx": prob.nx, "ny": prob.ny, "kernel": args.kernel,
                       "steps_per_launch": args.k, "epoch_steps": E, "l2": "inputs larger than L2 (5.4 GB state)",
                       "theta": args.theta, "friction": "vector norm" if args.friction else "own component",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "bytes_per_cell": BYTES_PER_CELL, "kernel_ms": kern_ms, "steps_per_launch": per_launch,
                         "dram_gbs": traffic / (kern_ms * 1e-3) / 1e9 if traffic else None,
                         "dram_frac": traffic / (kern_ms * 1e-3) / 1e9 / peak if traffic else None,
                         "issue": issue_roofline(args.kernel, per_launch, ncell, kern_ms, clk, args),
                         "note": ("one-step algorithmic bytes (32 B per cell-update) over the launch time; with "
                                  f"{per_launch} steps per launch the kernel moves {traffic / ncell / per_launch:.1f} "
                                  "B of DRAM traffic per cell-update and is bound by instruction issue, so the "
                                  "fraction can pass 1") if per_launch > 1 and traffic else None},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "ledger": {k: L[k] for k in ("t", "dt", "V_in", "V_out", "V_clip", "volume")}}
    sim.close()
    del sim
    if not args.no_temporal and not variant:     # the tiled kernel runs Eq. 3 as printed
        if args.kernel != "tiled":
            line["temporal_blocking"] = temporal_leg(F, torch, prob, args, local, dist, ncell, peak)
        else:
            line["one_step"] = temporal_leg(F, torch, prob, args, local, dist, ncell, peak, K=1, kernel="stream")
    if not args.no_sweep:
        line["resolution_sweep"] = resolution_sweep(F, torch, prob, args, local, dist, total_ms / steps)
    if not args.no_adjoint:
        line["adjoint"] = adjoint_ratio(F, torch)
    if not args.no_decomp and not variant:
        line["decomposition"] = decomposition_leg(F, torch, prob, value, steps)
    if not args.no_ensemble:
        shape = [int(v) for v in args.ensemble_shape.split(",")] if args.ensemble_shape else None
        line["ensemble"] = ensemble_throughput(F, torch, value, shape=shape)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, seconds_target=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def issue_roofline(kernel: str, per_launch: int, ncell: int, kern_ms: float, clk, args):
    """Instruction-issue roofline of an issue-bound kernel: warp instructions per
    launch (ncu count per cell-update x the launch's cell-updates) over the launch
    time, against 152 SMs x 4 issue slots x the SM clock sampled meanwhile."""
    if args.workload != "c3" or args.theta != 1.0:
        return None
    table = INST_VEC_PER_CELL_UPDATE if args.friction == 1 else INST_PER_CELL_UPDATE
    ipc = table.get((kernel, per_launch))
    if ipc is None:
        return None
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    achieved = ipc * ncell * per_launch / (kern_ms * 1e-3)
    peak = SMS * ISSUE_PER_SM_CYCLE * mhz * 1e6
    return {"bound": "alu", "unit": "warp-instructions/s", "achieved": achieved, "peak": peak,
            "frac": achieved / peak, "inst_per_cell_update": ipc}


def temporal_leg(F, torch, prob, args, local, dist, ncell, peak, K: int = 4, kernel: str = "tiled"):
    """The same workload on another kernel: the temporal-blocking kernel (K
    steps per launch) beside a one-step headline, or the one-step stream kernel
    beside a temporal-blocking headline.  Whole-job Gcell-updates/s, and the
    kernel time as a fraction of the one-step HBM roofline (32 B per
    cell-update), beside the DRAM bytes it actually moves per launch."""
    run = timed_run(F, torch, prob, kernel, K if kernel == "tiled" else 0, (0, 0), args.graph, args.steps,
                    args.warmup, local, dist)
    run["sim"].close()
    value = ncell * run["steps"] / (run["total_ms"] * 1e-3) / 1e9
    eq = BYTES_PER_CELL * ncell * K / (run["kern_ms"] * 1e-3) / 1e9
    tr = TRAFFIC_B_PER_CELL.get((kernel, K)) if args.workload == "c3" else None
    return {"kernel": kernel, "steps_per_launch": K, "value": value, "unit": UNIT,
            "ms_per_step": run["total_ms"] / run["steps"], "kernel_ms_per_launch": run["kern_ms"],
            "equivalent_gbs": eq, "frac_of_one_step_roofline": eq / peak,
            "traffic_per_launch": tr * ncell if tr else None, "clocks": run["clocks"]}


def resolution_sweep(F, torch, prob, args, local, dist, ms_per_step_1m: float):
    """Steps/s of the step at 1, 2, 4 and 8 m: the workload's DEM, Manning field and
    initial depth coarsened by block averaging on the GPU (flood_coarsen), the way
    the paper derives its coarser grids from the 1 m DEM, each timed like the main
    leg; the paper's steps/s per TPU v3 core (Table 1) beside them as context."""
    from inputs import Problem
    # the library's own choice per grid (AUTO) unless a kernel family was asked for
    sweep_kernel = "auto" if args.kernel in ("stream", "reference") else args.kernel
    rows = [{"dx_m": prob.dx, "nx": prob.nx, "ny": prob.ny, "steps_per_s": 1e3 / ms_per_step_1m,
             "gcell_s": prob.nx * prob.ny / ms_per_step_1m / 1e6}]
    for f in (2, 4, 8):
        z, n = F.coarsen(prob.z, f), F.coarsen(prob.n, f)
        h0 = None if prob.h0 is None else F.coarsen(prob.h0, f)
        sub = Problem(f"{prob.name}_coarse{f}", z.shape[1], z.shape[0], prob.dx * f, z, n, prob.sections,
                      prob.opts, h0=h0)
        run = timed_run(F, torch, sub, sweep_kernel, args.k, (0, 0), args.graph, args.steps, args.warmup, local,
                        dist)
        run["sim"].close()
        ms = run["total_ms"] / run["steps"]
        rows.append({"dx_m": sub.dx, "nx": sub.nx, "ny": sub.ny, "steps_per_s": 1e3 / ms,
                     "gcell_s": sub.nx * sub.ny / ms / 1e6})
    return {"kernel": sweep_kernel + " at 2, 4, 8 m (" + args.kernel + " at 1 m)", "rows": rows,
            "paper_steps_per_s_one_tpu_v3_core": {"2 m, 248 M cells": 7.57, "4 m, 62 M cells": 30.2,
                                                  "8 m, 15.5 M cells": 118.0}}


def adjoint_ratio(F, torch, steps: int = 2000, checkpoints: int = 40):
    """Adjoint/forward time on the 1024^2 calibration workload (16 gauges, FP32).

    per_step: device time of one reverse step (the adjoint kernels, including
    their inline recompute of the forward faces) over that of one forward step,
    both measured by the library's event profiling inside the same
    flood_adjoint call; end_to_end: the gradient with 40 snapshots (binomial
    checkpointing, 5097 forward replays) over the plain 2000-step forward run,
    CUDA events around the library calls on the library's stream;
    auto_checkpoints: the same gradient with the snapshot count sized by the
    free device memory (every state kept on a GB300)."""
    import inputs
    p = inputs.c5_calibration(truth=False, steps=steps)
    g = p.gauges
    seed = np.ones((steps, len(g)))
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    s = F.Sim(p)
    s.step(32)                                              # warm-up
    s2 = F.Sim(p)
    t_fwd = timed(lambda: s2.step(steps))
    s3 = F.Sim(p)
    s3.adjoint(64, g, seed[:64], n_checkpoints=8)           # warm-up of the adjoint path
    t_grad = timed(lambda: s3.adjoint(steps, g, seed, n_checkpoints=checkpoints))
    replays = s3.adjoint_forward_steps()
    # the snapshot count sized by the free device memory (n_checkpoints = 0): every state kept
    t_grad_auto = timed(lambda: s3.adjoint(steps, g, seed, n_checkpoints=0))
    replays_auto = s3.adjoint_forward_steps()
    s3.adjoint_profile(True)
    s3.adjoint(steps, g, seed, n_checkpoints=checkpoints)
    prof = s3.adjoint_times()
    per_rev = prof["reverse_ms"] / max(prof["reverse_steps"], 1)
    per_fwd = prof["forward_ms"] / max(prof["forward_steps"], 1)
    for x in (s, s2, s3):
        x.close()
    return {"workload": f"calibration_{p.nx}x{p.ny}_{steps}_steps_{len(g)}_gauges_fp32",
            "forward_ms_per_step": per_fwd, "adjoint_ms_per_step": per_rev,
            "per_step_ratio": per_rev / per_fwd, "end_to_end_ratio": t_grad / t_fwd,
            "checkpoints": checkpoints, "forward_replays": replays,
            "gradient_ms": t_grad, "forward_run_ms": t_fwd,
            "auto_checkpoints": {"end_to_end_ratio": t_grad_auto / t_fwd, "gradient_ms": t_grad_auto,
                                 "forward_replays": replays_auto,
                                 "what": "n_checkpoints = 0: snapshots sized by half the free device memory "
                                         "(all 2000 states here)"}}


def ensemble_throughput(F, torch, single_value: float, n: int = 96, steps: int = 5000, shape=None):
    """96 uneven scenarios (256^2 .. 2048^2, own terrain seed, n ~ U(0.02, 0.08),
    hydrograph peak ~ U(100, 1000) m^3/s), primed ~30 % wet, stepped together
    with the autotuned launch shape; Gcell-updates/s over all scenarios."""
    import inputs
    from paper_2204_10323_gb300 import autotune
    probs = []
    for s in range(n):
        p = inputs.c4_scenario(s, steps=5000)
        p.h0 = inputs.wet_start(p.z, p.dx, 0.3)
        probs.append(p)
    ens = F.Ensemble(probs)
    if shape:                              # a fixed launch shape instead of tuning
        autotune.apply(ens, tuple(shape))
        tune = {"shape": list(shape), "trials": []}
    else:
        tune = autotune.tune_ensemble(ens, use_cache=False)
    spg = tune["shape"][3]                 # (K, warps, rows, steps per graph)
    steps = max(spg, steps // spg * spg)
    ens.step(spg)
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    ens.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    value = ens.cells * steps / (ms * 1e-3) / 1e9
    shapes = sorted({(p.nx, p.ny) for p in probs})
    out = {"workload": f"{n}_scenarios_uneven_{'_'.join(f'{x}x{y}' for x, y in shapes)}_fp32",
           "scenarios": n, "cells": ens.cells, "steps": steps, "value": value, "unit": UNIT,
           "ratio_to_single_grid": value / single_value, "launch_shape": tune["shape"],
           "autotune_ms_per_step": [[s, round(t, 4)] for s, t in tune["trials"]]}
    ens.close()
    return out


def decomposition_leg(F, torch, prob, single_value: float, steps: int, parts=(2, 4), halo: int = 4):
    """The same workload split into 1 x N row strips with `halo`-row halos,
    exchanged every `halo` steps (all parts on this GPU, each on a stream of its own): whole-job
    Gcell-updates/s and the ratio to the single grid, the cost of the halo rows'
    redundant steps, the exchanges and the per-part launches."""
    out = []
    E = prob.opts.epoch_steps
    n = max(steps, 2 * E)
    for n_parts in parts:
        stream = torch.cuda.current_stream()
        d = F.Decomp(prob, n_parts, halo, precision=F.F32, stream=stream)
        d.step(E)                                   # warm-up: one epoch
        d.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        d.step(n)
        b.record(stream)
        torch.cuda.synchronize()
        d.sync()
        ms = a.elapsed_time(b)
        value = prob.nx * prob.ny * n / (ms * 1e-3) / 1e9
        out.append({"parts": n_parts, "halo": halo, "steps": n, "value": value, "unit": UNIT,
                    "ratio_to_single_grid": value / single_value})
        d.close()
    return {"what": "1 x N row strips with halo exchange on one GPU (the paper's subgrids)", "runs": out}


def sim_inflows(prob):
    return any(s.kind == 0 for s in prob.sections)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # defaults: the 16384^2 protocol, 200 warm-up steps and five timed runs of 500 steps
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--repeats", type=int, default=5, help="timed runs of --steps steps; the median is reported")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c3")
    ap.add_argument("--kernel", default="tiled", choices=["stream", "rows", "tiled", "tma", "reference"])
    ap.add_argument("--k", type=int, default=4, help="steps per launch (tiled kernel)")
    ap.add_argument("--graph", action="store_true")
    ap.add_argument("--tile", default="", help="stream kernel launch shape: warps,rows")
    ap.add_argument("--traffic-bytes", type=float, default=None)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-decomp", action="store_true", help="skip the row-strip decomposition leg")
    ap.add_argument("--no-temporal", action="store_true", help="skip the temporal-blocking leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 1/2/4/8 m resolution sweep")
    ap.add_argument("--theta", type=float, default=1.0, help="face-flux weighting (1 = Eq. 3 as printed)")
    ap.add_argument("--friction", type=int, default=0, help="1: vector-norm |q| in the friction term")
    ap.add_argument("--ensemble-shape", default="", help="K,warps,rows,steps_per_graph instead of autotuning")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
