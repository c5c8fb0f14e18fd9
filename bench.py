#!/usr/bin/env python3
"""Benchmark of the coupled pressure-temperature multigrid on GB300.

Workload (one "step"): for each of two bubble problems, coefficient set-up
(mg_set_coeffs: elimination, coarsening, exact coarsest inverse) and a full
FP64 solve (mg_solve: V(2,2) cycles, red-black block Gauss-Seidel, stop at
1e-10 reduction of both per-field residual norms):
  - 2D 1024 x 1024, 16 seeded bubbles (radii 0.02-0.08), walls;
  - axisymmetric 512 x 1024 (r, z), one bubble of radius 0.2 on the axis.
Metric: Mcell * V-cycles per second (finest cells times cycles, summed over the
step, per second of device time), plus solves per second.

Schedule (--schedule): "concurrent" (default) gives each problem its own
handle and stream and runs them at once, problem 0 through mg_solve (its
cycle graphs carry the timing hooks of the dominant kernel) and the others
through mg_solve_async; the problems are independent, so the kernels of one
fill the SMs that the other's coarse levels and host waits leave idle, and
every result is bit for bit that of a solve alone.  "serial" solves them one
after the other on one stream.  In the concurrent step the timed sweep shares
the SMs with the other problem's kernels, so the roofline also reports the
same kernel timed in serial steps after the timed region ("isolated").

Arms:
  default            the CUDA library through its C ABI (inputs resident in HBM);
                     `e2e` repeats the step through the library's host-buffer
                     path (mg_set_coeffs / mg_solve with on_device = 0: every
                     copy inside the timed region).  With one GPU the same run
                     adds `sub_results`: the workload in mixed precision, its
                     stiff variant at the paper's bubble scale (cycles per solve,
                     convergence factor), the 256-problem batch (batched and
                     looped, FP64 and mixed) and one serving rate (p50 / p99).
  --impl reference   the FP64 CPU oracle on the host cores (OpenMP over
                     same-colour cells, every core), a bounded sample of the
                     same workload per step (one V-cycle per problem).

Multi-GPU (torchrun): replicas only.  Each rank solves its own copy of the
workload; value = units of all ranks / max-over-ranks time (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled p-T MG Mcell-Vcycles/s & solves/s at 1e-10 resid; HBM %peak; p50/p99"
UNIT = "Mcell-Vcycles/s"
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes per launch of a dominant kernel, from ncu captures of that
# kernel; an entry holds while the kernel's source is unchanged.
# "cold": ncu's default capture (caches flushed before the launch, the
# recipe's figure); "warm": caches as the solve leaves them (median of the
# 16 finest-level launches of one solve sequence).
TRAFFIC = {
    "k_rbgs_colour<double,2> on the finest level of bubbles16_1024x1024": {
        "cold": 103.9e6, "warm": 32.4e6,
        "source": "ncu capture of k_rbgs_colour<double,2> on the 1024^2 level: --set full (cold, mean of the "
                  "first two launches), --cache-control none over two solve sequences (warm, median of 16)"},
}
L2_FLUSH_BYTES = 256 << 20
# algorithmic bytes per finest cell of one full red-black sweep: read x 16 +
# bt 16 (Dinv b) + W 32 (the cell's 2x2 update matrix) + faces (2D 32, 3D 48),
# write x 16 (FP64); half of that for the FP32 cycles of mixed precision
SWEEP_BYTES_PER_CELL = {("fp64", 2): 112.0, ("fp64", 3): 128.0, ("mixed", 2): 56.0, ("mixed", 3): 64.0}
# FP64 instructions per cell update of a sweep (each cell once per sweep): the
# two neighbour sums 2*2*dim (first a multiply, the rest FMAs), then
# x = bt - W (sT, sp) as 4 FMAs
SWEEP_FP64_INST_PER_CELL = {2: 12.0, 3: 16.0}
# GB300 FP64 pipe: 1.25 TFLOP/s nominal = 2 FP64 FMA per clock per SM
# (1.25e12 / (2 * 152 * 2.07e9) = 1.99); 152 SMs at 2.07 GHz.  Used only when
# the measurement below fails; the run measures the rate with the library's
# register-FMA kernel (mg_fp64_fma_rate).
FP64_INST_PEAK_G = 152 * 2 * 2.07


def fp64_peak():
    """(G FP64 instructions/s, source): measured on this device in this run."""
    try:
        from paper_2206_11294_gb300 import binding as B
        return B.fp64_fma_rate(10), "measured in this run: independent register FMA chains (mg_fp64_fma_rate), " \
                                    "fastest of 10 launches"
    except Exception as e:        # noqa: BLE001
        return FP64_INST_PEAK_G, f"derived (measurement failed: {e}): 152 SMs x 2 FP64 inst/clk/SM x 2.07 GHz"


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def replica_value(local_units: float, local_seconds: float, world: int, device: str = "cuda"):
    """Weak-scaling value of replicas: units of all ranks / the slowest rank's time."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t.item())
    return local_units * world / tmax, tmax


def workload_problems():
    from paper_2206_11294_gb300 import inputs as I
    return [I.bubbles_1024(), I.bubble_axi()]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                v = d[k]
                return float(v["value"] if isinstance(v, dict) else v), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if device_id:
                cmd += ["-i", device_id]
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        try:
            self.proc.terminate()
            self.proc.wait(timeout=5)
        except Exception:
            pass
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                try:
                    rows.append(parts)
                except Exception:
                    pass
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[0]) for r in rows if r[0].replace(".", "").isdigit())
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[4 + q].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_identity(torch, dev):
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def solve_concurrently(solvers, data, main, allow=False):
    """One set-up + solve of every problem, each handle on its own stream,
    forked from and joined back into `main`.  Problems 1.. are enqueued first
    with mg_solve_async (the stop test runs on the device, the host does not
    wait); problem 0 then runs mg_solve, whose per-cycle graphs carry the
    timing hooks; then the others' statistics are collected.  The problems are
    independent, so their kernels overlap on the device; every result is bit
    for bit the one of a solve alone."""
    import torch
    fork = torch.cuda.Event()
    fork.record(main)
    for s in solvers:
        s.stream.wait_event(fork)
    for s, d in list(zip(solvers, data))[1:]:
        s.set_coeffs(d["lam"], d["fa"], d["fk"])
        s.solve_async(d["b"], d["x"])
    s0, d0 = solvers[0], data[0]
    s0.set_coeffs(d0["lam"], d0["fa"], d0["fk"])
    out = [s0.solve(d0["b"], d0["x"], allow_not_converged=allow)]
    out += [s.async_stats(allow_not_converged=allow) for s in solvers[1:]]
    for s in solvers:
        e = torch.cuda.Event()
        e.record(s.stream)
        main.wait_event(e)
    return out


def solve_serially(solvers, data, allow=False):
    """The same step with the problems one after the other (mg_solve each)."""
    return [(s.set_coeffs(d["lam"], d["fa"], d["fk"]), s.solve(d["b"], d["x"], allow_not_converged=allow))[1]
            for s, d in zip(solvers, data)]


def in_threads(fns):
    """Runs the callables in one host thread each (the library's calls release
    the interpreter lock) and returns their results in order."""
    import threading
    out, err = [None] * len(fns), []

    def run(i):
        try:
            out[i] = fns[i]()
        except BaseException as e:        # noqa: BLE001
            err.append(e)
    th = [threading.Thread(target=run, args=(i,)) for i in range(len(fns))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if err:
        raise err[0]
    return out


def sweep_timing(solver, precision, dim):
    """Launch count and average duration of the finest-level smoothing pass
    timed by the handle's hooks, with its algorithmic bytes and FP64
    instructions per launch."""
    c = solver.counters()
    spl = c["smooth_sweeps"] / max(1, c["smooth_launches"])
    avg_s = c["smooth_ms"] / 1e3 / max(1, c["smooth_launches"])
    return {"launches": c["smooth_launches"], "avg_s": avg_s,
            "bytes": SWEEP_BYTES_PER_CELL[(precision, dim)] * c["smooth_cells"] * spl,
            "fp64_inst": SWEEP_FP64_INST_PER_CELL[dim] * c["smooth_cells"] * spl}


def face_bytes(p):
    return sum(8 * (a.size + b.size) for a, b in zip(p.fa, p.fk))


# ----------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2206_11294_gb300.binding import Solver, TILE_SHAPES

    dev = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    probs = workload_problems()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda(dev)
    dev_in = []
    solvers = []
    for p in probs:
        # one stream per handle: independent problems overlap on the device
        s = Solver(p.grid, precision=args.precision, rtol=1e-10, max_cycles=50, device=dev,
                   stream=torch.cuda.Stream(dev), cycle=args.cycle)
        dev_in.append(dict(lam=T(p.lam), fa=[T(f) for f in p.fa], fk=[T(f) for f in p.fk], b=T(p.b),
                           x0=T(p.x0), x=T(p.x0)))
        solvers.append(s)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{dev}")
    # kernel choices from the library's autotuner (before warm-up, untimed)
    tunings = {}
    if not args.no_tune:
        from paper_2206_11294_gb300.autotune import TuningTable, describe
        table = TuningTable(args.tuning_table)      # a stored table is applied, not measured again
        for p, s, d in zip(probs, solvers, dev_in):
            s.set_coeffs(d["lam"], d["fa"], d["fk"])
            tunings[p.name] = describe(table.tune(s, reps=args.tune_reps))
        table.save()
    torch.cuda.synchronize()

    def step(collect, schedule=args.schedule):
        if schedule == "concurrent":
            collect += solve_concurrently(solvers, dev_in, stream)
        else:
            collect += solve_serially(solvers, dev_in)

    def timed_steps(n, collect, schedule=args.schedule):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for k in range(n):
            flush.zero_()                           # L2 flushed between timed steps
            for d in dev_in:
                d["x"].copy_(d["x0"])
            ev[k][0].record(stream)
            step(collect, schedule)
            ev[k][1].record(stream)
        return ev

    # timing hooks of the dominant kernel: one finest-level smoothing pass per
    # cycle of problem 0 only (the hooks cost the step ~1%; every handle's
    # launch counter runs regardless)
    solvers[0].set_timing(True)
    for _ in range(args.warmup):
        for d in dev_in:
            d["x"].copy_(d["x0"])
        step([])
    torch.cuda.synchronize()
    solvers[0].set_timing(True)      # reset counters after warm-up
    for s in solvers[1:]:
        s.set_timing(False)          # (also resets their launch counters)
    stats = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_identity(torch, dev)) if rank == 0 else None
    wall0 = time.perf_counter()
    ev = timed_steps(args.steps, stats)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_ms = sum(step_ms)
    counters = [s.counters() for s in solvers]
    live = sweep_timing(solvers[0], args.precision, probs[0].grid.dim)
    units = sum(p.grid.N * st["cycles"] for p, st in zip(probs * args.steps, stats)) / 1e6
    solves = len(stats)
    value, tmax = replica_value(units, dev_ms / 1e3, world, device=f"cuda:{dev}")
    # the same kernel with the problems one after the other (steps after the
    # timed region): in the concurrent step its launches share the SMs with
    # the other problem's kernels, so their duration there is the share it got
    isolated = None
    if args.schedule == "concurrent":
        for s in solvers[1:]:
            s.set_timing(False)
        solvers[0].set_timing(True)
        timed_steps(max(3, args.steps // 2), [], "serial")
        torch.cuda.synchronize()
        isolated = sweep_timing(solvers[0], args.precision, probs[0].grid.dim)
    # roofline of the dominant kernel, from its live event timings
    peak, peak_kind = measured_peak()
    fpeak, fpeak_src = fp64_peak()
    dim0 = probs[0].grid.dim
    t0 = solvers[0].tuning()
    rname = "double" if args.precision == "fp64" else "float"
    if t0["sweep"][0] in ("fused", "fused2"):
        tx, ty = TILE_SHAPES[t0["tile"][0]]
        kernel = f"k_rbgs_fused2d{'_x2' if t0['sweep'][0] == 'fused2' else ''}<{rname},{tx},{ty}>"
    else:
        kernel = f"k_rbgs_colour<{rname},{dim0}>"
    kernel += " on the finest level of " + probs[0].name
    tr = TRAFFIC.get(kernel)
    traffic = args.traffic if args.traffic is not None else (tr["cold"] if tr else None)
    traffic_note = None if args.traffic is not None or not tr else dict(tr)

    def roofline_of(t):
        avg_s = t["avg_s"]
        achieved = t["bytes"] / avg_s / 1e9 if avg_s > 0 else None
        hbm = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
               "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
               "algorithmic_bytes_per_launch": t["bytes"], "avg_launch_us": avg_s * 1e6,
               "launches_timed": t["launches"], "traffic": traffic, "traffic_ncu": traffic_note}
        if args.precision != "fp64":
            return hbm
        ach_i = t["fp64_inst"] / avg_s / 1e9 if avg_s > 0 else None
        return {"bound": "alu", "kernel": kernel, "achieved": ach_i, "peak": fpeak,
                "unit": "G FP64 inst/s", "frac": (ach_i / fpeak) if ach_i else None,
                "peak_source": fpeak_src,
                "algorithmic_fp64_inst_per_launch": t["fp64_inst"], "avg_launch_us": avg_s * 1e6,
                "launches_timed": t["launches"], "traffic": traffic, "traffic_ncu": traffic_note,
                "hbm": hbm}

    roofline = roofline_of(live)
    if isolated is not None:
        roofline["timed_in"] = "the concurrent step (the other problem's kernels share the SMs)"
        iso = roofline_of(isolated)
        iso["timed_in"] = "serial steps after the timed region (the problems one after the other)"
        roofline["isolated"] = {k: iso[k] for k in ("achieved", "frac", "avg_launch_us", "launches_timed",
                                                    "timed_in")}
        if "hbm" in iso:
            roofline["isolated"]["hbm_frac"] = iso["hbm"]["frac"]
    cycles = [st["cycles"] for st in stats[: len(probs)]]

    # end to end through the library's host-buffer path: mg_set_coeffs and
    # mg_solve with on_device = 0 take pinned host arrays and copy them in
    # inside the call, and mg_solve copies the result back; every copy is in
    # the timed region.  Each step starts from its own host copy of the
    # initial guess (prepared before timing), since the solve overwrites it.
    e2e = None
    if not args.no_e2e:
        for s, d in zip(solvers, dev_in):
            s.set_timing(False)
            d["x"].copy_(d["x0"])
            s.solve(d["b"], d["x"])            # graphs re-captured without event nodes, untimed
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        host = [dict(lam=pin(p.lam), fa=[pin(f) for f in p.fa], fk=[pin(f) for f in p.fk], b=pin(p.b))
                for p in probs]
        xs = [[pin(p.x0) for p in probs] for _ in range(args.steps)]
        for p, s, hd in zip(probs, solvers, host):     # untimed: the set-up graph of the staging inputs
            s.set_coeffs(hd["lam"], hd["fa"], hd["fk"])
            s.solve(hd["b"], pin(p.x0))
        torch.cuda.synchronize()
        def one(s, hd, xh):
            s.set_coeffs(hd["lam"], hd["fa"], hd["fk"])
            return s.solve(hd["b"], xh)

        e_units = 0.0
        w0 = time.perf_counter()
        for k in range(args.steps):
            work = [lambda s=s, hd=hd, xh=xh: one(s, hd, xh) for s, hd, xh in zip(solvers, host, xs[k])]
            # concurrent: one host thread per handle, each on its own stream
            sts = in_threads(work) if args.schedule == "concurrent" else [w() for w in work]
            e_units += sum(p.grid.N * st["cycles"] for p, st in zip(probs, sts)) / 1e6
        torch.cuda.synchronize()
        e_wall = time.perf_counter() - w0
        tt = torch.tensor([e_wall], dtype=torch.float64, device=f"cuda:{dev}")
        if world > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        h2d = sum(32 * p.grid.N + face_bytes(p) + 32 * p.grid.N for p in probs)
        d2h = sum(16 * p.grid.N for p in probs)
        e2e = {"value": e_units * world / float(tt.item()), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "seconds": float(tt.item()),
               "copies": "through the C ABI with on_device = 0: pinned host lambda, faces, rhs and x in, x out, "
                         "inside mg_set_coeffs / mg_solve (synchronous calls, no overlap between steps)",
               "schedule": ("one host thread per problem, each handle on its own stream"
                            if args.schedule == "concurrent" else "the problems one after the other"),
               "check": bool(all(np.array_equal(xs[-1][q].numpy(), dev_in[q]["x"].cpu().numpy())
                                 for q in range(len(probs))))}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(probs, batch_sample=not args.no_sub and not args.no_batch)

    subs = None
    if rank == 0 and world == 1 and not args.no_sub:
        subs = sub_results(args, dev, stream, flush, fp64_result=[d["x"].cpu().numpy() for d in dev_in])

    if rank != 0:
        return None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded bubble fields; Eqs. 29-34 coefficients)",
        "config": {"workload": "bubbles16_1024x1024 + axi_512x1024, set-up + solve to 1e-10 per step",
                   "cells_per_step": sum(p.grid.N for p in probs), "cycles_per_solve": cycles,
                   "solves_per_s": solves * world / tmax, "precision": args.precision,
                   "step_ms_p10_p50_p90": [float(np.percentile(step_ms, q)) for q in (10, 50, 90)],
                   "cycle": f"{args.cycle}(2,2) red-black block GS, exact coarsest solve",
                   "l2": "flushed between steps",
                   "parallelism": f"replicas x{world}",
                   "schedule": ("concurrent: each problem on its own handle and stream, problem 0 by mg_solve, "
                                "the others by mg_solve_async" if args.schedule == "concurrent"
                                else "serial: mg_solve of each problem in turn, one stream"),
                   "tuning": tunings or "library defaults (--no-tune)"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "sub_results": subs,
        "gpu_launches": int(sum(c["launches"] for c in counters)),
        "clocks": clk,
        "wall_s": wall,
    }
    return out


# ----------------------------------------------------------------- sub-results
def time_arm(probs, precision, steps, warmup, dev, stream, flush, tune=True, tune_reps=5, max_cycles=50,
             sweep_roofline=False, schedule="concurrent"):
    """Set-up + solve to 1e-10 of every problem per step, inputs resident in
    HBM, L2 flushed between steps, device events around each step, the
    problems scheduled as the headline's (`schedule`).  Returns the figures
    and the final solutions.  sweep_roofline: also the finest-level sweeps of
    problem 0 timed live (event hooks) against the measured HBM bandwidth, in
    the step and (concurrent schedule) in serial steps after it."""
    import numpy as np
    import torch
    from paper_2206_11294_gb300.binding import Solver
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda(dev)
    solvers, din = [], []
    for p in probs:
        s = Solver(p.grid, precision=precision, rtol=1e-10, max_cycles=max_cycles, device=dev,
                   stream=torch.cuda.Stream(dev))
        d = dict(lam=T(p.lam), fa=[T(f) for f in p.fa], fk=[T(f) for f in p.fk], b=T(p.b), x0=T(p.x0), x=T(p.x0))
        s.set_coeffs(d["lam"], d["fa"], d["fk"])
        if tune:
            s.autotune(tune_reps)
        solvers.append(s)
        din.append(d)
    torch.cuda.synchronize()
    stats = []

    def step(out, how=schedule):
        for d in din:
            d["x"].copy_(d["x0"])
        if how == "concurrent":
            out += solve_concurrently(solvers, din, stream, allow=True)
        else:
            out += solve_serially(solvers, din, allow=True)

    def timed(n, out, how=schedule):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for k in range(n):
            flush.zero_()
            ev[k][0].record(stream)
            step(out, how)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return ev

    if sweep_roofline:
        solvers[0].set_timing(True)
    for _ in range(warmup):
        step([])
    torch.cuda.synchronize()
    if sweep_roofline:
        solvers[0].set_timing(True)          # counters from the timed steps only
    ev = timed(steps, stats)
    secs = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    units = sum(p.grid.N * st["cycles"] for p, st in zip(probs * steps, stats)) / 1e6
    first = stats[: len(probs)]
    out = {"mcell_vcycles_per_s": units / secs, "solves_per_s": len(stats) / secs, "ms_per_step": secs * 1e3 / steps,
           "cycles_per_solve": [st["cycles"] for st in first], "outer_steps": [st["outer"] for st in first],
           "status": [st["status"] for st in first], "schedule": schedule,
           "convergence_factor": [[(st["rfinal"][f] / st["r0"][f]) ** (1.0 / max(1, st["cycles"]))
                                   if st["r0"][f] > 0 else 0.0 for f in range(2)] for st in first]}
    if sweep_roofline:
        dim0 = probs[0].grid.dim
        peak, peak_kind = measured_peak()
        t0 = solvers[0].tuning()

        def hbm_of(t):
            ach = t["bytes"] / t["avg_s"] / 1e9 if t["avg_s"] > 0 else None
            return ach, (ach / peak) if ach else None

        live = sweep_timing(solvers[0], precision, dim0)
        ach, frac = hbm_of(live)
        out["sweep_roofline"] = {"bound": "hbm", "kernel": f"finest-level {t0['sweep'][0]} sweep of {probs[0].name}",
                                 "achieved": ach, "peak": peak, "unit": "GB/s",
                                 "frac": frac, "peak_source": peak_kind,
                                 "algorithmic_bytes_per_launch": live["bytes"], "avg_launch_us": live["avg_s"] * 1e6,
                                 "launches_timed": live["launches"]}
        if schedule == "concurrent":
            solvers[0].set_timing(True)
            timed(max(3, steps // 2), [], "serial")
            iso = sweep_timing(solvers[0], precision, dim0)
            ach_i, frac_i = hbm_of(iso)
            out["sweep_roofline"]["timed_in"] = "the concurrent step"
            out["sweep_roofline"]["isolated"] = {"achieved": ach_i, "frac": frac_i,
                                                 "avg_launch_us": iso["avg_s"] * 1e6,
                                                 "launches_timed": iso["launches"],
                                                 "timed_in": "serial steps after the timed region"}
    xs = [d["x"].cpu().numpy() for d in din]
    for s in solvers:
        s.close()
    return out, xs


def rel_dev(x, ref, x0):
    import numpy as np
    return max(float(np.linalg.norm(x[:, f] - ref[:, f]) / max(np.linalg.norm(ref[:, f] - x0[:, f]), 1e-300))
               for f in range(2))


def sub_results(args, dev, stream, flush, fp64_result):
    """Figures beside the headline in the same run (one GPU): mixed precision
    on the headline workload (and its distance to the FP64 result), the stiff
    variant at the paper's bubble scale in FP64 and mixed, the 256-problem
    batch in four arms, and one serving rate."""
    from paper_2206_11294_gb300 import inputs as I
    out = {}
    t0 = time.perf_counter()
    probs = workload_problems()
    mixed, xm = time_arm(probs, "mixed", args.steps, args.warmup, dev, stream, flush, tune=not args.no_tune,
                         sweep_roofline=True, tune_reps=args.tune_reps, schedule=args.schedule)
    mixed["vs_fp64_rel_l2_of_deviation"] = max(rel_dev(a, b, p.x0) for a, b, p in zip(xm, fp64_result, probs))
    mixed["workload"] = "bubbles16_1024x1024 + axi_512x1024, mixed precision (FP32 cycles, FP64 residual and update)"
    out["mixed"] = mixed
    stiff = {"workload": "the same two geometries at the paper's bubble scale (domain 6.4 mm = 64 R0 with "
                         "R0 = 0.1 mm, dt = 1e-5): Laplacian-dominated p-row, density ratio 1000",
             "max_cycles": 200}
    sp = [I.stiff(I.bubbles_1024), I.stiff(I.bubble_axi)]
    for prec in ("fp64", "mixed"):
        stiff[prec], _ = time_arm(sp, prec, max(2, args.steps // 4), 1, dev, stream, flush, tune=not args.no_tune,
                                  tune_reps=args.tune_reps, max_cycles=200, schedule=args.schedule)
    out["stiff"] = stiff
    if not args.no_batch:
        bargs = argparse.Namespace(**vars(args))
        bargs.steps, bargs.warmup = args.batch_steps, 1
        out["batch"] = run_batch(bargs, modes=("batched_mixed", "batched_fp64", "loop_fp64", "loop_mixed"))
    if not args.no_serve:
        sargs = argparse.Namespace(**vars(args))
        sargs.serve_rates = [args.sub_serve_rate]
        sargs.serve_seconds = args.sub_serve_seconds
        out["serve"] = run_serve(sargs)
    out["seconds"] = time.perf_counter() - t0
    return out


# ----------------------------------------------------------------- other workloads
def run_batch(args, modes=("batched_mixed", "loop_fp64")):
    """256 independent 2D problems (sizes log-uniform 64..1024, multiples of 32,
    1-8 bubbles, density ratio 1000), each step set-up + solve to 1e-10 of all
    of them, in the given arms: batched_* through one mg_batch per step,
    loop_* looping the single-problem solver; *_mixed / *_fp64 the precision.
    batched_mixed against loop_fp64 is the headline speed-up; the other two
    arms separate the gain from batching from the gain from precision."""
    import numpy as np
    import torch
    from paper_2206_11294_gb300 import inputs as I
    from paper_2206_11294_gb300.binding import Batch, Solver
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    probs = I.batch_problems(count=args.batch_count)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dev = [dict(lam=T(p.lam), fa=[T(f) for f in p.fa], fk=[T(f) for f in p.fk], b=T(p.b), x0=T(p.x0),
                x=T(p.x0)) for p in probs]
    cells = sum(p.grid.N for p in probs)
    out = {"workload": f"batch of {len(probs)} 2D problems, {cells} cells", "metric": "solves/s at 1e-10"}
    for mode in modes:
        prec = "mixed" if mode.endswith("mixed") else "fp64"
        solvers = [Solver(p.grid, precision=prec, rtol=1e-10, max_cycles=60, stream=stream) for p in probs]
        batch = Batch(solvers) if mode.startswith("batched") else None
        # kernel choices from the library's autotuner (untimed): the batch's own
        # search, or the per-hierarchy table (equal shapes measured once)
        tuned = None
        if not args.no_tune:
            from paper_2206_11294_gb300.autotune import TuningTable
            if batch is not None:
                batch.set_coeffs([d["lam"] for d in dev], [d["fa"] for d in dev], [d["fk"] for d in dev])
                bt, bms = batch.autotune(reps=args.tune_reps)
                tuned = {"blocks_per_sm": bt["blocks_per_sm"],
                         "sweeps": ",".join("C" if s == "colour" else f"F{t}" for s, t in zip(bt["sweep"], bt["tile"])),
                         "cycle_ms": bms}
            else:
                table = TuningTable(None)
                for s, d in zip(solvers, dev):
                    s.set_coeffs(d["lam"], d["fa"], d["fk"])
                    table.tune(s, reps=args.tune_reps)
                tuned = {"hierarchies_measured": table.measured, "reused": table.reused}

        def step(stats):
            for d in dev:
                d["x"].copy_(d["x0"])
            if batch is not None:
                batch.set_coeffs([d["lam"] for d in dev], [d["fa"] for d in dev], [d["fk"] for d in dev])
                stats.extend(batch.solve([d["b"] for d in dev], [d["x"] for d in dev]))
            else:
                for s, d in zip(solvers, dev):
                    s.set_coeffs(d["lam"], d["fa"], d["fk"])
                    stats.append(s.solve(d["b"], d["x"]))

        for _ in range(args.warmup):
            step([])
        torch.cuda.synchronize()
        st = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(st)
        e1.record(stream)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        cyc = [s["cycles"] for s in st[: len(probs)]]
        out[mode] = {"solves_per_s": len(st) / secs, "ms_per_step": secs * 1e3 / args.steps,
                     "mcell_vcycles_per_s": sum(p.grid.N * c for p, c in zip(probs, cyc)) * args.steps / secs / 1e6,
                     "cycles_mean": float(np.mean(cyc)), "launches": batch.launches() if batch else None,
                     "tuning": tuned}
        if batch is not None:
            batch.close()
        for s in solvers:
            s.close()
    sp = lambda a, b: out[a]["solves_per_s"] / out[b]["solves_per_s"] if a in out and b in out else None
    out["speedup_batched_mixed_vs_loop_fp64"] = sp("batched_mixed", "loop_fp64")
    out["speedup_batching_fp64"] = sp("batched_fp64", "loop_fp64")
    out["speedup_batching_mixed"] = sp("batched_mixed", "loop_mixed")
    out["speedup_mixed_looped"] = sp("loop_mixed", "loop_fp64")
    out["speedup_mixed_batched"] = sp("batched_mixed", "batched_fp64")
    return out


def run_wall3d(args):
    """256^3 bubble 0.2 above a no-flux wall, Dirichlet p = 1e5, T = 300 on the
    other faces: FP64 and mixed precision to 1e-10 (set-up + solve per step)."""
    import numpy as np
    import torch
    from paper_2206_11294_gb300 import inputs as I
    from paper_2206_11294_gb300.binding import Solver
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    p = I.bubble_wall_3d(args.n3d)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d = dict(lam=T(p.lam), fa=[T(f) for f in p.fa], fk=[T(f) for f in p.fk], b=T(p.b), x0=T(p.x0), x=T(p.x0))
    out = {"workload": f"wall3d_{args.n3d}^3, set-up + solve to 1e-10 per step", "cells": p.grid.N}
    peak, peak_kind = measured_peak()
    results = {}
    for prec in ("fp64", "mixed"):
        s = Solver(p.grid, precision=prec, rtol=1e-10, max_cycles=60, stream=stream)
        tuned = "library defaults (--no-tune)"
        if not args.no_tune:                   # the library's autotuner, before the warm-up (untimed)
            from paper_2206_11294_gb300.autotune import describe
            s.set_coeffs(d["lam"], d["fa"], d["fk"])
            t, _ = s.autotune(args.tune_reps)
            tuned = describe(t)
        s.set_timing(True)
        for _ in range(args.warmup):
            d["x"].copy_(d["x0"])
            s.set_coeffs(d["lam"], d["fa"], d["fk"])
            s.solve(d["b"], d["x"])
        torch.cuda.synchronize()
        s.set_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = []
        e0.record(stream)
        for _ in range(args.steps):
            d["x"].copy_(d["x0"])
            s.set_coeffs(d["lam"], d["fa"], d["fk"])
            st.append(s.solve(d["b"], d["x"]))
        e1.record(stream)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        c = s.counters()
        spl = c["smooth_sweeps"] / max(1, c["smooth_launches"])
        avg = c["smooth_ms"] / 1e3 / max(1, c["smooth_launches"])
        byts = SWEEP_BYTES_PER_CELL[(prec, 3)] * c["smooth_cells"] * spl
        ent = {"mcell_vcycles_per_s": sum(p.grid.N * x["cycles"] for x in st) / secs / 1e6,
               "solves_per_s": len(st) / secs, "ms_per_step": secs * 1e3 / args.steps, "cycles": st[0]["cycles"],
               "outer": st[0]["outer"], "sweep_us": avg * 1e6, "tuning": tuned,
               "sweep_hbm": {"achieved_GBs": byts / avg / 1e9, "frac": byts / avg / 1e9 / peak, "peak": peak,
                             "peak_source": peak_kind}}
        if prec == "fp64":
            inst = SWEEP_FP64_INST_PER_CELL[3] * c["smooth_cells"] * spl
            ent["sweep_alu"] = {"achieved_G_fp64_inst_s": inst / avg / 1e9,
                                "frac": inst / avg / 1e9 / FP64_INST_PEAK_G}
        results[prec] = d["x"].cpu().numpy()
        out[prec] = ent
        s.close()
    dev = results["fp64"] - p.x0
    out["mixed_vs_fp64_rel_l2"] = max(float(np.linalg.norm(results["mixed"][:, f] - results["fp64"][:, f]) /
                                            np.linalg.norm(dev[:, f])) for f in range(2))
    out["speedup_mixed_vs_fp64"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


class nvtx_range:
    """An NVTX range around a timed loop, so that a profiler can take its
    kernels alone (ncu --nvtx --nvtx-include "<name>/")."""

    def __init__(self, name: str):
        self.name = name

    def __enter__(self):
        import torch
        torch.cuda.nvtx.range_push(self.name)

    def __exit__(self, *exc):
        import torch
        torch.cuda.nvtx.range_pop()


def run_coarse(args):
    """Grids whose coarsest level is large (an odd factor of 9 or more: 2D n =
    480, 736, 992, coarsest 15^2, 23^2, 31^2; 3D n = 96, 160, 224, coarsest
    6^3, 5^3, 7^3), set-up + solve to 1e-10 per step, FP64 and mixed, with the
    coarsest level solved from its LU factors (coarse_solve AUTO) and through
    the inverse formed at set-up (INVERSE); literal units, autotuned."""
    import numpy as np
    import torch
    from paper_2206_11294_gb300 import inputs as I
    from paper_2206_11294_gb300.binding import Solver
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    probs = [I.bubble_2d(n=n, seed=5, n_bubbles=4, rmin=0.02, rmax=0.08, centred=False) for n in (480, 736, 992)]
    probs += [I.bubble_wall_3d(n=n, seed=700) for n in (96, 160, 224)]
    out = {"workload": "large coarsest levels: set-up + solve to 1e-10 per step", "cases": []}
    for p in probs:
        d = dict(lam=T(p.lam), fa=[T(f) for f in p.fa], fk=[T(f) for f in p.fk], b=T(p.b), x0=T(p.x0), x=T(p.x0))
        case = {"grid": "x".join(str(v) for v in p.grid.n[:p.grid.dim]), "cells": p.grid.N}
        for prec in ("fp64", "mixed"):
            for coarse in ("auto", "inverse"):
                s = Solver(p.grid, precision=prec, rtol=1e-10, max_cycles=60, stream=stream, coarse=coarse)
                case["coarsest"] = "x".join(str(v) for v in s.levels()[-1][:p.grid.dim])
                s.set_coeffs(d["lam"], d["fa"], d["fk"])
                if not args.no_tune:
                    s.autotune(args.tune_reps)
                for _ in range(args.warmup):
                    d["x"].copy_(d["x0"])
                    s.set_coeffs(d["lam"], d["fa"], d["fk"])
                    s.solve(d["b"], d["x"])
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                with nvtx_range(f"coarse_{case['grid']}_{prec}_{coarse}"):
                    for _ in range(args.steps):
                        d["x"].copy_(d["x0"])
                        s.set_coeffs(d["lam"], d["fa"], d["fk"])
                        st = s.solve(d["b"], d["x"])
                e1.record(stream)
                torch.cuda.synchronize()
                case[f"{prec}_{coarse}"] = {"ms_per_step": e0.elapsed_time(e1) / args.steps, "cycles": st["cycles"],
                                            "workspace_mb": s.workspace_bytes / 1e6}
                s.close()
        out["cases"].append(case)
    out["l2"] = "not flushed (one problem resident)"
    out["data"] = "synthetic (seeded bubble fields)"
    return out


def run_adaptive(args):
    """A refined-patch (adaptive) grid against the uniform grid of its finest
    spacing: one bubble of radius 0.1 at the centre of the unit square, walls;
    the composite grid is a 512^2 base grid whose box around the bubble is
    refined 2:1 (finest spacing 1/1024 there), the uniform one 1024^2.  Each
    is set up and solved to a 1e-10 reduction of its residual norms, in the
    workloads' units and at the paper's bubble scale, in FP64 and in mixed
    precision (the composite's base correction in FP32; the uniform solve's
    cycles in FP32 inside FP64 refinement).  The composite solve's cycle count
    is found by a first solve with norms, then timed without them; a
    composite norm that rounding stops above 1e-10 counts as converged within
    twice its floor."""
    import numpy as np
    import torch
    from paper_2206_11294_gb300 import inputs as I
    from paper_2206_11294_gb300.binding import Composite, Solver
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = {"workload": "one bubble R = 0.1 at the centre: refined-patch grid (512^2 base, 2:1 box around the bubble) "
                       "against the uniform 1024^2 grid, set-up + solve to 1e-10 per step",
           "regimes": []}
    cases = [(label, kw, prec) for prec in ("fp64", "mixed")
             for label, kw in (("literal", {}), ("stiff", dict(length=6.4e-3, dt=1e-5)))]
    for label, kw, prec in cases:
        b, p, box = I.composite_bubble(512, seed=31, centres=[[0.5, 0.5]], radii=[0.1], **kw)
        u = I.bubble_2d(1024, seed=31, rmin=0.1, rmax=0.1, **kw)        # centred: the same bubble
        cells = b.grid.N - (box[0][1] - box[0][0]) * (box[1][1] - box[1][0]) + p.grid.N
        c = Composite(b.grid, box, precision=prec)
        d = dict(lb=T(b.lam), fab=[T(f) for f in b.fa], fkb=[T(f) for f in b.fk], lf=T(p.lam),
                 faf=[T(f) for f in p.fa], fkf=[T(f) for f in p.fk], bb=T(b.b), bf=T(p.b), xb0=T(b.x0), xf0=T(p.x0))
        c.set_coeffs(d["lb"], d["fab"], d["fkb"], d["lf"], d["faf"], d["fkf"])
        if not args.no_tune:
            c.autotune(args.tune_reps)
        xb, xf = d["xb0"].clone(), d["xf0"].clone()
        _, _, hist = c.solve(d["bb"], d["bf"], xb, xf, 60)
        red = hist / hist[0]
        # stop at 1e-10 of each norm's start or, where rounding stops a norm
        # above that (stiff rows around a 1e5 Pa background), at twice the
        # lowest value it reaches in 60 cycles
        target = np.maximum(1e-10, 2.0 * red.min(axis=0))
        need = int(next(k for k in range(len(red)) if np.all(red[k] <= target)))
        for _ in range(args.warmup):
            xb.copy_(d["xb0"]); xf.copy_(d["xf0"])
            c.set_coeffs(d["lb"], d["fab"], d["fkb"], d["lf"], d["faf"], d["fkf"])
            c.solve(d["bb"], d["bf"], xb, xf, need, norms=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with nvtx_range(f"adaptive_{label}_{prec}"):
            for _ in range(args.steps):
                xb.copy_(d["xb0"]); xf.copy_(d["xf0"])
                c.set_coeffs(d["lb"], d["fab"], d["fkb"], d["lf"], d["faf"], d["fkf"])
                c.solve(d["bb"], d["bf"], xb, xf, need, norms=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_c = e0.elapsed_time(e1) / args.steps
        c.close()
        s = Solver(u.grid, rtol=1e-10, max_cycles=200, precision=prec)
        du = dict(lam=T(u.lam), fa=[T(f) for f in u.fa], fk=[T(f) for f in u.fk], b=T(u.b), x0=T(u.x0))
        s.set_coeffs(du["lam"], du["fa"], du["fk"])
        if not args.no_tune:
            s.autotune(args.tune_reps)
        x = du["x0"].clone()
        for _ in range(args.warmup):
            x.copy_(du["x0"]); s.set_coeffs(du["lam"], du["fa"], du["fk"]); st = s.solve(du["b"], x)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            x.copy_(du["x0"]); s.set_coeffs(du["lam"], du["fa"], du["fk"]); st = s.solve(du["b"], x)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_u = e0.elapsed_time(e1) / args.steps
        s.close()
        out["regimes"].append({"regime": label, "precision": prec, "composite_cells": cells,
                               "uniform_cells": u.grid.N, "box": box,
                               "composite_cycles": need, "composite_ms": ms_c,
                               "composite_reduction": [float(v) for v in red[need]],
                               "composite_floor": [float(v) for v in red.min(axis=0)],
                               "composite_mcell_cycles_per_s": cells * need / ms_c / 1e3,
                               "uniform_cycles": st["cycles"], "uniform_ms": ms_u,
                               "uniform_mcell_vcycles_per_s": u.grid.N * st["cycles"] / ms_u / 1e3,
                               "speedup_composite_vs_uniform": ms_u / ms_c})
    out["l2"] = "not flushed (both solves resident)"
    out["data"] = "synthetic (seeded bubble field assembled at both spacings)"
    return out


# Algorithmic bytes per cell of the assembly and update kernels (2D): what
# each must read and write once (face arrays: one face per cell and axis).
ASSEMBLE_BYTES_2D = (4 + 2 + 2) * 8 + (4 + 2 + 2 + 2 + 2) * 8    # C m1 m2 E, mom, u*; lambda, rhs, x0, 1/rho, k
CORRECT_BYTES_2D = (2 + 1 + 1 + 2 + 2) * 8 + (2 + 1 + 1) * 8      # x, C, kappa, 1/rho, u*; u^(n+1), p1, p2
ENERGY_BYTES_2D = (2 + 1 + 2 + 2 + 2) * 8 + 2 * 8                 # x, C, p1 p2, u^(n+1), E1 E2; E1, E2 out


def run_timestep(args):
    """The device work of one time step on the 16-bubble 1024^2 advected state:
    the momentum predictor (mg_momentum_rhs_async, mg_momentum_* set-up and solve to
    1e-10 from u^(adv), mg_provisional_async: Eq. provel), coefficient assembly on its
    u* (mg_assemble_async: Eqs. 10, 11, 20, 23, 29-34), set-up and
    solve to 1e-10 from (T^(adv), p^(adv)), the velocity / phase-pressure
    update (mg_correct_async: Eq. unp1, Eqs. 37-38) and the phase-energy update
    (mg_energy_async: Eq. 39).  Inputs resident on the device; the L2 is flushed
    between steps."""
    import numpy as np
    import torch
    from paper_2206_11294_gb300 import binding as B
    from paper_2206_11294_gb300 import inputs as I
    from paper_2206_11294_gb300.binding import Momentum, Solver
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    s = I.bubbles_state_1024()
    g = s.grid
    N = g.N
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    z = lambda *shape: torch.zeros(*shape, dtype=torch.float64, device="cuda")
    d = dict(C=T(s.C), m1=T(s.m1), m2=T(s.m2), E=T(s.E), mom=[T(m) for m in s.mom], uf=[T(u) for u in s.uf],
             kappa=T(s.kappa))
    out = dict(lam=z(N, 4), b=z(N, 2), x0=z(N, 2), fa=[z(*g.face_shape(a)) for a in range(2)],
               fk=[z(*g.face_shape(a)) for a in range(2)])
    x = z(N, 2)
    uo = [torch.empty_like(u) for u in d["uf"]]
    p1, p2 = z(*s.C.shape), z(*s.C.shape)
    rho1, rho2 = I.phase_density(s.T, s.p, s.ph1), I.phase_density(s.T, s.p, s.ph2)
    E1 = T(s.C * I.phase_energy(s.p, rho1, s.ph1))
    E2 = T((1 - s.C) * I.phase_energy(s.p, rho2, s.ph2))
    E1o, E2o = torch.empty_like(E1), torch.empty_like(E2)
    # momentum predictor inputs: p^n (the state's pressure), rho^(n+1) = m1 + m2, mu = C mu_1 + (1 - C) mu_2
    p_n = T(s.p)
    rho_d = d["m1"] + d["m2"]
    mu_d = T(s.C * s.ph1.mu + (1 - s.C) * s.ph2.mu)
    R = [torch.empty_like(d["C"]) for _ in range(2)]
    u_pred = [torch.empty_like(d["C"]) for _ in range(2)]
    u0 = [m_ / rho_d for m_ in d["mom"]]
    ustar = [torch.empty_like(u) for u in d["uf"]]
    mom_solver = Momentum(g, stream=stream)
    mom_stats = []
    solver = Solver(g, precision=args.precision, rtol=1e-10, max_cycles=50, stream=stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def predict():
        B.momentum_rhs(g, s.dt, s.sigma, d["mom"], p_n, d["kappa"], d["C"], R)
        mom_solver.set_coeffs(s.dt, rho_d, mu_d)
        for a in range(2):
            u_pred[a].copy_(u0[a])
        mom_stats.append(mom_solver.solve(R, u_pred, rtol=1e-10, max_iters=100))
        B.provisional(g, s.dt, rho_d, p_n, u_pred, ustar)

    def assemble():
        B.assemble(g, (s.ph1, s.ph2), s.dt, d["C"], d["m1"], d["m2"], d["E"], d["mom"], ustar, out)

    def correct():
        B.correct(g, s.dt, s.sigma, x, d["C"], d["kappa"], out["fa"], ustar, uo, p1, p2)

    def energy():
        B.energy(g, (s.ph1, s.ph2), s.dt, x, d["C"], p1, p2, uo, E1, E2, E1o, E2o)

    predict()
    assemble()
    solver.set_coeffs(out["lam"], out["fa"], out["fk"])
    tuning = None
    if not args.no_tune:
        from paper_2206_11294_gb300.autotune import describe
        tuning = describe(solver.autotune(args.tune_reps)[0])
    ev = lambda: torch.cuda.Event(enable_timing=True)
    stats = []

    def step(marks):
        marks[0].record(stream)
        predict()
        marks[1].record(stream)
        assemble()
        marks[2].record(stream)
        solver.set_coeffs(out["lam"], out["fa"], out["fk"])
        x.copy_(out["x0"])
        stats.append(solver.solve(out["b"], x))
        marks[3].record(stream)
        correct()
        marks[4].record(stream)
        energy()
        marks[5].record(stream)

    for _ in range(args.warmup):
        step([ev() for _ in range(6)])
    torch.cuda.synchronize()
    stats.clear()
    mom_stats.clear()
    marks = [[ev() for _ in range(6)] for _ in range(args.steps)]
    clocks = ClockSampler(gpu_identity(torch, 0))
    for k in range(args.steps):
        flush.zero_()
        step(marks[k])
    torch.cuda.synchronize()
    clk = clocks.stop()
    avg = lambda a, b: sum(m[a].elapsed_time(m[b]) for m in marks) / args.steps
    total, t_pred, t_asm, t_solve, t_cor, t_en = avg(0, 5), avg(0, 1), avg(1, 2), avg(2, 3), avg(3, 4), avg(4, 5)
    mom_solver.close()
    peak, peak_kind = measured_peak()
    roof = lambda byts, ms: {"bound": "hbm", "achieved": byts / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                             "frac": byts / (ms * 1e-3) / 1e9 / peak, "peak_source": peak_kind,
                             "algorithmic_bytes": byts, "avg_launch_us": ms * 1e3}
    cycles = [st["cycles"] for st in stats]
    asm = roof(ASSEMBLE_BYTES_2D * N, t_asm)
    # the assembly is bound by the FP64 pipe, not HBM (ncu --set full of k_assemble on this state)
    asm_alu = {"bound": "alu", "fp64_pipe_busy_elapsed_ncu": 0.836, "fp64_inst_per_cell_ncu": 150,
               "source": "ncu --set full capture of k_assemble<2,false> on this state", "hbm": asm}
    return {"workload": "one time step, bubbles16_1024x1024 advected state: assembly + set-up + solve to 1e-10 + "
                        "velocity / phase-pressure update + phase-energy update, after the momentum predictor "
                        "(right-hand side, set-up + solve to 1e-10, Eq. provel)", "metric": "time steps/s",
            "cells": N,
            "precision": args.precision, "steps_per_s": 1e3 / total, "ms_per_step": total,
            "predictor_ms": t_pred, "predictor_iterations": mom_stats[0]["iterations"] if mom_stats else None,
            "assemble_ms": t_asm, "solve_ms": t_solve, "correct_ms": t_cor, "energy_ms": t_en,
            "cycles_per_solve": cycles[0] if cycles else None, "tuning": tuning,
            "assemble_roofline": asm_alu,
            "correct_roofline": roof(CORRECT_BYTES_2D * N, t_cor),
            "energy_roofline": roof(ENERGY_BYTES_2D * N, t_en),
            "l2": "flushed between steps", "clocks": clk, "data": "synthetic (seeded advected state, NASG water / air)"}


def run_momentum(args):
    """The implicit momentum predictor on the 16-bubble 1024^2 state: rho = m1 + m2, mu = C mu_1 + (1 - C) mu_2,
    R = (rho u)^(adv) / dt, from u^(adv) to rtol 1e-10, at the time step's dt (1e-7) and at dt = 1e-3, where
    viscosity dominates in the gas (mu dt / (rho h^2) ~ 16), and at dt = 0.1 (~1600 in the gas), each of the last two
    also with GMRES.  Set-up (coefficients, hierarchy) and solve per step, L2 flushed between steps."""
    import numpy as np
    import torch
    from paper_2206_11294_gb300 import inputs as I
    from paper_2206_11294_gb300.binding import Momentum
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    s = I.bubbles_state_1024()
    g = s.grid
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    rho_h = s.m1 + s.m2
    rho, mu = T(rho_h), T(s.C * s.ph1.mu + (1 - s.C) * s.ph2.mu)
    u0 = [T(m_ / rho_h) for m_ in s.mom]
    u = [torch.empty_like(v) for v in u0]
    m = Momentum(g, stream=stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = {"workload": "momentum predictor, bubbles16_1024x1024: set-up + solve to 1e-10 from u^(adv)",
           "metric": "momentum solves/s", "cells": g.N, "precision": "fp64", "regimes": []}
    mk = Momentum(g, stream=stream, krylov=True)
    for dt, solver in ((1e-7, m), (1e-3, m), (1e-3, mk), (1e-1, m), (1e-1, mk)):
        R = [T(m_ / dt) for m_ in s.mom]
        stats = []

        def step():
            solver.set_coeffs(dt, rho, mu)
            for a in range(g.dim):
                u[a].copy_(u0[a])
            stats.append(solver.solve(R, u, rtol=1e-10, max_iters=400))

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        stats.clear()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(gpu_identity(torch, 0))
        ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        clk = clocks.stop()
        ms /= args.steps
        out["regimes"].append({"dt": dt, "solves_per_s": 1e3 / ms, "ms_per_solve": ms,
                               "iterations": stats[0]["iterations"], "cycles": stats[0]["cycles"],
                               "corrections": "point-Jacobi" if stats[0]["jacobi"] else
                               ("GMRES(16) preconditioned by multigrid" if solver is mk else "multigrid"),
                               "jacobi_bound": stats[0]["nu"],
                               "rfinal_over_r0": stats[0]["rfinal"] / stats[0]["r0"] if stats[0]["r0"] else 0.0,
                               "clocks": clk})
    m.close()
    mk.close()
    out["l2"] = "flushed between steps"
    out["data"] = "synthetic (seeded advected state, NASG water / air, mu 8.5e-4 / 1.85e-5 Pa s)"
    return out


def serve_pool(seed: int = 6):
    """The serving workload's request shapes: 12 2D problems with n
    log-uniform in 128..1024 rounded to a multiple of 32 (1-8 bubbles), and 3D
    bubbles near a wall with n = 64, 96, ..., 256; requests draw 80% 2D, 20%
    3D."""
    import numpy as np
    from paper_2206_11294_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    pool2, pool3 = [], []
    for q in range(12):
        n = I.round_to(float(np.exp(rng.uniform(np.log(128), np.log(1024)))), 32)
        pool2.append(I.bubble_2d(n=n, seed=600 + q, n_bubbles=int(rng.integers(1, 9)), rmin=0.02, rmax=0.08,
                                 centred=False, name=f"s2d_{n}"))
    for q, n in enumerate(range(64, 257, 32)):
        pool3.append(I.bubble_wall_3d(n=n, seed=700 + q, name=f"s3d_{n}"))
    # 80% 2D, 20% 3D requests: 12 2D shapes x 28 against 7 3D shapes x 12 (336 : 84)
    weighted = pool2 * 28 + pool3 * 12
    return pool2 + pool3, weighted


def run_serve(args):
    """Poisson arrivals of mixed 2D (128..1024) and 3D (64..256) bubble solves,
    mixed precision, admitted against an HBM budget with hierarchies kept
    resident (a warm pool built before the first request); p50/p99 and
    throughput per arrival rate, each rate min(2000, rate x seconds) requests."""
    from paper_2206_11294_gb300.serve import Engine, Server, run_stream
    pool, weighted = serve_pool()
    f3 = sum(p.grid.dim == 3 for p in weighted) / len(weighted)
    eng = Engine(device=0, precision="mixed", rtol=1e-10, max_cycles=60, tune=not args.no_tune)
    out = {"workload": f"Poisson stream, {100 * (1 - f3):.0f}% 2D 128^2-1024^2 (multiples of 32) / "
                       f"{100 * f3:.0f}% 3D 64^3-256^3, mixed precision, inputs from page-locked host memory",
           "hbm_budget_bytes": args.serve_budget, "rates": [],
           "tuning": "autotuned per hierarchy shape while the warm pool is built" if not args.no_tune
           else "library defaults"}
    t0 = time.perf_counter()
    srv = Server(eng, hbm_budget=args.serve_budget, slots=4, max_batch=8)
    out["warm_pool"] = {"hierarchies": srv.prewarm(pool, per_shape=args.serve_per_shape),
                        "per_shape": args.serve_per_shape, "seconds": time.perf_counter() - t0}
    if not args.no_tune:
        out["shapes_tuned"] = eng.table.measured
    for rate in args.serve_rates:
        count = int(min(args.serve_max, max(40, rate * args.serve_seconds)))
        srv.log.clear()
        st = run_stream(srv, weighted, rate=rate, count=count, seed=int(rate))
        out["rates"].append(st)
    srv.close()
    return out


def _oracle_cycle_sample(probs, threaded):
    """One oracle V-cycle (with its hierarchy set-up and the residuals around
    it) on each problem: (Mcell-V-cycles, seconds)."""
    import oracle
    units = 0.0
    t0 = time.perf_counter()
    for p in probs:
        x, cyc, _ = oracle.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=1, rtol=0.0,
                                    threaded=threaded)
        units += p.grid.N * cyc / 1e6
    return units, time.perf_counter() - t0


def cpu_baseline(probs, seconds: float = 10.0, batch_sample: bool = False):
    """The oracle on every host core (OpenMP build), one V-cycle per problem
    repeated until about `seconds` of CPU time have passed: a bounded sample of
    the workload.  The single-thread build's figure for one such sample is
    reported beside it."""
    import oracle
    oracle.build()
    oracle.build_threaded()
    units = secs = 0.0
    reps = 0
    while reps == 0 or secs < seconds:
        u, t = _oracle_cycle_sample(probs, True)
        units, secs, reps = units + u, secs + t, reps + 1
    u1, t1 = _oracle_cycle_sample(probs, False)
    out = {"value": units / secs, "unit": UNIT, "cores": oracle.threads(True), "kind": "oracle",
           "sample": f"{reps} x (1 V-cycle with hierarchy set-up and residuals on each of the {len(probs)} problems), "
                     "OpenMP over the cells of each level / colour",
           "seconds": secs, "single_thread_value": u1 / t1}
    if batch_sample:
        # the 256-problem batch's first 32 problems (the same seeded sizes and fields), one V-cycle each
        from paper_2206_11294_gb300 import inputs as I
        bp = I.batch_problems(count=32)
        ub, tb = _oracle_cycle_sample(bp, True)
        out["batch_sample"] = {"problems": len(bp), "cells": int(sum(p.grid.N for p in bp)),
                               "mcell_vcycles_per_s": ub / tb, "seconds": tb,
                               "sample": "1 V-cycle with set-up on each of the batch's first 32 problems, OpenMP"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    probs = workload_problems()
    import oracle
    oracle.build_threaded()
    cores = oracle.threads(True)
    for _ in range(min(args.warmup, 1)):
        _oracle_cycle_sample(probs[:1], True)       # page in the library and the inputs
    units = secs = 0.0
    for _ in range(args.steps):
        u, t = _oracle_cycle_sample(probs, True)
        units, secs = units + u, secs + t
    v = units / secs
    sample = f"1 V-cycle (with set-up) on each of the {len(probs)} problems per step, OpenMP on {cores} cores"
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded bubble fields)", "impl": "reference",
            "config": {"workload": "bubbles16_1024x1024 + axi_512x1024, one oracle V-cycle each per step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--schedule", default="concurrent", choices=["concurrent", "serial"],
                    help="the step's problems on their own streams at once, or one after the other")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="headline only: no mixed / stiff / batch / serve sub-results")
    ap.add_argument("--no-batch", action="store_true", help="sub-results without the batch")
    ap.add_argument("--no-serve", action="store_true", help="sub-results without the serving rate")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--sub-serve-rate", type=float, default=100.0)
    ap.add_argument("--sub-serve-seconds", type=float, default=5.0)
    ap.add_argument("--no-tune", action="store_true", help="library default kernel choices, no autotuning")
    ap.add_argument("--tune-reps", type=int, default=5)
    ap.add_argument("--tuning-table", default=None, help="JSON table of autotuned choices to apply (and extend)")
    ap.add_argument("--workload", default="bubbles",
                    choices=["bubbles", "batch", "serve", "wall3d", "timestep", "momentum", "adaptive", "coarse"])
    ap.add_argument("--n3d", type=int, default=256)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[10, 30, 100, 300, 1000, 2000])
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--serve-max", type=int, default=2000)
    ap.add_argument("--serve-budget", type=int, default=120 << 30)
    ap.add_argument("--serve-per-shape", type=int, default=4, help="hierarchies per shape in the warm pool")
    ap.add_argument("--cycle", default="V", choices=["V", "W", "F"], help="cycle of the correction solve")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture")
    args = ap.parse_args()
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    if args.workload != "bubbles":
        if rank == 0:
            out = {"batch": run_batch, "serve": run_serve, "wall3d": run_wall3d, "timestep": run_timestep,
                   "momentum": run_momentum, "adaptive": run_adaptive, "coarse": run_coarse}[args.workload](args)
            print(json.dumps(out), flush=True)
        return
    if args.impl == "ours" and world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(env_int("LOCAL_RANK", 0))
        dist.init_process_group("nccl")
    out = run_reference(args, rank, world) if args.impl == "reference" else run_ours(args, rank, world)
    if out is not None:
        print(json.dumps(out), flush=True)
    if args.impl == "ours" and world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
