#!/usr/bin/env python
"""Benchmark of the analytic-pulse gather + relativistic Boris push.

Workload (one GPU): the Gaussian-beam workload -- 1e7 electrons at rest in a
20 x 20 x 40 lambda box, paraxial Gaussian w0 = 3 lambda, a0 = 10, Gaussian
envelope (intensity FWHM 30), first-order longitudinal fields, plus a 256^3
static FP32 grid field gathered trilinearly; 4000 Boris steps of dt = 0.02,
float arithmetic with a float-float phase argument and position.

One bench step = restore the initial particle state (device copy) + one
ap_gather_push call that advances all 1e7 particles by 4000 fused steps.
The metric is particle-steps per second; inputs (360 MB of particle state,
402 MB of grid) exceed the 126 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU, each rank pushing its own
1e7-particle shard (weak scaling, no data-path collective); rank 0 prints
one JSON line.  --impl reference times the CPU oracle on the host cores.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (analytic field+Boris)"
UNIT = "particle-steps/s"

# FP32-pipe operations per particle-step of the float-float Gaussian + grid
# kernel, counted from the formulas the kernel evaluates (see the design doc,
# "Roofline"): phase unit 65, envelope 2, Gaussian profile with longitudinal
# terms and field assembly 57, trilinear gather from the cached cell 72,
# Boris rotation 42, float-float position update 27.
ALGO_FP32_OPS = 265
ALGO_MUFU_OPS = 7
SM_COUNT = 152
FP32_LANES = 128      # FP32 operations per clock per SM
MUFU_LANES = 16       # special-function operations per clock per SM
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None, help="particles per GPU (default 1e7)")
    ap.add_argument("--nsteps", type=int, default=None, help="Boris steps per call (default 4000)")
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="core-seconds of oracle work")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- helpers

def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_rate(cfg, parts, grid_np, lo, hi, n_steps, core_seconds, threads):
    """CPU oracle throughput on a bounded sample of the workload's particles:
    a probe sizes the sample to about `core_seconds` of single-core work."""
    import oracle
    probe_n, probe_steps = 8, 200
    sub = {k: v[:probe_n] for k, v in parts.items()}
    t = time.perf_counter()
    oracle.push(cfg["pulse"], sub, cfg["t0"], cfg["dt"], probe_steps, grid=(grid_np, lo, hi))
    per = (time.perf_counter() - t) / (probe_n * probe_steps)
    m = int(max(threads, min(len(parts["x"]), core_seconds / (per * n_steps))))
    m = max(threads, (m // threads) * threads)
    sub = {k: v[:m] for k, v in parts.items()}
    t = time.perf_counter()
    oracle.push(cfg["pulse"], sub, cfg["t0"], cfg["dt"], n_steps, grid=(grid_np, lo, hi), threads=threads)
    wall = time.perf_counter() - t
    return m * n_steps / wall, m, wall


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2307_04843_gb300 import _lib, workloads

    ws, rank, local = dist_info()
    if ws != args.gpus and args.gpus != 1:
        pass
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cfg = workloads.config(2)
    n = args.n or cfg["n"]
    n_steps = args.nsteps or cfg["n_steps"]
    t0, dt = cfg["t0"], cfg["dt"]
    parts = workloads.particles(cfg, n=n, seed=workloads.seed_for(2) + 7919 * rank)
    lo, hi = workloads.grid_box(cfg)
    grid = workloads.grid_field(cfg["box"], args.grid, torch_device="cuda")
    stream = torch.cuda.current_stream()

    h = _lib.Handle(cfg["pulse"])
    init = _lib.to_device(parts, "fp32")
    work = {k: v.clone() for k, v in init.items()}
    g = (grid, lo, hi)

    def step():
        for k in work:
            work[k].copy_(init[k], non_blocking=True)
        h.push(work, t0, dt, n_steps, precision="fp32", grid=g)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if h.status() != 0:
        raise RuntimeError("device status after warm-up: %d" % h.status())

    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    e0.record(stream)
    for k in range(args.steps):
        for kk in work:
            work[kk].copy_(init[kk], non_blocking=True)
        kev[k][0].record(stream)
        h.push(work, t0, dt, n_steps, precision="fp32", grid=g)
        kev[k][1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if ws > 1:
        dist.barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    kern = sum(a.elapsed_time(b) for a, b in kev) / 1e3 / args.steps
    tt = torch.tensor([elapsed, kern], dtype=torch.float64, device="cuda")
    if ws > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    elapsed, kern = float(tt[0]), float(tt[1])
    status = h.status()
    if status != 0:
        raise RuntimeError("device status after timed steps: %d" % status)
    units = float(n) * n_steps * args.steps * ws
    value = units / elapsed

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        host = {k: v.cpu().pin_memory() for k, v in init.items()}
        out = {k: torch.empty_like(v).pin_memory() for k, v in host.items()}
        dev = {k: torch.empty_like(v) for k, v in init.items()}
        h2d = sum(v.numel() * v.element_size() for v in host.values())

        def e2e_step():
            for k in dev:
                dev[k].copy_(host[k], non_blocking=True)
            h.push(dev, t0, dt, n_steps, precision="fp32", grid=g)
            for k in dev:
                out[k].copy_(dev[k], non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        te = torch.tensor([a.elapsed_time(b) / 1e3], dtype=torch.float64, device="cuda")
        if ws > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": units / float(te[0]), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(h2d)}

    # comparison variants on one GPU: native-FP64-phase and plain FP64 paths
    variants = {}
    if rank == 0 and not args.no_variants:
        for prec, nv, sv in (("fp32_phase64", min(n, 2_000_000), n_steps), ("fp64", min(n, 500_000), n_steps)):
            sub = {k: v[:nv] for k, v in parts.items()}
            d0 = _lib.to_device(sub, prec)
            d1 = {k: v.clone() for k, v in d0.items()}
            h.push(d1, t0, dt, 200, precision=prec, grid=g)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.push(d0, t0, dt, sv, precision=prec, grid=g)
            b.record(stream)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) / 1e3
            variants[prec] = {"value": nv * sv / sec, "unit": UNIT,
                              "sample": "%d particles x %d steps, one call" % (nv, sv)}
        for prec in variants:
            variants[prec]["fp32_speedup"] = (units / ws / args.steps / kern) / variants[prec]["value"]

    # CPU oracle baseline on rank 0 (bounded sample of the same workload)
    cpu = None
    if rank == 0 and not args.no_cpu:
        threads = os.cpu_count() or 1
        rate, m, wall = oracle_rate(cfg, parts, grid.cpu().numpy(), lo, hi, n_steps, args.cpu_seconds, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "first %d particles of the workload x %d steps (%.1f s wall)" % (m, n_steps, wall)}

    # roofline of the push kernel (FP32 pipe)
    sm_mhz = SM_MAX_MHZ
    peak_ops = SM_COUNT * FP32_LANES * sm_mhz * 1e6 / 1e12  # TOP/s
    achieved = ALGO_FP32_OPS * (float(n) * n_steps / kern) / 1e12
    roofline = {"bound": "alu", "pipe": "fp32", "achieved": achieved, "peak": peak_ops, "unit": "TOP/s",
                "frac": achieved / peak_ops, "traffic": None,
                "algo_ops_per_particle_step": ALGO_FP32_OPS, "kernel_ms": kern * 1e3,
                "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz (max SM clock)"}
    if ck and ck.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (SM_COUNT * FP32_LANES * ck["sm_mhz"] * 1e6 / 1e12)
        roofline["mufu_frac"] = (ALGO_MUFU_OPS * float(n) * n_steps / kern) / (SM_COUNT * MUFU_LANES * sm_mhz * 1e6)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded PCG64 particles and grid)",
        "config": {"workload": "gauss-grid: paraxial Gaussian w0=3 lambda a0=10 FWHM 30 + longitudinal, "
                               "256^3 FP32 grid, float-float phase",
                   "particles_per_gpu": n, "boris_steps_per_call": n_steps, "dt": dt, "grid": args.grid,
                   "l2": "inputs larger than L2 (36 B/particle state, 402 MB grid); no flush",
                   "parallelism": "dp%d (independent shards)" % ws},
        "gpu_launches": args.steps,
        "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": ck, "variants": variants,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------- reference arm

def run_reference(args):
    """The CPU oracle as it stands, on the host cores, same workload and
    metric; each step is a bounded sample of particles over all 4000 steps."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle
    from paper_2307_04843_gb300 import workloads
    cfg = workloads.config(2)
    n_steps = args.nsteps or cfg["n_steps"]
    lo, hi = workloads.grid_box(cfg)
    grid = workloads.grid_field(cfg["box"], args.grid)
    threads = os.cpu_count() or 1
    parts = workloads.particles(cfg, n=4096)
    # size one step to ~ (cpu_seconds / (steps + warmup)) core-seconds
    probe = {k: v[:8] for k, v in parts.items()}
    t = time.perf_counter()
    oracle.push(cfg["pulse"], probe, cfg["t0"], cfg["dt"], 100, grid=(grid, lo, hi))
    per = (time.perf_counter() - t) / 800
    budget = max(2.0, 120.0 / max(1, args.steps + args.warmup))  # wall seconds per step
    m = int(max(threads, min(4096, budget * threads / (per * n_steps))))
    m = max(threads, (m // threads) * threads)
    sub = {k: v[:m] for k, v in parts.items()}
    for _ in range(args.warmup):
        oracle.push(cfg["pulse"], {k: v[:threads] for k, v in sub.items()}, cfg["t0"], cfg["dt"], 10,
                    grid=(grid, lo, hi), threads=threads)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.push(cfg["pulse"], sub, cfg["t0"], cfg["dt"], n_steps, grid=(grid, lo, hi), threads=threads)
    wall = time.perf_counter() - t
    value = m * n_steps * args.steps / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded PCG64 particles and grid)",
        "config": {"workload": "gauss-grid: paraxial Gaussian w0=3 lambda a0=10 FWHM 30 + longitudinal, "
                               "256^3 FP32 grid (CPU FP64 oracle)",
                   "particles_per_step": m, "boris_steps_per_call": n_steps, "grid": args.grid},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "first %d particles of the workload x %d steps per step" % (m, n_steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_2307_04843_gb300 import build
        if not os.path.exists(build.LIB):
            build.build()
        run_ours(args)


if __name__ == "__main__":
    main()
