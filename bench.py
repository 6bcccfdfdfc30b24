#!/usr/bin/env python
"""Benchmark of the analytic-pulse gather + relativistic Boris push.

Default workload (one GPU): the Gaussian-beam workload -- 1e7 electrons at
rest in a 20 x 20 x 40 lambda box, paraxial Gaussian w0 = 3 lambda, a0 = 10,
Gaussian envelope (intensity FWHM 30), first-order longitudinal fields, plus
a 256^3 static FP32 grid field gathered trilinearly; 4000 Boris steps of
dt = 0.02, float arithmetic with a float-float phase argument and position.

One bench step = restore the initial particle state (device copy) + one
gather + push call that advances every particle by all its fused steps.  The
metric is particle-steps per second; the inputs (particle state, grid)
exceed the 126 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 1..5]

N > 1 runs under torchrun, one rank per GPU, each rank pushing its own
shard of the same size (weak scaling, no data-path collective); rank 0
prints one JSON line.  --impl reference times the CPU oracle on the host
cores.  --workload selects the other workloads (1 plane FP64, 3 inverse-
Compton LG with the gamma histogram, 4 flying focus, 5 batched sets in a
CUDA graph plus the adjoint).
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
SM_COUNT = 152
FP32_LANES = 128      # FP32 operations per clock per SM
MUFU_LANES = 16       # special-function operations per clock per SM
SM_MAX_MHZ = 2070.0

# FP32-pipe operations per particle-step, counted from the formulas each
# kernel evaluates, and MUFU operations.
# Workload 2 (Gaussian + longitudinal + grid, float-float phase): local
# coordinates and phase 34, envelope 2, Gaussian profile + longitudinal +
# assembly 28, trilinear gather from the cached cell 57, Boris 42,
# compensated position update 18, z for the gather 1.
ALGO = {
    1: dict(fp32=0, mufu=0, fp64=60),
    2: dict(fp32=182, mufu=7),
    3: dict(fp32=190, mufu=8),
    4: dict(fp32=2300, mufu=258),
    5: dict(fp32=125, mufu=7),
    6: dict(fp32=125, mufu=7),
}
# FP32 operations per particle-step of the adjoint of workload 5 (Gaussian,
# longitudinal terms, linear polarisation, no grid), from its formulas: the
# forward sweep 125, the recomputation 125 and the reverse step 307 (local
# coordinates and phase 34, envelope 2, field value 28, F = a0 f 4, the Boris
# cotangent 123, the closed-form field derivatives contracted with it 116).
ADJ_OPS = 557
# DRAM bytes per particle-step of the workload-2 push kernel from the committed
# ncu capture of the 1.6e6-particle x 4000-step case, scaled by particle-steps
# (an upper bound at 1e7 particles: more particles share each cached cell);
# None when the kernel changed after the capture.  The capture is of the
# two-particle kernel with the hybrid cell cache (the autotuner's choice).
TRAFFIC_PER_PARTICLE_STEP = {
    "nodes": None,
    "cells": 6.0486,  # (38.6484e9 read + 0.0626e9 written) / 6.4e9
    "arrays": None,
}
TRAFFIC_KERNEL = dict(pairs=1, grid_cache=2)  # the launch setting the capture was taken with


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=2, choices=[1, 2, 3, 4, 5, 6])
    ap.add_argument("--n", type=int, default=None, help="particles per GPU (default: the workload's)")
    ap.add_argument("--nsteps", type=int, default=None, help="Boris steps per call (default: the workload's)")
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--grid-layout", default="cells", choices=["cells", "nodes", "arrays"],
                    help="grid read by the push: per-cell coefficients, node-interleaved copy, "
                         "or the six component arrays")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--launch", default=None,
                    help="fixed launch shape BLOCK[,BLOCKS_PER_SM[,GRID_CACHE[,PAIRS[,TILE]]]] instead of "
                         "the autotuner's")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="wall seconds of oracle work on all host cores (cpu_baseline)")
    ap.add_argument("--lines-only", action="store_true",
                    help="run only the Sec. 4 lines, one split-line and one traditional-line call "
                         "(a small case for profiling); prints their rates")
    ap.add_argument("--legs-only", action="store_true",
                    help="run only the grid-node, 1-D Yee and Sec. 4 line calls of the bench (the grid_node "
                         "key; a case for profiling those kernels); prints their rates")
    ap.add_argument("--split-steps", type=int, default=200)
    ap.add_argument("--plasma-steps", type=int, default=2000)
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


def oracle_rate(pulse, parts, t0, dt, n_steps, wall_seconds, threads, grid=None):
    """CPU oracle throughput on a bounded sample of the workload's particles:
    a threaded probe sizes the sample to about `wall_seconds` on `threads`
    host cores."""
    import oracle
    # probe: 64 particles per core over all steps, then scale to the target
    probe_n = min(len(parts["x"]), 64 * threads)
    sub = {k: v[:probe_n] for k, v in parts.items()}
    t = time.perf_counter()
    oracle.push(pulse, sub, t0, dt, n_steps, grid=grid, threads=threads)
    wall0 = time.perf_counter() - t
    m = int(max(threads, min(len(parts["x"]), probe_n * wall_seconds / max(wall0, 1e-3))))
    m = max(threads, (m // threads) * threads)
    sub = {k: v[:m] for k, v in parts.items()}
    t = time.perf_counter()
    oracle.push(pulse, sub, t0, dt, n_steps, grid=grid, threads=threads)
    wall = time.perf_counter() - t
    return m * n_steps / wall, m, wall


class Workload:
    """Device inputs and the step callable of one workload on this rank."""

    def __init__(self, idx, args, rank):
        import numpy as np
        import torch
        from paper_2307_04843_gb300 import _lib, shard, workloads
        self.idx = idx
        cfg = workloads.config(idx)
        self.cfg = cfg
        self.t0, self.dt = cfg["t0"], cfg["dt"]
        self.n_steps = args.nsteps or cfg["n_steps"]
        self.precision = cfg["precision"]
        self.grid = None
        self.grid_host = None
        self.diag = None
        self.graph = None
        seed = shard.shard_seed(workloads.seed_for(idx), rank)
        if idx == 5:
            sets, counts = workloads.batch_sets(cfg)
            if args.n:
                counts = workloads.scaled_counts(counts, args.n)
            off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
            self.n = int(off[-1])
            self.parts = workloads.particles_uniform(cfg["box"], self.n, seed)
            self.pulses = sets
            self.h = _lib.Handle(sets)
            self.off = torch.as_tensor(off).cuda()
            self.off_host = off
            self.ws = torch.zeros(_lib.ap_batch_workspace_bytes(self.h.h) // 4, dtype=torch.int32, device="cuda")
            self.diag = dict(set_sum=torch.zeros(len(sets), dtype=torch.float64, device="cuda"))
        elif idx == 6:
            per = max(1, args.n // cfg["n_sets"]) if args.n else None
            sets, self.parts, off = workloads.sweep_lines(cfg, per_set=per, seed=seed)
            self.n = int(off[-1])
            self.pulses = sets
            self.h = _lib.Handle(sets)
            self.off = torch.as_tensor(off).cuda()
            self.off_host = off
            self.ws = torch.zeros(_lib.ap_batch_workspace_bytes(self.h.h) // 4, dtype=torch.int32, device="cuda")
            self.diag = dict(set_sum=torch.zeros(len(sets), dtype=torch.float64, device="cuda"))
        else:
            self.n = args.n or cfg["n"]
            self.parts = workloads.particles(cfg, n=self.n, seed=seed)
            self.pulses = [cfg["pulse"]]
            self.h = _lib.Handle(cfg["pulse"])
            if idx == 1:
                self.diag = dict(lightfront=torch.zeros(self.n_steps, dtype=torch.float64, device="cuda"))
            if idx == 3:
                d = cfg["diag"]
                self.diag = dict(hist=torch.zeros(d["hist_bins"], dtype=torch.int32, device="cuda"),
                                 hist_lo=d["hist_lo"], hist_hi=d["hist_hi"])
        if cfg.get("grid") is not None:
            lo, hi = workloads.grid_box(cfg)
            g = workloads.grid_field(cfg["box"], args.grid, torch_device="cuda")
            self.grid = (g, lo, hi) if args.grid_layout == "arrays" else \
                _lib.pack_grid((g, lo, hi), layout=args.grid_layout)
            self.grid_host = (g, lo, hi)
        self.init = _lib.to_device(self.parts, self.precision)
        self.work = {k: v.clone() for k, v in self.init.items()}
        self.tuned = None
        if args.launch:
            shape = [int(v) for v in args.launch.split(",")] + [0, 0, 0, 0]
            self.h.set_launch(shape[0], shape[1], shape[2], shape[3], shape[4])
            self.tuned = {"block": shape[0], "blocks_per_sm": shape[1], "grid_cache": shape[2],
                          "pairs": shape[3], "tile": shape[4], "fixed": True}
        elif not args.no_autotune and idx not in (5, 6):
            from paper_2307_04843_gb300 import autotune
            self.tuned = autotune.tune(self.h, self.init, self.t0, self.dt, self.precision, self.grid,
                                       sample_n=min(self.n, 2_000_000), sample_steps=min(self.n_steps, 200))
        elif not args.no_autotune:
            from paper_2307_04843_gb300 import autotune
            self.tuned = autotune.tune_batched(self.h, self.init, self.off, self.t0, self.dt, self.precision,
                                               self.grid, self.diag, sample_steps=min(self.n_steps, 100))
        if idx in (5, 6):
            self.stream = torch.cuda.Stream()
            self.graph = _lib.ap_batch_graph_create(self.h.h, self.work, self.off, None, self.t0, self.dt,
                                                    self.n_steps, self.precision, self.diag, self.ws,
                                                    self.stream)

    def restore(self):
        for k in self.work:
            self.work[k].copy_(self.init[k], non_blocking=True)

    def push(self):
        import torch
        from paper_2307_04843_gb300 import _lib
        if self.graph is not None:
            cur = torch.cuda.current_stream()
            self.stream.wait_stream(cur)
            _lib.ap_graph_launch(self.graph, self.stream)
            cur.wait_stream(self.stream)
        else:
            self.h.push(self.work, self.t0, self.dt, self.n_steps, precision=self.precision, grid=self.grid,
                        diag=self.diag)

    def close(self):
        from paper_2307_04843_gb300 import _lib
        if self.graph is not None:
            _lib.ap_graph_destroy(self.graph)
            self.graph = None
        self.h.close()


def describe(wl, args):
    c = wl.cfg
    names = {1: "plane-fp64: LP plane wave a0=1, sin^2 10 cycles, 1e4 e- at rest, FP64",
             2: "gauss-grid: paraxial Gaussian w0=3 lambda a0=10 FWHM 30 + longitudinal, "
                "256^3 FP32 grid, float-float phase",
             3: "ics-lg12: CP LG_{1,2} w0=2 lambda a0=20 sin^2 20 cycles, gamma~1000 beam, "
                "1024-bin gamma histogram, float-float phase",
             4: "flying-focus: 64 Gaussian spectral components, v_f=0.99, a0=5, float-float phase",
             5: "batched-gauss: 256 Gaussian sets, log-uniform counts, one persistent launch in a CUDA graph, "
                "per-set mean gamma, float-float phase",
             6: "ics-sweep-1d3v: 30 radii x 1e5 electrons (gamma 5088, 1D-3V) in a Gaussian a0=50, "
                "w0=2.55 lambda, 15 fs, one batched launch in a CUDA graph, float-float phase"}
    cfg = {"workload": names[wl.idx], "particles_per_gpu": wl.n, "boris_steps_per_call": wl.n_steps,
           "dt": c["dt"], "l2": "inputs larger than L2 (36 B/particle state%s); no flush" %
           ((", 402 MB grid" + {"cells": " + 3.2 GB cell-coefficient copy",
                                "nodes": " + 537 MB node-interleaved copy", "arrays": ""}[args.grid_layout])
            if wl.grid is not None else ""),
           "parallelism": "dp%d (independent shards)" % dist_info()[0]}
    if wl.grid is not None:
        cfg["grid"] = args.grid
        cfg["grid_layout"] = {"cells": "per-cell trilinear coefficients (ap_grid_pack, AP_PACK_CELLS)",
                              "nodes": "node-interleaved (ap_grid_pack, AP_PACK_NODES)",
                              "arrays": "six component arrays"}[args.grid_layout]
    if wl.tuned:
        cfg["launch"] = launch_desc(wl)
    return cfg


def launch_desc(wl):
    t = wl.tuned or {}
    gc = t.get("grid_cache", 0)
    pairs = t.get("pairs", 0)
    d = {"block": t.get("block"), "blocks_per_sm": t.get("blocks_per_sm"),
         "particles_per_thread": 2 if pairs else 1,
         "grid_cache": None if wl.grid is None else
         ("first particle's cell in registers, second's in shared memory" if pairs and gc == 2 else
          "registers" if gc else "shared memory"),
         "autotuned": bool(t) and not t.get("fixed", False)}
    if wl.graph is not None or wl.idx in (5, 6):
        d["tile"] = t.get("tile") or (t.get("block") or 128) * (2 if pairs else 1)
    return d


# ---------------------------------------------------------------- our arm

NODE_N = 256           # staggered grid edge for the node-evaluation rate
# FP32 operations of the Gaussian (longitudinal terms on) on the six
# staggered positions of the nodes: the position part once per component of a
# node (transverse exponent, angle and its reduction, complex assembly, the one
# component written: 21).  The z/t part (float-float carrier phase and
# envelope argument 32, envelope 2, q = 1/(1 - i zeta) 3, for each of the two
# z levels) is computed once per z index per warp's run of rows: fewer than
# 0.01 operations per node, not counted.
NODE_OPS_PER_NODE = 6 * 21
NODE_OPS_PER_ROW = 0
YEE_LINES, YEE_NZ, YEE_STEPS = 152, 8192, 2000
# 1-D lines with a cold-plasma current (Sec. 4): n_e = 1e-3 n_c, a g = 4
# super-Gaussian of tau = 30 at 20 cells per wavelength, c dt/dz = 0.9
LINE_LINES, LINE_NZ, SPLIT_STEPS, PLASMA_STEPS = 304, 4096, 2000, 20000
SPLIT_MUFU_PER_NODE_STEP = 6  # E1: ex2, sin, cos; J1: ex2 and the sin, cos of its phase shift (its
                              # carrier is E1's rotated by omega dt/2)


def closed_form_rate(wl, stream, sum_rate):
    """The same electrons and steps under the closed-form flying focus
    (Sec. 3.3: one Gaussian whose focus moves at v_f) instead of the
    64-component sum: focus at the middle of the focal range at the time it
    is there, same a0, w0, v_f and longitudinal terms, no envelope."""
    import torch
    from paper_2307_04843_gb300 import _lib
    p = wl.pulses[0]
    zm = p["z_focus"] + 0.5 * p["ff_length"]
    tm = p["t_focus"] + 0.5 * p["ff_length"] / p["beta_f"]
    cf = dict(kind="flying_cf", pol=p.get("pol", "x"), env="cw", a0=p["a0"], w0=p["w0"], beta_f=p["beta_f"],
              z_focus=zm, t_focus=tm, longitudinal=p.get("longitudinal", False))
    with _lib.Handle(cf) as h:
        d = {k: v.clone() for k, v in wl.init.items()}
        h.push(d, wl.t0, wl.dt, 50, precision=wl.precision)
        for k in d:
            d[k].copy_(wl.init[k])
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.push(d, wl.t0, wl.dt, wl.n_steps, precision=wl.precision)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        st = h.status()
    if st != 0:
        raise RuntimeError("closed-form flying focus: device status %d" % st)
    rate = wl.n * wl.n_steps / sec
    return {"value": rate, "unit": UNIT, "sample": "the workload's %d electrons x %d steps" % (wl.n, wl.n_steps),
            "vs_64_component_sum": rate / sum_rate}


def grid_node_rates(wl, stream):
    """Rates of ap_eval_nodes (the workload's pulse onto a 256^3 Yee grid,
    six float arrays, float-float phase) and ap_yee1d_run (float lines)."""
    import torch
    from paper_2307_04843_gb300 import _lib

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / reps

    n = NODE_N
    f = [torch.empty((n, n, n), dtype=torch.float32, device="cuda") for _ in range(6)]
    from paper_2307_04843_gb300 import workloads
    lo, hi = workloads.grid_box(wl.cfg)
    d = tuple((hi[a] - lo[a]) / (n - 1) for a in range(3))
    sec = timed(lambda: wl.h.eval_nodes(f, lo, d, 0.0, precision="fp32"), 3)
    nodes = float(n) ** 3
    bytes_ = 24.0 * nodes
    ops = NODE_OPS_PER_NODE * nodes + NODE_OPS_PER_ROW * float(n) ** 2
    peak_ops = SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6
    hbm = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hbm = float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        pass
    # a plane wave (fields depend on z and t only): one evaluation per row of
    # nodes, streamed along it; all six arrays written
    plane = dict(kind="plane", pol="x", env="sgauss", sg_order=4, env_len=30.0, a0=1.0)
    with _lib.Handle(plane) as hp:
        psec = timed(lambda: hp.eval_nodes(f, lo, d, 0.0, precision="fp32"), 3)
    del f
    E = torch.zeros((YEE_LINES, YEE_NZ), dtype=torch.float32, device="cuda")
    B = torch.zeros_like(E)
    E[:, YEE_NZ // 2] = 1.0
    ysec = timed(lambda: _lib.ap_yee1d_run(E, B, 0.05, 0.0475, YEE_STEPS), 2)
    del E, B
    lines = line_rates(SPLIT_STEPS, PLASMA_STEPS, timed)
    return {
        "eval_nodes": {"value": nodes / sec, "unit": "nodes/s", "ms": sec * 1e3,
                       "grid": "%d^3, 6 staggered components, float arrays, float-float phase" % n,
                       "alu_frac": ops / sec / peak_ops,
                       "hbm_frac": (bytes_ / sec / 1e9 / hbm) if hbm else None,
                       "ops_per_node": NODE_OPS_PER_NODE + NODE_OPS_PER_ROW / n, "bytes_per_node": 24},
        "eval_nodes_plane": {"value": nodes / psec, "unit": "nodes/s", "ms": psec * 1e3,
                             "grid": "%d^3, 6 staggered components, float arrays, plane wave" % n,
                             "hbm_frac": (bytes_ / psec / 1e9 / hbm) if hbm else None,
                             "bytes_per_node": 24},
        "yee1d": {"value": YEE_LINES * YEE_NZ * YEE_STEPS / ysec, "unit": "node-steps/s",
                  "ms": ysec * 1e3, "lines": YEE_LINES, "nz": YEE_NZ, "steps": YEE_STEPS,
                  "dtype": "f32"},
        **lines,
    }


def line_rates(split_steps, plasma_steps, timed=None):
    """Rates of the Sec. 4 lines: the split line with E1, J1 evaluated in the
    kernel every step (ap_apt1d_run) and the traditional Yee + current line
    (ap_plasma1d_run), float, LINE_LINES x LINE_NZ.  timed(fn, reps) times
    repetitions after a warm-up call; without it each runs once."""
    import torch
    from paper_2307_04843_gb300 import _lib

    def once(fn, reps):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    timed = timed or once
    wp = math.sqrt(1e-3)
    dzl = 2.0 * math.pi / 20.0
    dtl = 0.9 * dzl
    sp = dict(kind="plane", pol="x", env="sgauss", sg_order=4, env_len=30.0, a0=1.0, omega_p=wp,
              yee=True, yee_dx=dzl, yee_dt=dtl)
    E = torch.zeros((LINE_LINES, LINE_NZ), dtype=torch.float32, device="cuda")
    B, J = torch.zeros_like(E), torch.zeros_like(E)
    z0 = -0.5 * LINE_NZ * dzl
    with _lib.Handle(sp) as hs:
        ssec = timed(lambda: hs.apt1d(E, B, J, z0, dzl, 0.0, dtl, split_steps, omega_p=wp), 2)
        if hs.status() != 0:
            raise RuntimeError("device status after the split line")
    tsec = timed(lambda: _lib.ap_plasma1d_run(E, B, J, dzl, dtl, plasma_steps, omega_p=wp), 2)
    split_rate = LINE_LINES * LINE_NZ * split_steps / ssec
    mufu_peak = SM_COUNT * MUFU_LANES * SM_MAX_MHZ * 1e6
    return {
        "apt1d_split": {"value": split_rate, "unit": "node-steps/s", "ms": ssec * 1e3,
                        "lines": LINE_LINES, "nz": LINE_NZ, "steps": split_steps, "dtype": "f32",
                        "mufu_frac": split_rate * SPLIT_MUFU_PER_NODE_STEP / mufu_peak,
                        "mufu_per_node_step": SPLIT_MUFU_PER_NODE_STEP},
        "plasma1d": {"value": LINE_LINES * LINE_NZ * plasma_steps / tsec, "unit": "node-steps/s",
                     "ms": tsec * 1e3, "lines": LINE_LINES, "nz": LINE_NZ, "steps": plasma_steps,
                     "dtype": "f32"},
    }

def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def roofline_frac(idx, rate):
    return ALGO[idx]["fp32"] * rate / (SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6)


def _auxiliary(fn, *args):
    """An auxiliary measurement of the line (grid-node legs, the other
    workloads): a failure there is recorded in its key instead of losing the
    headline, which is already measured."""
    try:
        return fn(*args)
    except Exception as exc:  # noqa: BLE001 - any failure is reported, none is hidden
        return {"error": "%s: %s" % (type(exc).__name__, str(exc)[:300])}


def other_workloads(args, stream):
    """Every other workload at its full configuration, autotuned, one timed
    call each (after one untimed call): rate, kernel milliseconds and the
    FP32 roofline fraction by the same operation count as the headline; the
    closed-form flying focus beside the 64-component sum and the adjoint of
    the batched sets."""
    import torch
    res = {}
    for idx in (3, 4, 5, 6):
        sub = argparse.Namespace(**vars(args))
        sub.workload, sub.n, sub.nsteps, sub.launch = idx, None, None, None
        wl = Workload(idx, sub, 0)
        wl.restore()
        wl.push()
        torch.cuda.synchronize()
        wl.restore()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        wl.push()
        b.record(stream)
        torch.cuda.synchronize()
        if wl.h.status() != 0:
            raise RuntimeError("device status after workload %d" % idx)
        sec = a.elapsed_time(b) / 1e3
        rate = wl.n * wl.n_steps / sec
        r = {"value": rate, "unit": UNIT, "kernel_ms": sec * 1e3, "roofline_frac": roofline_frac(idx, rate),
             "algo_ops_per_particle_step": ALGO[idx]["fp32"], "particles": wl.n, "steps": wl.n_steps,
             "workload": describe(wl, sub)["workload"], "launch": launch_desc(wl)}
        if idx == 4:
            r["closed_form"] = closed_form_rate(wl, stream, rate)
        if idx == 5:
            from paper_2307_04843_gb300.autograd import adjoint as run_adjoint
            run_adjoint(wl.pulses, wl.init, wl.off, wl.t0, wl.dt, 200, ckpt_every=100, precision="fp32")
            torch.cuda.synchronize()
            a.record(stream)
            run_adjoint(wl.pulses, wl.init, wl.off, wl.t0, wl.dt, wl.n_steps, ckpt_every=wl.cfg["ckpt_every"],
                        precision="fp32")
            b.record(stream)
            torch.cuda.synchronize()
            asec = a.elapsed_time(b) / 1e3
            arate = wl.n * wl.n_steps / asec
            r["adjoint"] = {"value": arate, "unit": UNIT, "seconds": asec,
                            "roofline_frac": ADJ_OPS * arate / (SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6),
                            "algo_ops_per_particle_step": ADJ_OPS,
                            "vs_forward": asec / sec, "ckpt_every": wl.cfg["ckpt_every"]}
        res[str(idx)] = r
        wl.close()
        del wl
        torch.cuda.empty_cache()
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2307_04843_gb300 import _lib, shard

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = Workload(args.workload, args, rank)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        wl.restore()
        wl.push()
    torch.cuda.synchronize()
    st = wl.h.status()
    if st != 0:
        raise RuntimeError("device status after warm-up: %d" % st)

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
        wl.restore()
        kev[k][0].record(stream)
        wl.push()
        kev[k][1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if ws > 1:
        dist.barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    kern = sum(a.elapsed_time(b) for a, b in kev) / 1e3 / args.steps
    tt = torch.tensor([elapsed, kern], dtype=torch.float64, device="cuda")
    shard.reduce_max(tt)
    elapsed, kern = float(tt[0]), float(tt[1])
    status = wl.h.status()
    if status != 0:
        raise RuntimeError("device status after timed steps: %d" % status)
    units_rank = float(wl.n) * wl.n_steps
    units = units_rank * args.steps * ws
    value = units / elapsed

    # end to end through the public API from pinned host buffers: every step
    # copies its inputs in (H2D) and its results out (D2H); two device buffers
    # and separate copy streams let step k's push overlap step k+1's input copy
    # and step k-1's result copy (a buffer is refilled only after its previous
    # results are out)
    e2e = None
    if not args.no_e2e and wl.graph is None:
        host = {k: v.cpu().pin_memory() for k, v in wl.init.items()}
        outs = [{k: torch.empty_like(v).pin_memory() for k, v in host.items()} for _ in range(2)]
        bufs = [wl.work, {k: torch.empty_like(v) for k, v in wl.work.items()}]
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def e2e_steps(count, start_ev=None):
            if start_ev is not None:
                s_in.wait_event(start_ev)
            for kk in range(count):
                b = kk % 2
                if kk >= 2:
                    s_in.wait_event(ev_out[b])
                with torch.cuda.stream(s_in):
                    for k in bufs[b]:
                        bufs[b][k].copy_(host[k], non_blocking=True)
                ev_in[b].record(s_in)
                stream.wait_event(ev_in[b])
                wl.h.push(bufs[b], wl.t0, wl.dt, wl.n_steps, precision=wl.precision, grid=wl.grid,
                          diag=wl.diag, stream=stream)
                ev_done[b].record(stream)
                s_out.wait_event(ev_done[b])
                with torch.cuda.stream(s_out):
                    for k in bufs[b]:
                        outs[b][k].copy_(bufs[b][k], non_blocking=True)
                ev_out[b].record(s_out)
            for b in range(min(count, 2)):
                stream.wait_event(ev_out[b])

        e2e_steps(2)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_steps(args.steps, start_ev=a)
        b_.record(stream)
        torch.cuda.synchronize()
        if wl.h.status() != 0:
            raise RuntimeError("device status after the end-to-end steps")
        te = torch.tensor([a.elapsed_time(b_) / 1e3], dtype=torch.float64, device="cuda")
        shard.reduce_max(te)
        e2e = {"value": units / float(te[0]), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(h2d),
               "overlap": "pipelined: two device buffers and separate H2D and D2H streams, so step k's "
                          "push overlaps step k+1's input copy and step k-1's result copy (throughput, "
                          "not the latency of one call)"}

    # comparison variants on one GPU: native-FP64-phase and plain FP64 paths
    variants = {}
    if rank == 0 and not args.no_variants and args.workload in (2, 3, 4):
        # workload 2 at its full size; the others on a prefix (the plain FP64
        # flying-focus sum runs at ~1e8 particle-steps/s)
        full = args.workload == 2
        for prec, nv in (("fp32_phase64", wl.n if full else min(wl.n, 2_000_000)),
                         ("fp64", wl.n if full else min(wl.n, 500_000))):
            if args.workload == 4:
                nv = max(1, nv // 16)
            sub = {k: v[:nv] for k, v in wl.parts.items()}
            d0 = _lib.to_device(sub, prec)
            d1 = {k: v[:200_000].clone() for k, v in d0.items()}
            wl.h.set_launch(0, 0)
            wl.h.push(d1, wl.t0, wl.dt, 100, precision=prec, grid=wl.grid)
            del d1
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            wl.h.push(d0, wl.t0, wl.dt, wl.n_steps, precision=prec, grid=wl.grid)
            b.record(stream)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) / 1e3
            variants[prec] = {"value": nv * wl.n_steps / sec, "unit": UNIT, "kernel_ms": sec * 1e3,
                              "sample": "%d particles x %d steps, one call" % (nv, wl.n_steps)}
            if prec == "fp32_phase64":
                variants[prec]["roofline_frac"] = ALGO[args.workload]["fp32"] * nv * wl.n_steps / sec / (
                    SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6)
            del d0
            torch.cuda.empty_cache()
        for prec in variants:
            variants[prec]["fp32_speedup"] = (units_rank / kern) / variants[prec]["value"]
        if args.workload == 4:
            variants["closed_form"] = closed_form_rate(wl, stream, units_rank / kern)

    # grid-node form: analytic E1/B1 on the staggered nodes of a 256^3 Yee
    # grid (six float arrays), and independent 1-D vacuum Yee lines
    grid_node = None
    if rank == 0 and not args.no_variants and args.workload == 2:
        grid_node = _auxiliary(grid_node_rates, wl, stream)
    # every other workload at its full configuration
    others = None
    if rank == 0 and not args.no_variants and args.workload == 2:
        wl_h_status = wl.h.status()
        if wl_h_status != 0:
            raise RuntimeError("device status before the other workloads: %d" % wl_h_status)
        others = _auxiliary(other_workloads, args, stream)

    # the adjoint of the batched workload: forward + reverse sweep
    adjoint = None
    if rank == 0 and args.workload == 5:
        from paper_2307_04843_gb300.autograd import adjoint as run_adjoint
        run_adjoint(wl.pulses, wl.init, wl.off, wl.t0, wl.dt, 200, ckpt_every=100, precision="fp32")
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run_adjoint(wl.pulses, wl.init, wl.off, wl.t0, wl.dt, wl.n_steps,
                    ckpt_every=wl.cfg["ckpt_every"], precision="fp32")
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        adjoint = {"value": units_rank / sec, "unit": UNIT, "seconds": sec,
                   "roofline_frac": ADJ_OPS * units_rank / sec / (SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6),
                   "algo_ops_per_particle_step": ADJ_OPS,
                   "vs_forward": sec / kern, "ckpt_every": wl.cfg["ckpt_every"]}

    # CPU oracle baseline on rank 0 (bounded sample of the same workload)
    cpu = None
    if rank == 0 and not args.no_cpu:
        threads = os.cpu_count() or 1
        g_np = None
        if wl.grid_host is not None:
            g_np = (wl.grid_host[0].cpu().numpy(), wl.grid_host[1], wl.grid_host[2])
        rate, m, wall = oracle_rate(wl.pulses[0], wl.parts, wl.t0, wl.dt, wl.n_steps, args.cpu_seconds,
                                    threads, grid=g_np)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "cpu_model": cpu_model(), "kind": "oracle",
               "sample": "first %d particles of the workload x %d steps (%.1f s wall)" % (m, wl.n_steps, wall)}
        # the same oracle on one core (a smaller sample, about a quarter of the time)
        r1, m1, w1 = oracle_rate(wl.pulses[0], wl.parts, wl.t0, wl.dt, wl.n_steps, args.cpu_seconds / 4, 1,
                                 grid=g_np)
        cpu["single_thread"] = {"value": r1, "unit": UNIT, "cores": 1,
                                "sample": "first %d particles x %d steps (%.1f s wall)" % (m1, wl.n_steps, w1)}

    # roofline of the push kernel
    al = ALGO[args.workload]
    rate_k = units_rank / kern
    if args.workload == 1:
        roofline = {"bound": "fp64", "note": "1e4 threads: latency-bound, FP64 path", "achieved": None,
                    "peak": None, "unit": None, "frac": None, "traffic": None, "kernel_ms": kern * 1e3}
    else:
        peak_ops = SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6 / 1e12  # TOP/s
        achieved = al["fp32"] * rate_k / 1e12
        traffic = None
        if args.workload == 2 and TRAFFIC_PER_PARTICLE_STEP.get(args.grid_layout) is not None and \
                all((wl.tuned or {}).get(k, 0) == v for k, v in TRAFFIC_KERNEL.items()):
            traffic = TRAFFIC_PER_PARTICLE_STEP[args.grid_layout] * units_rank
        roofline = {"bound": "alu", "pipe": "fp32", "achieved": achieved, "peak": peak_ops, "unit": "TOP/s",
                    "frac": achieved / peak_ops, "traffic": traffic,
                    "algo_ops_per_particle_step": al["fp32"], "kernel_ms": kern * 1e3,
                    "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz (max SM clock), of derived peak",
                    "mufu_frac": al["mufu"] * rate_k / (SM_COUNT * MUFU_LANES * SM_MAX_MHZ * 1e6)}
        if ck and ck.get("sm_mhz"):
            roofline["frac_at_sampled_clock"] = achieved / (SM_COUNT * FP32_LANES * ck["sm_mhz"] * 1e6 / 1e12)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if wl.precision == "fp64" else "f32",
        "data": "synthetic (seeded PCG64 particles and grid)",
        "config": describe(wl, args),
        "gpu_launches": args.steps,
        "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": ck, "variants": variants,
    }
    if adjoint is not None:
        line["adjoint"] = adjoint
    if grid_node is not None:
        line["grid_node"] = grid_node
    if others is not None:
        line["workloads"] = others
    if rank == 0:
        print(json.dumps(line), flush=True)
    wl.close()
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------- reference arm

def run_reference(args):
    """The CPU oracle as it stands, on the host cores, same workload and
    metric; each step is a bounded sample of particles over all steps."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle
    from paper_2307_04843_gb300 import workloads
    cfg = workloads.config(2)
    n_steps = args.nsteps or cfg["n_steps"]
    lo, hi = workloads.grid_box(cfg)
    grid = workloads.grid_field(cfg["box"], args.grid, torch_device="cpu").numpy()
    threads = os.cpu_count() or 1
    parts = workloads.particles(cfg, n=4096)
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
                               "%d^3 FP32 grid (CPU FP64 oracle)" % args.grid,
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
        if not build.up_to_date():
            build.build()
        if args.lines_only:
            import torch
            torch.cuda.set_device(0)
            print(json.dumps(line_rates(args.split_steps, args.plasma_steps)))
            return
        if args.legs_only:
            import torch
            from paper_2307_04843_gb300 import _lib, workloads
            torch.cuda.set_device(0)
            cfg = workloads.config(2)
            legs = argparse.Namespace(cfg=cfg, h=_lib.Handle(cfg["pulse"]))
            print(json.dumps(grid_node_rates(legs, torch.cuda.current_stream())))
            legs.h.close()
            return
        run_ours(args)


if __name__ == "__main__":
    main()
