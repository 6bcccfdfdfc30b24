"""Launch-shape autotuner for the push kernels.

The best block size and residency depend on the kernel variant (pulse kind,
arithmetic, grid on/off -- register counts range from ~40 to ~130 per
thread) and on the problem size.  ``tune`` times a short push of a sample of
the caller's particles for each candidate shape with CUDA events and keeps
the fastest; results are cached in a JSON file keyed by GPU name, kind,
precision, grid layout and a size bucket.  Every shape gives bit-identical
particle states (the per-particle arithmetic does not depend on the launch).
With a per-cell coefficient grid the sweep also tries keeping the cell in
registers instead of shared memory (``grid_cache``), which trades occupancy
for shared-memory traffic; both give bit-identical states too.
"""
import json
import math
import os
import threading

from . import _lib

CANDIDATES = ((32, 0), (64, 0), (96, 0), (128, 0), (192, 0), (256, 0), (128, 2), (128, 3), (64, 6),
              (64, 8))
_lock = threading.Lock()


def default_cache_path():
    return os.environ.get("APT_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "apt_autotune.json"))


def _grid_tag(grid):
    """The grid read by the push: none, the component arrays, or a packed copy
    in its layout (the layouts differ in registers and shared memory)."""
    if grid is None:
        return "nogrid"
    if len(grid) > 3 and grid[3] is not None:
        return "grid-" + (grid[4] if len(grid) > 4 else "nodes")
    return "grid-arrays"


def _key(gpu, kind, precision, grid, n):
    bucket = int(math.log2(max(1, n)))
    return "%s|%s|%s|%s|n2^%d" % (gpu, kind, precision, _grid_tag(grid), bucket)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(handle, particles, t0, dt, precision="fp32", grid=None, sample_n=2_000_000, sample_steps=200,
         candidates=CANDIDATES, cache_path=None, force=False):
    """Pick and set the fastest launch shape for `handle` (a _lib.Handle).
    particles: dict of CUDA tensors (only a copy of a sample is pushed).
    Returns dict(block=..., blocks_per_sm=..., rate=..., cached=bool)."""
    import torch
    n = particles["x"].numel()
    kind = handle.pulses[0].get("kind", "plane")
    gpu = torch.cuda.get_device_name()
    key = _key(gpu, kind, precision, grid, n)
    path = cache_path or default_cache_path()
    with _lock:
        cache = _load(path)
    if not force and key in cache:
        best = cache[key]
        handle.set_launch(best["block"], best["blocks_per_sm"], best.get("grid_cache", 0))
        return dict(best, cached=True)
    caches = (0, 1) if _grid_tag(grid) == "grid-cells" and precision != "fp64" else (0,)
    m = int(min(n, sample_n))
    sample = {k: v[:m].clone() for k, v in particles.items()}
    work = {k: v.clone() for k, v in sample.items()}
    results = []
    for (block, bps), gc in [(c, g) for g in caches for c in candidates]:
        handle.set_launch(block, bps, gc)
        for k in work:
            work[k].copy_(sample[k])
        handle.push(work, t0, dt, 8, precision=precision, grid=grid)  # warm (module load, caches)
        for k in work:
            work[k].copy_(sample[k])
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        handle.push(work, t0, dt, sample_steps, precision=precision, grid=grid)
        b.record()
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        results.append((m * sample_steps / sec, block, bps, gc))
    rate, block, bps, gc = max(results)
    handle.set_launch(block, bps, gc)
    best = dict(block=block, blocks_per_sm=bps, grid_cache=gc, rate=rate,
                sweep=[dict(block=b_, blocks_per_sm=p_, grid_cache=g_, rate=r_) for r_, b_, p_, g_ in results])
    with _lock:
        cache = _load(path)
        cache[key] = best
        _store(path, cache)
    return dict(best, cached=False)

