"""Launch-shape autotuner for the push kernels.

The best launch shape depends on the kernel variant (pulse kind,
arithmetic, grid layout -- register counts range from ~40 to ~190 per
thread) and on the problem size.  ``tune`` times a short push of a sample of
the caller's particles for each candidate shape with CUDA events and keeps
the fastest; ``tune_batched`` does the same for the batched persistent launch
over the caller's own set mix.  The dimensions searched:

- threads per block and resident blocks per SM (0: as many as fit);
- particles per thread (``pairs``, float-float arithmetic only): one, or two
  with every FP32 operation packed over the pair;
- with a per-cell coefficient grid, where a thread keeps its particles'
  cells (``grid_cache``): shared memory, registers, or -- two particles per
  thread -- one of each;
- for the batched launch, the particles per tile (a multiple of what a block
  carries per pass).

Results are cached in a JSON file keyed by GPU name, the library build (a
hash of libapt.so, so that a rebuilt kernel is tuned afresh), kind,
precision, grid layout and a size bucket.  Within one particles-per-thread
setting every shape gives bit-identical particle states (the per-particle
arithmetic does not depend on the launch); the one- and two-particle kernels
differ only in float rounding.
"""
import hashlib
import json
import math
import os
import threading

from . import _lib, build

CANDIDATES = ((32, 0), (64, 0), (96, 0), (128, 0), (192, 0), (256, 0), (128, 2), (128, 3), (64, 6),
              (64, 8))
BATCH_CANDIDATES = ((64, 0), (128, 0), (256, 0), (128, 2), (128, 4))
TILE_MULTIPLES = (1, 2, 4, 8)
_lock = threading.Lock()
_build_id = None


def default_cache_path():
    return os.environ.get("APT_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "apt_autotune.json"))


def build_id():
    """Short hash of the loaded library file: shapes tuned for another build
    of the kernels are not reused."""
    global _build_id
    if _build_id is None:
        h = hashlib.sha1()
        with open(build.LIB, "rb") as f:
            for chunk in iter(lambda: f.read(1 << 20), b""):
                h.update(chunk)
        _build_id = h.hexdigest()[:16]
    return _build_id


def _grid_tag(grid):
    """The grid read by the push: none, the component arrays, or a packed copy
    in its layout (the layouts differ in registers and shared memory)."""
    if grid is None:
        return "nogrid"
    if len(grid) > 3 and grid[3] is not None:
        return "grid-" + (grid[4] if len(grid) > 4 else "nodes")
    return "grid-arrays"


def _key(gpu, kind, precision, grid, n, extra=""):
    bucket = int(math.log2(max(1, n)))
    return "%s|%s|%s|%s|%s|n2^%d%s" % (gpu, build_id(), kind, precision, _grid_tag(grid), bucket, extra)


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


def _modes(precision, grid):
    """(pairs, grid_cache) combinations the kernels have for this call."""
    cells = _grid_tag(grid) == "grid-cells"
    modes = [(0, 0)]
    if cells and precision != "fp64":
        modes.append((0, 1))
    if precision == "fp32" and _grid_tag(grid) in ("nogrid", "grid-cells"):
        modes += [(1, 0), (1, 1), (1, 2)] if cells else [(1, 0)]
    return modes


def _apply(handle, shape):
    handle.set_launch(shape["block"], shape["blocks_per_sm"], shape.get("grid_cache", 0),
                      shape.get("pairs", 0), shape.get("tile", 0))


def _cached(path, key, force):
    with _lock:
        cache = _load(path)
    return None if force else cache.get(key)


def _save(path, key, best):
    with _lock:
        cache = _load(path)
        cache[key] = best
        _store(path, cache)


def tune(handle, particles, t0, dt, precision="fp32", grid=None, sample_n=2_000_000, sample_steps=200,
         candidates=CANDIDATES, cache_path=None, force=False):
    """Pick and set the fastest launch shape of ap_gather_push for `handle`
    (a _lib.Handle).  particles: dict of CUDA tensors (a copy of a sample is
    pushed).  Returns dict(block, blocks_per_sm, grid_cache, pairs, rate,
    cached)."""
    import torch
    n = particles["x"].numel()
    kind = handle.pulses[0].get("kind", "plane")
    key = _key(torch.cuda.get_device_name(), kind, precision, grid, n)
    path = cache_path or default_cache_path()
    best = _cached(path, key, force)
    if best is not None:
        _apply(handle, best)
        return dict(best, cached=True)
    m = int(min(n, sample_n))
    sample = {k: v[:m].clone() for k, v in particles.items()}
    work = {k: v.clone() for k, v in sample.items()}
    results = []
    for pairs, gc in _modes(precision, grid):
        for block, bps in candidates:
            shape = dict(block=block, blocks_per_sm=bps, grid_cache=gc, pairs=pairs)
            _apply(handle, shape)
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
            results.append(dict(shape, rate=m * sample_steps / (a.elapsed_time(b) / 1e3)))
    best = dict(max(results, key=lambda r: r["rate"]))
    _apply(handle, best)
    best["sweep"] = results
    _save(path, key, best)
    return dict(best, cached=False)


def tune_batched(handle, particles, set_offsets, t0, dt, precision="fp32", grid=None, diag=None,
                 sample_steps=100, candidates=BATCH_CANDIDATES, tile_multiples=TILE_MULTIPLES,
                 cache_path=None, force=False):
    """Pick and set the fastest shape of the batched persistent launch
    (ap_gather_push_batched) for the caller's own sets: every particle of
    every set is pushed `sample_steps` steps per candidate (block, blocks
    per SM, particles per thread, cell placement, tile multiple).  Returns
    dict(block, blocks_per_sm, grid_cache, pairs, tile, rate, cached)."""
    import torch
    n = particles["x"].numel()
    kind = handle.pulses[0].get("kind", "plane")
    key = _key(torch.cuda.get_device_name(), kind, precision, grid, n,
               "|batched|sets%d" % (set_offsets.numel() - 1))
    path = cache_path or default_cache_path()
    best = _cached(path, key, force)
    if best is not None:
        _apply(handle, best)
        return dict(best, cached=True)
    work = {k: v.clone() for k, v in particles.items()}
    ws = torch.zeros(_lib.ap_batch_workspace_bytes(handle.h) // 4, dtype=torch.int32,
                     device=particles["x"].device)
    results = []
    for pairs, gc in _modes(precision, grid):
        for block, bps in candidates:
            for mult in tile_multiples:
                shape = dict(block=block, blocks_per_sm=bps, grid_cache=gc, pairs=pairs,
                             tile=mult * block * (2 if pairs else 1))
                _apply(handle, shape)
                for k in work:
                    work[k].copy_(particles[k])
                _lib.ap_gather_push_batched(handle.h, work, set_offsets, grid, t0, dt, 4, precision, diag, ws)
                for k in work:
                    work[k].copy_(particles[k])
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                _lib.ap_gather_push_batched(handle.h, work, set_offsets, grid, t0, dt, sample_steps, precision,
                                            diag, ws)
                b.record()
                torch.cuda.synchronize()
                results.append(dict(shape, rate=n * sample_steps / (a.elapsed_time(b) / 1e3)))
    best = dict(max(results, key=lambda r: r["rate"]))
    _apply(handle, best)
    best["sweep"] = results
    _save(path, key, best)
    return dict(best, cached=False)
