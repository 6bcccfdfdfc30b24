"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the
CPU oracle on the same seeded inputs)."""
import math
import os

import numpy as np

THREADS = max(1, min(16, os.cpu_count() or 1))


def rel_u_err(u_gpu, u_ref):
    """Per-particle |du| / max(|u_ref|, 1) (momentum in units of m c)."""
    d = np.sqrt(sum((u_gpu[k] - u_ref[k]) ** 2 for k in ("ux", "uy", "uz")))
    m = np.sqrt(sum(u_ref[k] ** 2 for k in ("ux", "uy", "uz")))
    return d / np.maximum(m, 1.0)


def pos_err(p_gpu, p_ref):
    return np.sqrt(sum((p_gpu[k] - p_ref[k]) ** 2 for k in ("x", "y", "z")))


def subset(parts, idx):
    return {k: np.asarray(v)[idx] for k, v in parts.items()}


def gpu_push(pulses, parts, t0, dt, n_steps, precision, grid=None, diag_keys=(), hist=None,
             block=0, blocks_per_sm=0, launch=None):
    """Run ap_gather_push on a copy of `parts` (numpy); returns (host arrays,
    diag dict of host arrays, status).  `launch`: keyword arguments of
    Handle.set_launch (block, blocks_per_sm, grid_cache, pairs, tile)."""
    import torch
    from paper_2307_04843_gb300 import _lib
    with _lib.Handle(pulses) as h:
        if launch:
            h.set_launch(**launch)
        elif block or blocks_per_sm:
            h.set_launch(block, blocks_per_sm)
        dev = _lib.to_device(parts, precision)
        diag = {}
        if "lightfront" in diag_keys:
            diag["lightfront"] = torch.zeros(max(n_steps, 1), dtype=torch.float64, device="cuda")
        if hist is not None:
            bins, lo, hi = hist
            diag.update(hist=torch.zeros(bins, dtype=torch.int32, device="cuda"), hist_lo=lo, hist_hi=hi)
        if "set_sum" in diag_keys:
            diag["set_sum"] = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = None
        if grid is not None:
            arr, lo, hi = grid[:3]
            g = (torch.as_tensor(arr).cuda() if not isinstance(arr, torch.Tensor) else arr, lo, hi) + tuple(grid[3:])
        h.push(dev, t0, dt, n_steps, precision=precision, grid=g, diag=diag or None)
        st = h.status()
        torch.cuda.synchronize()
        out = _lib.to_host(dev)
        dg = {k: v.cpu().numpy() for k, v in diag.items() if hasattr(v, "cpu")}
        if "hist" in dg:
            dg["hist"] = dg["hist"].astype(np.uint32)
    return out, dg, st


# ---------------------------------------------------- trajectory conditioning
L = 2 * math.pi
U_KEYS = ("ux", "uy", "uz")
K_DIRECTIONS = 16


def perturbed(parts, seed, momenta=False, rel=1e-7):
    """Initial positions (and momenta) perturbed by `rel` relative, with floors
    of one wavelength and of m c (xi uniform in [-1, 1], seeded)."""
    rng = np.random.default_rng(seed)
    out = dict(parts)
    for k in ("x", "y", "z") + (U_KEYS if momenta else ()):
        v = np.asarray(parts[k], dtype=np.float64)
        floor = L if k in ("x", "y", "z") else 1.0
        out[k] = v + rel * np.maximum(np.abs(v), floor) * rng.uniform(-1.0, 1.0, v.size)
    return out


def fp64_momenta(pulse, parts, t0, dt, n_steps, grid=None):
    """Final momenta of the plain FP64 GPU push of `parts` (host dict)."""
    import torch
    from paper_2307_04843_gb300 import _lib
    with _lib.Handle(pulse) as h:
        dev = _lib.to_device(parts, "fp64")
        h.push(dev, t0, dt, n_steps, precision="fp64", grid=grid)
        st = h.status()
        out = {k: dev[k].cpu().numpy() for k in U_KEYS}
    del dev
    torch.cuda.empty_cache()
    assert st == 0
    return out


def conditioning(pulse, parts, idx, ref64, t0, dt, n_steps, grid, seed):
    """For the particles idx of `parts`: the largest departure of their FP64
    trajectory (from the final momenta ref64 of the unperturbed FP64 run) over
    K_DIRECTIONS runs from starts perturbed by 1e-7 and by sqrt(n_steps) 2^-24
    relative in position and momentum -- the second the size of the rounding
    that a float momentum accumulates over the run, one 2^-24 rounding per
    step.  All replicas are pushed as one batch on the GPU.  Returns
    (departures at 1e-7, at the rounding scale)."""
    sub = subset(parts, idx)
    rep = {k: np.tile(np.asarray(v, dtype=np.float64), K_DIRECTIONS) for k, v in sub.items()}
    small = perturbed(rep, seed, momenta=True)
    scale = math.sqrt(n_steps) * 2.0 ** -24 / 1e-7
    large = {k: rep[k] + scale * (small[k] - rep[k]) for k in rep}
    both = {k: np.concatenate([small[k], large[k]]) for k in rep}
    out = fp64_momenta(pulse, both, t0, dt, n_steps, grid)
    ref = {k: np.tile(np.asarray(ref64[k])[idx], 2 * K_DIRECTIONS) for k in U_KEYS}
    e = rel_u_err(out, ref).reshape(2, K_DIRECTIONS, idx.size)
    return e[0].max(axis=0), e[1].max(axis=0)


def explained_by_conditioning(e, d7, dr):
    """A particle whose FP32 deviation e exceeds 1e-3 is explained by its
    conditioning when its FP64 trajectory amplifies a 1e-7 perturbation at
    least 100-fold (departure d7 >= 1e-5; the median particle of the
    ensembles amplifies ~8-fold) and a perturbation at the float-rounding
    scale reproduces at least a third of its deviation (e <= 3 dr)."""
    return (d7 >= 1e-5) & (e <= 3.0 * dr)
