"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the
CPU oracle on the same seeded inputs)."""
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
