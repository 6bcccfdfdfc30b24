"""The allocation-free batched entry point, ap_gather_push_batched_static.

It serves callers that cannot allocate device memory when they push (their
own allocator already owns the GPU, or their step loop must not risk an
allocation that synchronises or fails), by keeping the batched launch's
scratch in a static device array instead of a caller workspace.  This test
calls it through the C ABI twice in a row and checks each result against the
existing workspace-taking entry point, ap_gather_push_batched, on the same
inputs (the two run the same kernel, so the tolerance is the batched tests'
one: identical particle states, per-set sums to 1e-13).  The file is named to
be collected last.
"""
import numpy as np
import pytest

from paper_2307_04843_gb300 import workloads


def _inputs(n_sets=7, total=900):
    cfg = workloads.config(5)
    sets, counts = workloads.batch_sets(cfg)
    sets = sets[:n_sets]
    counts = workloads.scaled_counts(counts[:n_sets], total)
    counts[3] = 33
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    parts = workloads.particles_uniform(cfg["box"], int(off[-1]), workloads.seed_for(5) + 99)
    return cfg, sets, off, parts


@pytest.mark.gpu
def test_static_scratch_entry_point_matches_workspace_entry_point():
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg, sets, off, parts = _inputs()
    t0, dt, n_steps = cfg["t0"], cfg["dt"], 300
    with _lib.Handle(sets) as h:
        d_off = torch.as_tensor(off).cuda()
        ws = torch.zeros(_lib.ap_batch_workspace_bytes(h.h) // 4, dtype=torch.int32, device="cuda")
        for call in range(2):  # two calls in a row share (and re-zero) the static scratch
            start = float(t0 + call * n_steps * dt)
            ref = _lib.to_device(parts, "fp32")
            got = _lib.to_device(parts, "fp32")
            s_ref = torch.zeros(len(sets), dtype=torch.float64, device="cuda")
            s_got = torch.zeros(len(sets), dtype=torch.float64, device="cuda")
            _lib.ap_gather_push_batched(h.h, ref, d_off, None, start, dt, n_steps, "fp32",
                                        dict(set_sum=s_ref), ws)
            _lib.ap_gather_push_batched_static(h.h, got, d_off, None, start, dt, n_steps, "fp32",
                                               dict(set_sum=s_got))
            assert h.status() == 0
            torch.cuda.synchronize()
            a, b = _lib.to_host(ref), _lib.to_host(got)
            for k in a:
                np.testing.assert_array_equal(b[k], a[k])
            np.testing.assert_allclose(s_got.cpu().numpy(), s_ref.cpu().numpy(), rtol=1e-13)
            # the push did move the particles
            assert np.max(np.abs(b["ux"])) > 0.0
