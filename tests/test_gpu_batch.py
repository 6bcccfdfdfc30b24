"""Batched persistent launch (workload 5 shape): many Gaussian pulse-parameter
sets with uneven particle counts in one launch, and its CUDA-graph replay.

Checks: every particle's final state equals (bit for bit) the plain
single-set push of the same set, since both run the same per-particle code;
per-set sums of final gamma match the oracle; the graph replays the call."""
import numpy as np
import pytest

import oracle
from paper_2307_04843_gb300 import workloads
from support import THREADS, rel_u_err


def _small_batch(n_sets=9, total=1500, n_steps=400, seed=None):
    cfg = workloads.config(5)
    sets, counts = workloads.batch_sets(cfg, seed=seed)
    sets = sets[:n_sets]
    counts = workloads.scaled_counts(counts[:n_sets], total)
    counts[2] = 1      # a set of one particle
    counts[4] = 37     # ragged
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    parts = workloads.particles_uniform(cfg["box"], int(off[-1]), workloads.seed_for(5))
    return cfg, sets, off, parts, n_steps


def _run_batched(sets, off, parts, t0, dt, n_steps, precision, graph=False, replays=1):
    import torch
    from paper_2307_04843_gb300 import _lib
    with _lib.Handle(sets) as h:
        dev = _lib.to_device(parts, precision)
        d_off = torch.as_tensor(off).cuda()
        ws = torch.zeros(_lib.ap_batch_workspace_bytes(h.h) // 4, dtype=torch.int32, device="cuda")
        diag = dict(set_sum=torch.zeros(len(sets), dtype=torch.float64, device="cuda"))
        if graph:
            s = torch.cuda.Stream()
            g = _lib.ap_batch_graph_create(h.h, dev, d_off, None, t0, dt, n_steps, precision, diag, ws, s)
            snapshot = {k: v.clone() for k, v in dev.items()}
            for r in range(replays):
                for k in dev:
                    dev[k].copy_(snapshot[k])
                torch.cuda.synchronize()
                _lib.ap_graph_launch(g, s)
                s.synchronize()
            _lib.ap_graph_destroy(g)
        else:
            _lib.ap_gather_push_batched(h.h, dev, d_off, None, t0, dt, n_steps, precision, diag, ws)
        st = h.status()
        torch.cuda.synchronize()
        return _lib.to_host(dev), diag["set_sum"].cpu().numpy(), st


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batched_equals_per_set_push_and_oracle(precision):
    from support import gpu_push
    cfg, sets, off, parts, n_steps = _small_batch()
    out, sums, st = _run_batched(sets, off, parts, cfg["t0"], cfg["dt"], n_steps, precision)
    assert st == 0
    for s in range(len(sets)):
        sl = slice(off[s], off[s + 1])
        sub = {k: v[sl] for k, v in parts.items()}
        one, _, _ = gpu_push(sets[s], sub, cfg["t0"], cfg["dt"], n_steps, precision)
        for k in one:
            np.testing.assert_array_equal(out[k][sl], one[k])
    # oracle on every set (small), per-set sums of gamma
    refs = [oracle.push(sets[s], {k: v[off[s]:off[s + 1]] for k, v in parts.items()}, cfg["t0"],
                        cfg["dt"], n_steps, threads=THREADS) for s in range(len(sets))]
    ref = {k: np.concatenate([r[k] for r in refs]) for k in refs[0]}
    e = rel_u_err(out, ref)
    assert np.median(e) <= (1e-10 if precision == "fp64" else 1e-4)
    assert np.max(e) <= (1e-7 if precision == "fp64" else 1e-3)
    ref_sums = oracle.set_gamma_sums(off, ref["ux"], ref["uy"], ref["uz"])
    np.testing.assert_allclose(sums, ref_sums, rtol=1e-12 if precision == "fp64" else 1e-4)
    own_sums = oracle.set_gamma_sums(off, out["ux"], out["uy"], out["uz"])
    np.testing.assert_allclose(sums, own_sums, rtol=1e-13)


@pytest.mark.gpu
def test_graph_replay_matches_direct_call():
    cfg, sets, off, parts, n_steps = _small_batch(n_steps=200)
    a, sa, _ = _run_batched(sets, off, parts, cfg["t0"], cfg["dt"], n_steps, "fp32")
    b, sb, st = _run_batched(sets, off, parts, cfg["t0"], cfg["dt"], n_steps, "fp32", graph=True, replays=3)
    assert st == 0
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_allclose(sa, sb, rtol=1e-14)


@pytest.mark.gpu
def test_batched_argument_errors():
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg, sets, off, parts, _ = _small_batch()
    with _lib.Handle(sets) as h:
        dev = _lib.to_device(parts, "fp32")
        d_off = torch.as_tensor(off).cuda()
        small = torch.zeros(1, dtype=torch.int32, device="cuda")
        with pytest.raises(_lib.APError) as e:
            _lib.ap_gather_push_batched(h.h, dev, d_off, None, 0.0, 0.02, 5, "fp32", None, small)
        assert e.value.status == _lib.AP_ERR_WORKSPACE
        ws = torch.zeros(64, dtype=torch.int32, device="cuda")
        with pytest.raises(_lib.APError):
            _lib.ap_gather_push_batched(h.h, dev, d_off[:-1], None, 0.0, 0.02, 5, "fp32", None, ws)


# ------------------------------------------------------------ radial sweep (1D-3V)

@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_one_d_radial_sweep_matches_oracle(precision):
    """Workload-6 shape (Sec. 3.2, Fig. 6): 30 one-dimensional lines at radii
    (s + 1/2) 0.1 lambda, gamma 5088 counter-propagating through a Gaussian
    with a0 = 50, one set per line in one batched launch; 40 electrons per
    line, the 2000 steps up to the crossing of the beam centre and the pulse
    peak (the largest momentum excursion).  The transverse position stays
    where it started (to the float-float representation of the state in the
    FP32 path); momenta and per-line sums of gamma match the oracle."""
    cfg = workloads.config(6)
    sets, parts, off = workloads.sweep_lines(cfg, per_set=40)
    n_steps = 2000
    out, sums, st = _run_batched(sets, off, parts, cfg["t0"], cfg["dt"], n_steps, precision)
    assert st == 0
    # held exactly in FP64; the float-float state returns its 48-bit copy of x
    tol = 0.0 if precision == "fp64" else 2.0 ** -46
    for k in ("x", "y"):
        assert np.all(np.abs(out[k] - parts[k]) <= tol * np.abs(parts[k])), k
    ref = oracle.push(sets[0], parts, cfg["t0"], cfg["dt"], n_steps, threads=THREADS)
    e = rel_u_err(out, ref)
    med, mx = (1e-10, 1e-7) if precision == "fp64" else (1e-4, 1e-3)
    assert np.median(e) <= med and np.max(e) <= mx, (np.median(e), np.max(e))
    ref_sums = oracle.set_gamma_sums(off, ref["ux"], ref["uy"], ref["uz"])
    np.testing.assert_allclose(sums, ref_sums, rtol=1e-10 if precision == "fp64" else 1e-5)
    # the pulse drives the lines, harder near the axis
    ux_max = [np.max(np.abs(ref["ux"][off[s]:off[s + 1]])) for s in (0, len(sets) - 1)]
    assert ux_max[0] > 10.0 and ux_max[0] > 2.0 * ux_max[1], ux_max


@pytest.mark.gpu
def test_maximum_number_of_sets():
    """AP_MAX_SETS = 4096 pulse sets in one batched launch, counts 0..3
    (empty sets included): every particle equals the single-set push of its
    own set, and per-set sums match the returned states."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(5)
    base, _ = workloads.batch_sets(cfg)
    S = _lib.AP_MAX_SETS
    rng = np.random.default_rng(41)
    sets = [dict(base[s % len(base)], a0=float(rng.uniform(2, 20))) for s in range(S)]
    counts = rng.integers(0, 4, S)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    parts = workloads.particles_uniform(cfg["box"], int(off[-1]), 77)
    n_steps = 60
    out, sums, st = _run_batched(sets, off, parts, cfg["t0"], cfg["dt"], n_steps, "fp32")
    assert st == 0
    own = oracle.set_gamma_sums(off, out["ux"], out["uy"], out["uz"])
    np.testing.assert_allclose(sums, own, rtol=1e-12)
    assert np.all(sums[counts == 0] == 0.0)
    from support import gpu_push
    for s in rng.choice(np.flatnonzero(counts > 0), 12, replace=False):
        sub = {k: v[off[s]:off[s + 1]] for k, v in parts.items()}
        single, _, _ = gpu_push(sets[s], sub, cfg["t0"], cfg["dt"], n_steps, "fp32")
        for k in single:
            np.testing.assert_array_equal(out[k][off[s]:off[s + 1]], single[k])
