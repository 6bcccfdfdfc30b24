"""Full-size workloads in the benchmark's launch configuration (the
autotuner's shape, the per-cell coefficient grid copy where there is a grid,
the batched graph launch for the set workloads), checked on particles
sampled from the full ensemble, which the oracle recomputes one by one, and
through properties that hold at any size (histogram mass, per-set sums equal
to the sums of the returned states, held transverse positions).

Tolerances as in test_gpu_push: FP32 median relative |du| <= 1e-4, max
<= 1e-3 (|du| / max(|u_ref|, 1))."""
import math

import numpy as np
import pytest

import oracle
from paper_2307_04843_gb300 import workloads
from support import THREADS, conditioning, explained_by_conditioning, fp64_momenta, rel_u_err, subset


def _check(out, ref):
    e = rel_u_err(out, ref)
    assert np.median(e) <= 1e-4 and np.max(e) <= 1e-3, (np.median(e), np.max(e))


def _tune(h, dev, cfg, grid, tmp_path):
    from paper_2307_04843_gb300 import autotune
    n = dev["x"].numel()
    return autotune.tune(h, dev, cfg["t0"], cfg["dt"], cfg["precision"], grid,
                         sample_n=min(n, 2_000_000), sample_steps=min(cfg["n_steps"], 200),
                         cache_path=str(tmp_path / "tune.json"))


def _sample(n, k, seed):
    idx = np.random.default_rng(seed).choice(n, k, replace=False)
    return np.unique(np.concatenate([idx, [0, n - 1]]))


@pytest.mark.gpu
def test_workload2_full_size_cells_autotuned(tmp_path):
    """1e7 particles, 256^3 grid read from its coefficient copy, 4000 steps."""
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    parts = workloads.particles(cfg)
    lo, hi = workloads.grid_box(cfg)
    g = workloads.grid_field(cfg["box"], 256, torch_device="cuda")
    grid = _lib.pack_grid((g, lo, hi), layout="cells")
    init = _lib.to_device(parts, "fp32")
    dev = {k: v.clone() for k, v in init.items()}
    with _lib.Handle(cfg["pulse"]) as h:
        _tune(h, init, cfg, grid, tmp_path)
        h.push(dev, cfg["t0"], cfg["dt"], cfg["n_steps"], precision="fp32", grid=grid)
        assert h.status() == 0
    out = _lib.to_host(dev)
    idx = _sample(cfg["n"], 30, 2)
    ref = oracle.push(cfg["pulse"], subset(parts, idx), cfg["t0"], cfg["dt"], cfg["n_steps"],
                      grid=(g.cpu().numpy(), lo, hi), threads=THREADS)
    _check(subset(out, idx), ref)


@pytest.mark.gpu
def test_workload3_full_size_histogram_and_samples(tmp_path):
    """3.2e7-electron beam through the CP LG_{1,2} pulse, 3000 steps, with
    the 1024-bin histogram: every particle lands in one bin, the histogram is
    the oracle's binning of the returned momenta, sampled trajectories match."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(3)
    parts = workloads.particles(cfg)
    d = cfg["diag"]
    init = _lib.to_device(parts, "fp32")
    dev = {k: v.clone() for k, v in init.items()}
    hist = torch.zeros(d["hist_bins"], dtype=torch.int32, device="cuda")
    with _lib.Handle(cfg["pulse"]) as h:
        _tune(h, init, cfg, None, tmp_path)
        h.push(dev, cfg["t0"], cfg["dt"], cfg["n_steps"], precision="fp32",
               diag=dict(hist=hist, hist_lo=d["hist_lo"], hist_hi=d["hist_hi"]))
        assert h.status() == 0
    out = _lib.to_host(dev)
    hh = hist.cpu().numpy().astype(np.uint32)
    assert int(hh.astype(np.int64).sum()) == cfg["n"]
    own = oracle.gamma_hist(out["ux"], out["uy"], out["uz"], d["hist_bins"], d["hist_lo"], d["hist_hi"])
    np.testing.assert_array_equal(hh, own)
    idx = _sample(cfg["n"], 40, 3)
    ref = oracle.push(cfg["pulse"], subset(parts, idx), cfg["t0"], cfg["dt"], cfg["n_steps"], threads=THREADS)
    _check(subset(out, idx), ref)


@pytest.mark.gpu
def test_workload4_full_size_samples(tmp_path):
    """1.6e7 electrons in the 64-component flying focus, 6000 steps."""
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(4)
    parts = workloads.particles(cfg)
    init = _lib.to_device(parts, "fp32")
    dev = {k: v.clone() for k, v in init.items()}
    with _lib.Handle(cfg["pulse"]) as h:
        _tune(h, init, cfg, None, tmp_path)
        h.push(dev, cfg["t0"], cfg["dt"], cfg["n_steps"], precision="fp32")
        assert h.status() == 0
    out = _lib.to_host(dev)
    # half the sample where the focus passes during the run, half anywhere
    st = oracle.state(cfg["pulse"])
    near = np.flatnonzero((np.abs(parts["z"] - st["z_mid"]) < 30.0) & (parts["x"] ** 2 + parts["y"] ** 2 < 25.0))
    idx = np.unique(np.concatenate([np.random.default_rng(4).choice(near, 8, replace=False),
                                    _sample(cfg["n"], 6, 4)]))
    ref = oracle.push(cfg["pulse"], subset(parts, idx), cfg["t0"], cfg["dt"], cfg["n_steps"], threads=THREADS)
    e = rel_u_err(subset(out, idx), ref)
    assert np.median(e) <= 1e-4, np.median(e)
    # electrons near the moving focus can be ill-conditioned (see
    # test_gpu_ensemble): above 1e-3 only where the conditioning explains it
    over = np.flatnonzero(e > 1e-3)
    if over.size:
        sub = subset(parts, idx)
        ref64 = fp64_momenta(cfg["pulse"], sub, cfg["t0"], cfg["dt"], cfg["n_steps"])
        d7, dr = conditioning(cfg["pulse"], sub, over, ref64, cfg["t0"], cfg["dt"], cfg["n_steps"], None, 97)
        assert np.all(explained_by_conditioning(e[over], d7, dr)), (e[over], d7, dr)
    assert np.max(np.abs(ref["ux"])) > 0.1


def _batched_full(cfg, sets, parts, off, tmp_path):
    import torch
    from paper_2307_04843_gb300 import _lib
    with _lib.Handle(sets) as h:
        dev = _lib.to_device(parts, "fp32")
        d_off = torch.as_tensor(off).cuda()
        ws = torch.zeros(_lib.ap_batch_workspace_bytes(h.h) // 4, dtype=torch.int32, device="cuda")
        diag = dict(set_sum=torch.zeros(len(sets), dtype=torch.float64, device="cuda"))
        s = torch.cuda.Stream()
        gr = _lib.ap_batch_graph_create(h.h, dev, d_off, None, cfg["t0"], cfg["dt"], cfg["n_steps"], "fp32",
                                        diag, ws, s)
        _lib.ap_graph_launch(gr, s)
        s.synchronize()
        _lib.ap_graph_destroy(gr)
        assert h.status() == 0
        return _lib.to_host(dev), diag["set_sum"].cpu().numpy()


@pytest.mark.gpu
def test_workload5_full_size_graph(tmp_path):
    """256 Gaussian sets, 1.6e7 electrons, one graph launch: per-set sums of
    gamma equal the sums over the returned states; sampled particles of
    sampled sets match the oracle under their own set's pulse."""
    cfg = workloads.config(5)
    sets, counts = workloads.batch_sets(cfg)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    parts = workloads.particles_uniform(cfg["box"], int(off[-1]), workloads.seed_for(5))
    out, sums = _batched_full(cfg, sets, parts, off, tmp_path)
    own = oracle.set_gamma_sums(off, out["ux"], out["uy"], out["uz"])
    np.testing.assert_allclose(sums, own, rtol=1e-10)  # summation order, n eps
    rng = np.random.default_rng(5)
    for s in rng.choice(len(sets), 6, replace=False):
        idx = off[s] + rng.choice(int(counts[s]), 5, replace=False)
        ref = oracle.push(sets[s], subset(parts, idx), cfg["t0"], cfg["dt"], cfg["n_steps"], threads=THREADS)
        _check(subset(out, idx), ref)


@pytest.mark.gpu
def test_workload6_full_size_sweep(tmp_path):
    """30 1D-3V lines x 1e5 electrons, 4000 steps, one graph launch: the
    transverse positions are held, per-line sums equal the sums over the
    returned states, sampled electrons match the oracle."""
    cfg = workloads.config(6)
    sets, parts, off = workloads.sweep_lines(cfg)
    out, sums = _batched_full(cfg, sets, parts, off, tmp_path)
    for k in ("x", "y"):
        assert np.all(np.abs(out[k] - parts[k]) <= 2.0 ** -46 * np.abs(parts[k]))
    own = oracle.set_gamma_sums(off, out["ux"], out["uy"], out["uz"])
    np.testing.assert_allclose(sums, own, rtol=1e-10)  # summation order, n eps
    idx = _sample(int(off[-1]), 40, 6)
    ref = oracle.push(sets[0], subset(parts, idx), cfg["t0"], cfg["dt"], cfg["n_steps"], threads=THREADS)
    _check(subset(out, idx), ref)


@pytest.mark.gpu
def test_workload5_adjoint_full_size():
    """The bench's adjoint call at full size (256 Gaussian sets, ~1.6e7
    electrons, 2000 steps, checkpoints every 100, FP32): the objective equals
    the forward push's per-set mean final gamma, and for three sampled sets
    the gradient with respect to (a0, w0, z_f) matches FP64 central
    differences of the GPU forward push over the whole set (the mean over the
    set is the objective) to the gradient bound, 1e-3 relative."""
    import torch
    from paper_2307_04843_gb300 import _lib
    from paper_2307_04843_gb300.autograd import adjoint
    cfg = workloads.config(5)
    sets, counts = workloads.batch_sets(cfg)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    parts = workloads.particles_uniform(cfg["box"], int(off[-1]), workloads.seed_for(5))
    dev = _lib.to_device(parts, "fp32")
    d_off = torch.as_tensor(off).cuda()
    J, dJ = adjoint(sets, dev, d_off, cfg["t0"], cfg["dt"], cfg["n_steps"], ckpt_every=cfg["ckpt_every"],
                    precision="fp32")
    J, dJ = J.cpu().numpy(), dJ.cpu().numpy()
    _, sums = _batched_full(cfg, sets, parts, off, None)
    np.testing.assert_allclose(J, sums / counts, rtol=1e-5)  # FP32 forward in both

    def mean_gamma64(pulse, sub):
        with _lib.Handle(pulse) as h:
            d = _lib.to_device(sub, "fp64")
            ss = torch.zeros(1, dtype=torch.float64, device="cuda")
            h.push(d, cfg["t0"], cfg["dt"], cfg["n_steps"], precision="fp64", diag=dict(set_sum=ss))
            assert h.status() == 0
            return float(ss.item()) / sub["x"].size

    rng = np.random.default_rng(55)
    for s in rng.choice(len(sets), 3, replace=False):
        sub = {k: v[off[s]:off[s + 1]] for k, v in parts.items()}
        for col, name in enumerate(("a0", "w0", "z_focus")):
            p = sets[s]
            h = 1e-4 * (abs(p[name]) if name != "z_focus" else 2 * math.pi)
            fd = (mean_gamma64(dict(p, **{name: p[name] + h}), sub) -
                  mean_gamma64(dict(p, **{name: p[name] - h}), sub)) / (2 * h)
            assert abs(dJ[s, col] - fd) <= 1e-3 * max(abs(fd), 1e-6), (s, name, dJ[s, col], fd)
