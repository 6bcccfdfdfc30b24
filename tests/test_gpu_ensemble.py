"""Ensemble-wide parity at the benchmark's sizes: every particle of the FP32
push (the benchmark's arithmetic: float fields and Boris, float-float phase
and position) against the plain FP64 GPU path on the same seeded inputs,
which stands in for the full ensemble, with the FP64 oracle recomputing a
seeded subsample.

Beside each comparison, the intrinsic sensitivity of the trajectories: the
FP64 path run again from initial positions perturbed by 1e-7 relative
(x' = x + 1e-7 max(|x|, lambda) xi, xi uniform in [-1, 1], seeded), compared
with the unperturbed FP64 run in the same metric.  An FP32 rounding error of
~6e-8 per operation enters every step; a trajectory that amplifies a 1e-7
perturbation amplifies those too, so the perturbed FP64 run measures how
much of the FP32 deviation the dynamics themselves produce.

Bounds (|du| / max(|u_ref|, 1) per particle): FP32 median <= 1e-4 and max
<= 1e-3 after the run; FP64 GPU vs oracle median <= 1e-10, max <= 1e-7;
final-gamma histograms (1024 bins) of the FP32 and FP64 ensembles differ by
sum |dcount| <= 1e-3 N (bin-edge flips).

Where the dynamics are ill-conditioned no arithmetic meets the max bound for
every particle: in the Gaussian and flying-focus ensembles the perturbed
FP64 run itself departs by more than 1e-3 for some particles.  There the
test holds the FP32 ensemble to the median bound and to the max bound at the
99.9th percentile, and requires every particle above 1e-3 to be explained by
its conditioning, measured by rerunning its FP64 trajectory from 16 starts
perturbed in position and momentum (momentum floor m c) at two sizes:
  - at 1e-7 relative its largest departure must exceed 1e-5, an amplification
    kappa >= 100 (the median particle amplifies ~8x): it is ill-conditioned;
  - at sqrt(N) 2^-24 relative -- the size of the rounding that the float
    momentum accumulates over the run's N steps, one 2^-24 rounding per step
    -- its largest departure must reach a third of its FP32 deviation.

Set APT_ENSEMBLE_REPORT to a file path to append the measured statistics as
JSON lines."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2307_04843_gb300 import workloads
from support import THREADS, conditioning, explained_by_conditioning, perturbed, rel_u_err, subset

U_KEYS = ("ux", "uy", "uz")
# the benchmark's launch shape for the float-float push: two particles per
# thread, the first particle's cell in registers and the second's in shared
# memory; and the one-particle shape with the cell in registers
PAIRS = dict(block=256, grid_cache=2, pairs=1)
SINGLE = dict(block=256, grid_cache=1, pairs=0)


def _report(name, **stats):
    path = os.environ.get("APT_ENSEMBLE_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(dict(test=name, **stats)) + "\n")


def _stats(e):
    return dict(median=float(np.median(e)), p999=float(np.quantile(e, 0.999)), max=float(np.max(e)),
                n_over_1e3=int(np.sum(e > 1e-3)), n=int(e.size))


def check_ensemble(name, e, s, explain=None, **extra):
    """Median and 99.9th-percentile bounds, and every particle above 1e-3
    explained by its conditioning (explain(idx) -> the largest perturbed-FP64
    departures of those particles at 1e-7 and at the rounding scale)."""
    over = np.flatnonzero(e > 1e-3)
    worst = None
    if over.size:
        assert explain is not None, (name, over.size, float(np.max(e)))
        d7, dr = explain(over)
        worst = dict(n=int(over.size), kappa_min=float(np.min(d7) / 1e-7),
                     ratio_max=float(np.max(e[over] / np.maximum(dr, 1e-300))),
                     fp32=[float(v) for v in e[over][:64]], at_1e7=[float(v) for v in d7[:64]],
                     at_rounding=[float(v) for v in dr[:64]])
    _report(name, fp32_vs_fp64=_stats(e), sensitivity=_stats(s), over=worst, **extra)
    assert np.median(e) <= 1e-4, np.median(e)
    assert np.quantile(e, 0.999) <= 1e-3, np.quantile(e, 0.999)
    if over.size:
        assert np.all(explained_by_conditioning(e[over], d7, dr)), (name, worst["kappa_min"], worst["ratio_max"])


def _push(pulse, parts, t0, dt, n_steps, precision, grid=None, launch=None, hist=None):
    """One full-size push through the C ABI; returns the final momenta (host)
    and the histogram when requested."""
    import torch
    from paper_2307_04843_gb300 import _lib
    with _lib.Handle(pulse) as h:
        if launch:
            h.set_launch(**launch)
        dev = _lib.to_device(parts, precision)
        diag = None
        if hist is not None:
            diag = dict(hist=torch.zeros(hist[0], dtype=torch.int32, device="cuda"), hist_lo=hist[1],
                        hist_hi=hist[2])
        h.push(dev, t0, dt, n_steps, precision=precision, grid=grid, diag=diag)
        st = h.status()
        out = {k: dev[k].double().cpu().numpy() for k in U_KEYS}
        hh = diag["hist"].cpu().numpy().astype(np.int64) if diag else None
    del dev
    torch.cuda.empty_cache()
    assert st == 0
    return out, hh


# ------------------------------------------------------------ workload 2

@pytest.fixture(scope="module")
def w2():
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    parts = workloads.particles(cfg)
    lo, hi = workloads.grid_box(cfg)
    g = workloads.grid_field(cfg["box"], 256, torch_device="cuda")
    cells = _lib.pack_grid((g, lo, hi), layout="cells")
    args = (cfg["t0"], cfg["dt"], cfg["n_steps"])
    r = dict(cfg=cfg, parts=parts, grid_host=(g.cpu().numpy(), lo, hi))
    r["fp32_pairs"] = _push(cfg["pulse"], parts, *args, "fp32", grid=cells, launch=PAIRS)[0]
    r["fp32_single"] = _push(cfg["pulse"], parts, *args, "fp32", grid=cells, launch=SINGLE)[0]
    r["fp64"] = _push(cfg["pulse"], parts, *args, "fp64", grid=(g, lo, hi))[0]
    r["fp64_perturbed"] = _push(cfg["pulse"], perturbed(parts, 71), *args, "fp64", grid=(g, lo, hi))[0]
    del g, cells
    return r


@pytest.mark.gpu
@pytest.mark.parametrize("variant", ["fp32_pairs", "fp32_single"])
def test_workload2_fp32_vs_fp64_every_particle(w2, variant):
    """All 1e7 electrons, 256^3 grid, 4000 steps."""
    cfg = w2["cfg"]
    e = rel_u_err(w2[variant], w2["fp64"])
    s = rel_u_err(w2["fp64_perturbed"], w2["fp64"])
    g, lo, hi = w2["grid_host"]

    def explain(idx):
        import torch
        return conditioning(cfg["pulse"], w2["parts"], idx, w2["fp64"], cfg["t0"], cfg["dt"], cfg["n_steps"],
                            (torch.as_tensor(g).cuda(), lo, hi), 83)

    check_ensemble("workload2_" + variant, e, s, explain)


@pytest.mark.gpu
def test_workload2_oracle_subsample(w2):
    """The oracle recomputes 1e4 seeded particles of the full ensemble: the
    FP64 GPU path within 1e-10 / 1e-7 of it, the FP32 path within 1e-4 / 1e-3."""
    cfg = w2["cfg"]
    idx = np.sort(np.random.default_rng(2307).choice(cfg["n"], 10_000, replace=False))
    ref = oracle.push(cfg["pulse"], subset(w2["parts"], idx), cfg["t0"], cfg["dt"], cfg["n_steps"],
                      grid=w2["grid_host"], threads=THREADS)
    e64 = rel_u_err(subset(w2["fp64"], idx), ref)
    e32 = rel_u_err(subset(w2["fp32_pairs"], idx), ref)
    _report("workload2_oracle_subsample", fp64_vs_oracle=_stats(e64), fp32_vs_oracle=_stats(e32))
    assert np.median(e64) <= 1e-10 and np.max(e64) <= 1e-7, (np.median(e64), np.max(e64))
    assert np.median(e32) <= 1e-4 and np.max(e32) <= 1e-3, (np.median(e32), np.max(e32))


# ------------------------------------------------------------ workload 3

@pytest.fixture(scope="module")
def w3():
    cfg = workloads.config(3)
    parts = workloads.particles(cfg)
    d = cfg["diag"]
    hist = (d["hist_bins"], d["hist_lo"], d["hist_hi"])
    args = (cfg["t0"], cfg["dt"], cfg["n_steps"])
    r = dict(cfg=cfg, hist=hist)
    r["fp32"], r["hist32"] = _push(cfg["pulse"], parts, *args, "fp32", launch=dict(block=128, pairs=1),
                                   hist=hist)
    r["fp64"], r["hist64"] = _push(cfg["pulse"], parts, *args, "fp64", hist=hist)
    r["fp64_perturbed"] = _push(cfg["pulse"], perturbed(parts, 73), *args, "fp64")[0]
    return r


@pytest.mark.gpu
def test_workload3_fp32_vs_fp64_every_particle_and_histogram(w3):
    """All 3.2e7 electrons of the inverse-Compton beam, 3000 steps: every
    particle within the bounds, and the two 1024-bin histograms of final
    gamma differ by at most 1e-3 N counts."""
    e = rel_u_err(w3["fp32"], w3["fp64"])
    s = rel_u_err(w3["fp64_perturbed"], w3["fp64"])
    n = e.size
    dcount = int(np.abs(w3["hist32"] - w3["hist64"]).sum())
    check_ensemble("workload3", e, s, hist_abs_diff=dcount)
    assert w3["hist32"].sum() == n and w3["hist64"].sum() == n
    assert dcount <= 1e-3 * n, dcount
    assert np.max(e) <= 1e-3, (np.max(e), int(np.argmax(e)))


# ------------------------------------------------------------ workload 4

@pytest.mark.gpu
def test_workload4_prefix_fp32_vs_fp64_every_particle():
    """The first 1e6 electrons of the flying-focus channel, 6000 steps of the
    64-component sum, every particle."""
    cfg = workloads.config(4)
    parts = {k: v[:1_000_000] for k, v in workloads.particles(cfg).items()}
    args = (cfg["t0"], cfg["dt"], cfg["n_steps"])
    u32 = _push(cfg["pulse"], parts, *args, "fp32", launch=dict(block=128, pairs=1))[0]
    u64 = _push(cfg["pulse"], parts, *args, "fp64")[0]
    u64p = _push(cfg["pulse"], perturbed(parts, 79), *args, "fp64")[0]
    e = rel_u_err(u32, u64)
    s = rel_u_err(u64p, u64)
    check_ensemble("workload4_prefix", e, s,
                   lambda idx: conditioning(cfg["pulse"], parts, idx, u64, *args, None, 89))


# ------------------------------------------------------------ workload 5 adjoint

def _adjoint_full(cfg, sets, parts, off, precision):
    import torch
    from paper_2307_04843_gb300 import _lib
    from paper_2307_04843_gb300.autograd import adjoint
    dev = _lib.to_device(parts, precision)
    J, dJ = adjoint(sets, dev, torch.as_tensor(off).cuda(), cfg["t0"], cfg["dt"], cfg["n_steps"],
                    ckpt_every=cfg["ckpt_every"], precision=precision)
    out = J.cpu().numpy(), dJ.cpu().numpy()
    del dev
    torch.cuda.empty_cache()
    return out


@pytest.mark.gpu
def test_workload5_adjoint_fp32_vs_fp64_every_set():
    """The adjoint at the benchmark's full size (256 Gaussian sets, ~1.6e7
    electrons, 2000 steps, checkpoints every 100): the per-set gradients
    d(mean final gamma)/d(a0, w0, z_f) of the FP32 adjoint (two particles per
    thread, float-float phase) against the FP64 adjoint on the same inputs,
    error |d32 - d64| / max(|d64|, 1e-3 max_s |d64|), every set.

    Beside it the FP64 adjoint again from positions perturbed by sqrt(N)
    2^-24 relative (N = 2000 steps; the size of the rounding the float state
    accumulates over the run, one 2^-24 rounding per step), in the same
    metric.  Bounds: the objective to 1e-5 relative; the a0 and w0 rows
    <= 1e-3 for every set; the z_f row median <= 1e-4, and every set above
    1e-3 within 3x of its perturbed-FP64 departure.  The z_f gradient of some
    sets is a near cancellation over the set's electrons (a few 1e-4 against
    0.33 for the largest set), so per-electron rounding shows up in it
    relative to its own size as the perturbed FP64 run shows."""
    cfg = workloads.config(5)
    sets, counts = workloads.batch_sets(cfg)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    parts = workloads.particles_uniform(cfg["box"], int(off[-1]), workloads.seed_for(5))
    J32, d32 = _adjoint_full(cfg, sets, parts, off, "fp32")
    J64, d64 = _adjoint_full(cfg, sets, parts, off, "fp64")
    rel = np.sqrt(cfg["n_steps"]) * 2.0 ** -24
    _, dp = _adjoint_full(cfg, sets, perturbed(parts, 97, rel=rel), off, "fp64")
    assert np.max(np.abs(J32 - J64) / np.abs(J64)) <= 1e-5
    stats = {}
    for col, name in enumerate(("a0", "w0", "z_focus")):
        ref = d64[:, col]
        scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
        e = np.abs(d32[:, col] - ref) / scale
        s = np.abs(dp[:, col] - ref) / scale
        stats[name] = dict(fp32=_stats(e), sensitivity=_stats(s),
                           over=[(int(i), float(e[i]), float(s[i])) for i in np.flatnonzero(e > 1e-3)])
    _report("workload5_adjoint", perturbation=float(rel), **stats)
    for col, name in enumerate(("a0", "w0", "z_focus")):
        ref = d64[:, col]
        scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
        e = np.abs(d32[:, col] - ref) / scale
        s = np.abs(dp[:, col] - ref) / scale
        if name == "z_focus":
            assert np.median(e) <= 1e-4, (name, np.median(e))
            over = np.flatnonzero(e > 1e-3)
            assert np.all(e[over] <= 3.0 * s[over]), (name, stats[name]["over"])
        else:
            assert np.max(e) <= 1e-3, (name, float(np.max(e)), int(np.argmax(e)))
