"""Push parity: ap_gather_push (all steps fused in one launch) against the
oracle on the same seeded inputs, for each workload at sizes the oracle
finishes in seconds (several blocks and a ragged tail), plus the edge cases.

Tolerances: FP64 GPU vs oracle, median relative |du| <= 1e-10 and max
<= 1e-7 (different math libraries and FMA contraction, amplified by the
trajectory); FP32 (double or float-float phase and position) median <= 1e-4
and max <= 1e-3, relative error |du| / max(|u_ref|, 1)."""
import math

import numpy as np
import pytest

import oracle
from paper_2307_04843_gb300 import workloads
from support import THREADS, gpu_push, pos_err, rel_u_err, subset

L = 2 * math.pi
FP32_MED, FP32_MAX = 1e-4, 1e-3
FP64_MED, FP64_MAX = 1e-10, 1e-7


def _check(out, ref, precision, pos_tol=None):
    e = rel_u_err(out, ref)
    med, mx = (FP64_MED, FP64_MAX) if precision == "fp64" else (FP32_MED, FP32_MAX)
    assert np.median(e) <= med, (precision, np.median(e))
    assert np.max(e) <= mx, (precision, np.max(e), int(np.argmax(e)))
    if pos_tol is not None:
        assert np.max(pos_err(out, ref)) <= pos_tol, np.max(pos_err(out, ref))


# ------------------------------------------------------------ workload 1

@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_phase64"])
def test_workload1_plane_full_size(precision):
    """1e4 electrons, 2000 steps, plane wave a0 = 1: final x and u match the
    oracle; the per-step light-front deviation matches and is O(dt^2)."""
    cfg = workloads.config(1)
    parts = workloads.particles(cfg)
    out, dg, st = gpu_push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], precision,
                           diag_keys=("lightfront",))
    assert st == 0
    ref, lf = oracle.push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], lf=True, threads=THREADS)
    _check(out, ref, precision, pos_tol=1e-9 if precision == "fp64" else 2e-4)
    if precision == "fp64":
        np.testing.assert_allclose(dg["lightfront"], lf, rtol=1e-6, atol=1e-15)
    else:
        # float gamma - u_z carries the FP32 trajectory error (rsqrt and
        # rounding of O(1) momenta, ~1e-7 per step accumulating): 1e-5 absolute
        assert np.max(np.abs(dg["lightfront"] - lf)) < 1e-5
        assert dg["lightfront"].max() < 2e-5
    assert lf.max() < 1e-5  # C dt^2 with dt = 0.02


# ------------------------------------------------------------ workload 2

def _grid_small(cfg, n=40):
    lo, hi = workloads.grid_box(cfg)
    g = workloads.grid_field(cfg["box"], n, amplitude=0.1, n_terms=16, kmax=4)
    return g, lo, hi


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_phase64"])
def test_workload2_gauss_grid_reduced(precision):
    """Gaussian a0 = 10 with longitudinal fields plus the static grid, 4000
    steps, on a 40^3 grid and 300 particles of the seeded ensemble."""
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=300)
    grid = _grid_small(cfg)
    out, _, st = gpu_push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], precision, grid=grid)
    assert st == 0
    ref = oracle.push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], grid=grid, threads=THREADS)
    _check(out, ref, precision)
    # the pulse did work on the particles
    assert np.max(np.abs(ref["ux"])) > 1.0


@pytest.mark.gpu
def test_workload2_full_size_sampled():
    """Full workload 2 (1e7 particles, 256^3 grid, 4000 steps, float-float
    phase) in the benchmark's launch configuration; 24 sampled particles
    recomputed one by one by the oracle."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    parts = workloads.particles(cfg)
    lo, hi = workloads.grid_box(cfg)
    g = workloads.grid_field(cfg["box"], 256, torch_device="cuda")
    dev = _lib.to_device(parts, "fp32")
    with _lib.Handle(cfg["pulse"]) as h:
        h.push(dev, cfg["t0"], cfg["dt"], cfg["n_steps"], precision="fp32", grid=(g, lo, hi))
        assert h.status() == 0
    out = _lib.to_host(dev)
    idx = np.random.default_rng(1).choice(cfg["n"], 24, replace=False)
    idx = np.concatenate([idx, [0, cfg["n"] - 1]])
    ref = oracle.push(cfg["pulse"], subset(parts, idx), cfg["t0"], cfg["dt"], cfg["n_steps"],
                      grid=(g.cpu().numpy(), lo, hi), threads=THREADS)
    _check(subset(out, idx), ref, "fp32")


# ------------------------------------------------------------ workload 3

@pytest.mark.gpu
def test_workload3_lg_ics_reduced_and_histogram():
    """Counter-propagating gamma ~ 1000 beam through the CP LG_{1,2} pulse,
    3000 steps, 600 particles: trajectories match; the 1024-bin histogram of
    final gamma equals, bit for bit, the oracle's binning of the GPU's own
    final momenta (same double arithmetic), and differs from the oracle
    trajectories' histogram only by bin-edge flips."""
    cfg = workloads.config(3)
    parts = workloads.particles(cfg, n=600)
    d = cfg["diag"]
    hist = (d["hist_bins"], d["hist_lo"], d["hist_hi"])
    out, dg, st = gpu_push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], "fp32", hist=hist)
    assert st == 0
    ref = oracle.push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], threads=THREADS)
    _check(out, ref, "fp32")
    own = oracle.gamma_hist(out["ux"], out["uy"], out["uz"], *hist)
    np.testing.assert_array_equal(dg["hist"], own)
    oh = oracle.gamma_hist(ref["ux"], ref["uy"], ref["uz"], *hist)
    # a particle can change bin only if its oracle gamma lies within
    # delta = max |gamma_gpu - gamma_oracle| of a bin edge
    g_ref = np.sqrt(1 + ref["ux"] ** 2 + ref["uy"] ** 2 + ref["uz"] ** 2)
    g_gpu = np.sqrt(1 + out["ux"] ** 2 + out["uy"] ** 2 + out["uz"] ** 2)
    delta = np.max(np.abs(g_gpu - g_ref))
    width = (hist[2] - hist[1]) / hist[0]
    f = (g_ref - hist[1]) / width
    near = np.sum(np.abs(f - np.rint(f)) * width <= delta)
    assert np.abs(dg["hist"].astype(np.int64) - oh.astype(np.int64)).sum() <= 2 * near
    assert dg["hist"].sum() == 600


# ------------------------------------------------------------ workload 4

@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_workload4_flying_focus_reduced(precision):
    """64-component flying focus, 24 particles near the moving focus, 1500
    steps (the oracle evaluates 64 beams with finite-difference derivatives
    per step)."""
    cfg = workloads.config(4)
    p = workloads.particles(cfg, n=24)
    st_ = oracle.state(cfg["pulse"])
    # place the sample where the focus passes during the run
    t0 = cfg["t0"]
    zc = st_["z_mid"] + 0.99 * (t0 + 15.0 - st_["t_mid"]) - 40.0
    p["z"] = zc + (p["z"] / (200 * L) - 0.5) * 20.0
    p["x"] = p["x"] * 0.3
    p["y"] = p["y"] * 0.3
    n_steps = 1500
    out, _, st = gpu_push(cfg["pulse"], p, t0, cfg["dt"], n_steps, precision)
    assert st == 0
    ref = oracle.push(cfg["pulse"], p, t0, cfg["dt"], n_steps, threads=THREADS)
    _check(out, ref, precision)
    assert np.max(np.abs(ref["ux"])) > 0.5


# ------------------------------------------------------------ closed-form flying focus

@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("beta_f", [-1.0, 0.5])
def test_flying_focus_closed_form_push(precision, beta_f):
    """Closed-form flying focus (a0 = 5, w0 = 3 lambda, longitudinal terms,
    Gaussian envelope), 200 electrons around the focal region, 2500 steps."""
    pulse = dict(kind="flying_cf", pol="x", env="gauss", env_len=30.0, a0=5.0, w0=3 * L, beta_f=beta_f,
                 z_focus=0.0, t_focus=0.0, longitudinal=True)
    rng = np.random.default_rng(23)
    n = 200
    parts = dict(x=rng.uniform(-1, 1, n) * 4 * L, y=rng.uniform(-1, 1, n) * 4 * L,
                 z=rng.uniform(-1, 1, n) * 6 * L, ux=np.zeros(n), uy=np.zeros(n), uz=np.zeros(n))
    t0, dt, n_steps = -40.0, 0.02, 2500
    out, _, st = gpu_push(pulse, parts, t0, dt, n_steps, precision)
    assert st == 0
    ref = oracle.push(pulse, parts, t0, dt, n_steps, threads=THREADS)
    _check(out, ref, precision)
    assert np.max(np.abs(ref["ux"])) > 0.5


# ------------------------------------------------------------ edge cases

@pytest.mark.gpu
def test_gyration_through_abi_fp64():
    """Uniform B = B0 z_hat from a 2^3 grid and a0 = 0: exact Boris rotation
    angle 2 atan(dt B0 / 2 gamma) per step and conserved |u|."""
    B0, dt, n_steps = 0.75, 0.05, 4000
    grid = np.zeros((6, 2, 2, 2), dtype=np.float32)
    grid[5] = B0
    lo, hi = (-1e6,) * 3, (1e6,) * 3
    u0 = np.array([1.3, -0.4, 0.25])
    parts = {k: np.array([v]) for k, v in dict(x=0.0, y=0.0, z=0.0, ux=u0[0], uy=u0[1], uz=u0[2]).items()}
    out, _, st = gpu_push(dict(kind="plane", a0=0.0), parts, 0.0, dt, n_steps, "fp64", grid=(grid, lo, hi))
    gamma = math.sqrt(1 + u0 @ u0)
    theta = 2 * math.atan(dt * B0 / (2 * gamma))
    ang = math.atan2(out["uy"][0], out["ux"][0])
    expect = math.atan2(u0[1], u0[0]) + n_steps * theta
    d = (ang - expect + math.pi) % (2 * math.pi) - math.pi
    assert abs(d) < 1e-10
    u = np.array([out["ux"][0], out["uy"][0], out["uz"][0]])
    assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_split_calls_equal_one_call(precision):
    """n_steps may be split across calls: 700 + 500 steps equal 1200 steps,
    bitwise in FP64 when t0 + 700 dt is exact (dt = 2^-6 here); with the
    float-float phase the second call re-derives its phase base from its own
    t0, so agreement is to float rounding."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=77)
    pulse = cfg["pulse"]
    with _lib.Handle(pulse) as h:
        a = _lib.to_device(parts, precision)
        b = _lib.to_device(parts, precision)
        dt = 2.0 ** -6
        h.push(a, -40.0, dt, 1200, precision=precision)
        h.push(b, -40.0, dt, 700, precision=precision)
        h.push(b, -40.0 + 700 * dt, dt, 500, precision=precision)
        torch.cuda.synchronize()
        ha, hb = _lib.to_host(a), _lib.to_host(b)
    for k in ha:
        if precision == "fp64":
            np.testing.assert_array_equal(ha[k], hb[k])
        else:
            np.testing.assert_allclose(ha[k], hb[k], rtol=1e-6, atol=1e-6)


@pytest.mark.gpu
@pytest.mark.parametrize("n", [0, 1, 31, 33, 1000])
def test_ragged_and_empty_sizes(n):
    """Empty input is a no-op; ragged sizes match the oracle particle by particle."""
    cfg = workloads.config(1)
    parts = workloads.particles(cfg, n=n)
    out, _, st = gpu_push(cfg["pulse"], parts, 30.0, 0.02, 300, "fp64")
    assert st == 0
    assert out["x"].size == n
    if n:
        ref = oracle.push(cfg["pulse"], parts, 30.0, 0.02, 300)
        _check(out, ref, "fp64")


@pytest.mark.gpu
def test_zero_steps_is_identity():
    cfg = workloads.config(1)
    parts = workloads.particles(cfg, n=50)
    out, _, st = gpu_push(cfg["pulse"], parts, 0.0, 0.02, 0, "fp32")
    for k in ("x", "y", "z"):
        np.testing.assert_array_equal(out[k], parts[k])


@pytest.mark.gpu
def test_nonfinite_input_reported():
    """A NaN momentum propagates; the kernel flags it and ap_sync_status
    returns AP_ERR_NONFINITE (no GPU fault involved)."""
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(1)
    parts = workloads.particles(cfg, n=64)
    parts["ux"][5] = np.nan
    _, _, st = gpu_push(cfg["pulse"], parts, 0.0, 0.02, 10, "fp32")
    assert st == _lib.AP_ERR_NONFINITE


@pytest.mark.gpu
def test_misaligned_and_wrong_dtype_rejected():
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(1)
    parts = workloads.particles(cfg, n=65)
    dev = _lib.to_device(parts, "fp32")
    with _lib.Handle(cfg["pulse"]) as h:
        bad = dict(dev)
        bad["x"] = torch.zeros(66, dtype=torch.float64, device="cuda")[1:]  # 8-byte offset
        with pytest.raises(_lib.APError) as e:
            h.push(bad, 0.0, 0.02, 1, precision="fp32")
        assert e.value.status == _lib.AP_ERR_ALIGN
        with pytest.raises(ValueError):
            h.push(dev, 0.0, 0.02, 1, precision="fp64")  # float32 momenta for an fp64 call


@pytest.mark.gpu
def test_launch_shapes_give_identical_results():
    """Block size and residency do not change any particle's arithmetic."""
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=1000)
    base, _, _ = gpu_push(cfg["pulse"], parts, -5.0, 0.02, 200, "fp32")
    for block, bps in ((32, 0), (64, 2), (256, 1)):
        out, _, _ = gpu_push(cfg["pulse"], parts, -5.0, 0.02, 200, "fp32", block=block, blocks_per_sm=bps)
        for k in base:
            np.testing.assert_array_equal(out[k], base[k])


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_packed_grid_layout_gives_identical_results(precision):
    """The node-interleaved grid copy (ap_grid_pack) changes only the layout:
    the push reads the same corner values and gives bit-identical states."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=2000)
    g, lo, hi = _grid_small(cfg, n=33)
    gd = torch.as_tensor(g).cuda()
    packed = _lib.pack_grid((gd, lo, hi))
    host = packed[3].view(-1, 8).cpu().numpy()
    np.testing.assert_array_equal(host[:, :6], g.reshape(6, -1).T)
    assert np.all(host[:, 6:] == 0)
    a, _, _ = gpu_push(cfg["pulse"], parts, -10.0, 0.02, 800, precision, grid=(gd, lo, hi))
    b, _, _ = gpu_push(cfg["pulse"], parts, -10.0, 0.02, 800, precision, grid=packed)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.gpu
def test_cell_coefficient_layout_reconstructs_corners():
    """AP_PACK_CELLS holds, per cell and component, the monomial coefficients
    of the trilinear interpolant: summing them back at the 8 corners gives the
    grid values to float rounding (each coefficient rounded once from double)."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    g, lo, hi = _grid_small(cfg, n=17)
    nz, ny, nx = g.shape[1:]
    packed = _lib.pack_grid((torch.as_tensor(g).cuda(), lo, hi), layout="cells")
    # record: component pairs (Ex, Ey), (Ez, Bx), (By, Bz); float 16 p + 2 k + h
    # is coefficient k of component 2 p + h
    a = packed[3].view(nz - 1, ny - 1, nx - 1, 3, 8, 2).double().cpu().numpy()
    a = np.swapaxes(a, -1, -2).reshape(nz - 1, ny - 1, nx - 1, 6, 8)
    f = g.astype(np.float64)
    for (i, j, k) in ((0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)):
        val = (a[..., 0] + i * a[..., 1] + j * a[..., 2] + k * a[..., 3] + i * j * a[..., 4] + j * k * a[..., 5]
               + i * k * a[..., 6] + i * j * k * a[..., 7])
        ref = np.moveaxis(f[:, k:k + nz - 1, j:j + ny - 1, i:i + nx - 1], 0, -1)
        assert np.max(np.abs(val - ref)) <= 3 * 2.0 ** -24, (i, j, k)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fp32_phase64", "fp64"])
def test_cell_coefficient_layout_push_matches_oracle(precision):
    """The float pushes read the per-cell coefficients (7 FMA per component);
    the FP64 push falls back to the component arrays.  Workload-2 shape on a
    40^3 grid, 300 particles, 4000 steps, against the oracle."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=300)
    g, lo, hi = _grid_small(cfg)
    gd = torch.as_tensor(g).cuda()
    packed = _lib.pack_grid((gd, lo, hi), layout="cells")
    out, _, st = gpu_push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], precision, grid=packed)
    assert st == 0
    ref = oracle.push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], grid=(g, lo, hi), threads=THREADS)
    _check(out, ref, precision)
    if precision == "fp64":  # identical to the component-array push
        a, _, _ = gpu_push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], precision, grid=(gd, lo, hi))
        for k in a:
            np.testing.assert_array_equal(a[k], out[k])


@pytest.mark.gpu
def test_cell_layout_without_arrays_rejected_for_fp64():
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    g, lo, hi = _grid_small(cfg, n=9)
    gd = torch.as_tensor(g).cuda()
    packed = _lib.pack_grid((gd, lo, hi), layout="cells")
    gs = _lib.grid_struct(packed)
    for c in range(6):
        gs.f[c] = None
    parts = _lib.to_device(workloads.particles(cfg, n=10), "fp64")
    with _lib.Handle(cfg["pulse"]) as h:
        ps = _lib.particles_struct(parts, "fp64")
        import ctypes
        rc = _lib.lib().ap_gather_push(h.h, ctypes.byref(ps), ctypes.byref(gs), 0.0, 0.02, 5, 0, None,
                                       _lib._stream(None))
        assert rc == _lib.AP_ERR_ARG
        assert h.status() == 0


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fp32_phase64"])
def test_cell_cache_in_registers_or_shared_memory_identical(precision):
    """The autotuner may keep a thread's grid cell in registers or in shared
    memory, with any block shape: the per-particle arithmetic is the same, so
    the states are bit-identical; the batched kernel too."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=3000)
    g, lo, hi = _grid_small(cfg, n=33)
    packed = _lib.pack_grid((torch.as_tensor(g).cuda(), lo, hi), layout="cells")
    base, _, _ = gpu_push(cfg["pulse"], parts, -10.0, 0.02, 600, precision, grid=packed)
    with _lib.Handle(cfg["pulse"]) as h:
        for block, bps, gc in ((128, 0, 1), (64, 2, 1), (256, 0, 0), (96, 0, 1)):
            h.set_launch(block, bps, gc)
            dev = _lib.to_device(parts, precision)
            h.push(dev, -10.0, 0.02, 600, precision=precision, grid=packed)
            out = _lib.to_host(dev)
            for k in base:
                np.testing.assert_array_equal(out[k], base[k], err_msg=str((block, bps, gc, k)))
        assert h.status() == 0


@pytest.mark.gpu
def test_float_float_step_limit_rejected():
    """The float-float time base counts steps in float and reduces the carrier
    phase with a magic-number rounding valid below 2^22 (2 pi): a float-float
    call of 2^23 or more steps is rejected before any launch; 2^23 - 1 steps
    (no particles: nothing to do) and the double-phase variants are accepted."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    empty = {k: v[:0] for k, v in workloads.particles(cfg, n=1).items()}
    with _lib.Handle(cfg["pulse"]) as h:
        dev = _lib.to_device(workloads.particles(cfg, n=4), "fp32")
        with pytest.raises(_lib.APError) as e:
            h.push(dev, 0.0, 0.02, 1 << 23, precision="fp32")
        assert e.value.status == _lib.AP_ERR_ARG
        h.push(_lib.to_device(empty, "fp32"), 0.0, 0.02, (1 << 23) - 1, precision="fp32")
        h.push(_lib.to_device(empty, "fp32_phase64"), 0.0, 0.02, 1 << 23, precision="fp32_phase64")
        torch.cuda.synchronize()
        assert h.status() == 0
