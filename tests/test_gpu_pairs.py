"""Two particles per thread (ap_launch_cfg.pairs = 1: every FP32 operation
packed over the two particles of a thread) against the oracle, with the
tolerances of the one-particle float-float push: median relative |du| <=
1e-4 and max <= 1e-3 after the run, |du| / max(|u_ref|, 1).

Covered: every pulse kind, every grid mode of the two-particle kernels (both
cells in shared memory, both in registers, one of each), the light-front and
histogram diagnostics, ragged sizes (a padding partner in the last pair),
the batched launch, and launch-shape independence: each half of a packed
instruction rounds like the scalar instruction, so a particle's arithmetic
does not depend on its partner, on the block size or on where its cell is
cached (bit-identical results)."""
import math

import numpy as np
import pytest

import oracle
from paper_2307_04843_gb300 import workloads
from support import THREADS, gpu_push, rel_u_err

L = 2 * math.pi
PAIRS = dict(block=128, pairs=1)


def _check(out, ref, med=1e-4, mx=1e-3):
    e = rel_u_err(out, ref)
    assert np.median(e) <= med, np.median(e)
    assert np.max(e) <= mx, (np.max(e), int(np.argmax(e)))


def _grid_small(cfg, n=40):
    lo, hi = workloads.grid_box(cfg)
    g = workloads.grid_field(cfg["box"], n, amplitude=0.1, n_terms=16, kmax=4)
    return g, lo, hi


@pytest.mark.gpu
def test_pairs_workload2_grid_cache_modes():
    """Gaussian a0 = 10 + longitudinal + a 40^3 grid read from its per-cell
    coefficient copy, 4000 steps, 301 particles (the last pair has a padding
    partner): every cache placement matches the oracle and they agree bit for
    bit with each other."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=301)
    g, lo, hi = _grid_small(cfg)
    packed = _lib.pack_grid((torch.as_tensor(g).cuda(), lo, hi), layout="cells")
    ref = oracle.push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], grid=(g, lo, hi), threads=THREADS)
    outs = []
    for gc in (0, 1, 2):
        out, _, st = gpu_push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], "fp32", grid=packed,
                              launch=dict(PAIRS, grid_cache=gc))
        assert st == 0
        _check(out, ref)
        outs.append(out)
    for o in outs[1:]:
        for k in o:
            np.testing.assert_array_equal(o[k], outs[0][k])
    assert np.max(np.abs(ref["ux"])) > 1.0


@pytest.mark.gpu
def test_pairs_workload3_lg_and_histogram():
    """CP LG_{1,2} inverse-Compton beam, 3000 steps, 601 particles: the
    trajectories match the oracle; the histogram equals the binning of the
    GPU's own final momenta bit for bit and holds every particle."""
    cfg = workloads.config(3)
    parts = workloads.particles(cfg, n=601)
    d = cfg["diag"]
    hist = (d["hist_bins"], d["hist_lo"], d["hist_hi"])
    out, dg, st = gpu_push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], "fp32", hist=hist,
                           launch=PAIRS)
    assert st == 0
    ref = oracle.push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], threads=THREADS)
    _check(out, ref)
    np.testing.assert_array_equal(dg["hist"], oracle.gamma_hist(out["ux"], out["uy"], out["uz"], *hist))
    assert dg["hist"].sum() == 601


@pytest.mark.gpu
def test_pairs_flying_focus_sum():
    """64-component flying focus, 25 particles placed where the focus passes,
    1500 steps."""
    cfg = workloads.config(4)
    p = workloads.particles(cfg, n=25)
    st_ = oracle.state(cfg["pulse"])
    t0 = cfg["t0"]
    zc = st_["z_mid"] + 0.99 * (t0 + 15.0 - st_["t_mid"]) - 40.0
    p["z"] = zc + (p["z"] / (200 * L) - 0.5) * 20.0
    p["x"] = p["x"] * 0.3
    p["y"] = p["y"] * 0.3
    out, _, st = gpu_push(cfg["pulse"], p, t0, cfg["dt"], 1500, "fp32", launch=PAIRS)
    assert st == 0
    ref = oracle.push(cfg["pulse"], p, t0, cfg["dt"], 1500, threads=THREADS)
    _check(out, ref)
    assert np.max(np.abs(ref["ux"])) > 0.5


@pytest.mark.gpu
@pytest.mark.parametrize("beta_f", [-1.0, 0.5])
def test_pairs_flying_focus_closed_form(beta_f):
    pulse = dict(kind="flying_cf", pol="x", env="gauss", env_len=30.0, a0=5.0, w0=3 * L, beta_f=beta_f,
                 z_focus=0.0, t_focus=0.0, longitudinal=True)
    rng = np.random.default_rng(23)
    n = 201
    parts = dict(x=rng.uniform(-1, 1, n) * 4 * L, y=rng.uniform(-1, 1, n) * 4 * L,
                 z=rng.uniform(-1, 1, n) * 6 * L, ux=np.zeros(n), uy=np.zeros(n), uz=np.zeros(n))
    out, _, st = gpu_push(pulse, parts, -40.0, 0.02, 2500, "fp32", launch=PAIRS)
    assert st == 0
    ref = oracle.push(pulse, parts, -40.0, 0.02, 2500, threads=THREADS)
    _check(out, ref)


@pytest.mark.gpu
def test_pairs_plane_wave_lightfront():
    """Workload 1 (plane wave, sin^2 envelope: its window is cleared per half
    of each pair) in float-float arithmetic with two particles per thread:
    final states match the oracle and the per-step light-front maximum over
    both halves tracks the oracle's."""
    cfg = workloads.config(1)
    parts = workloads.particles(cfg)
    out, dg, st = gpu_push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], "fp32",
                           diag_keys=("lightfront",), launch=PAIRS)
    assert st == 0
    ref, lf = oracle.push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], cfg["n_steps"], lf=True, threads=THREADS)
    _check(out, ref)
    assert np.max(np.abs(dg["lightfront"] - lf)) < 1e-5
    assert dg["lightfront"].max() < 2e-5


@pytest.mark.gpu
@pytest.mark.parametrize("n", [0, 1, 2, 63, 65, 257, 513])
def test_pairs_ragged_sizes(n):
    """Empty input is a no-op; sizes that leave a padding partner or a
    partial block match the oracle particle by particle (Gaussian beam, the
    particles inside the pulse)."""
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=n)
    for k in ("x", "y"):
        parts[k] = parts[k] * 0.2
    parts["z"] = parts["z"] * 0.05
    out, _, st = gpu_push(cfg["pulse"], parts, -10.0, 0.02, 800, "fp32", launch=PAIRS)
    assert st == 0
    assert out["x"].size == n
    if n:
        ref = oracle.push(cfg["pulse"], parts, -10.0, 0.02, 800, threads=THREADS)
        _check(out, ref)
        assert np.max(np.abs(ref["ux"])) > 1.0


@pytest.mark.gpu
def test_pairs_launch_shapes_bit_identical():
    """Block size and residency do not change a particle's arithmetic in the
    two-particle kernels either (its partner changes with the block size)."""
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=1001)
    base, _, _ = gpu_push(cfg["pulse"], parts, -5.0, 0.02, 300, "fp32", launch=dict(block=32, pairs=1))
    for block, bps in ((64, 2), (128, 0), (256, 1), (96, 0)):
        out, _, _ = gpu_push(cfg["pulse"], parts, -5.0, 0.02, 300, "fp32",
                             launch=dict(block=block, blocks_per_sm=bps, pairs=1))
        for k in base:
            np.testing.assert_array_equal(out[k], base[k], err_msg=str((block, bps, k)))


@pytest.mark.gpu
def test_pairs_split_calls():
    """700 + 500 steps agree with 1200 steps to float rounding (the second
    call re-derives its float-float phase base from its own t0)."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=77)
    with _lib.Handle(cfg["pulse"]) as h:
        h.set_launch(**PAIRS)
        a = _lib.to_device(parts, "fp32")
        b = _lib.to_device(parts, "fp32")
        dt = 2.0 ** -6
        h.push(a, -40.0, dt, 1200, precision="fp32")
        h.push(b, -40.0, dt, 700, precision="fp32")
        h.push(b, -40.0 + 700 * dt, dt, 500, precision="fp32")
        torch.cuda.synchronize()
        ha, hb = _lib.to_host(a), _lib.to_host(b)
    for k in ha:
        np.testing.assert_allclose(ha[k], hb[k], rtol=1e-6, atol=1e-6)


@pytest.mark.gpu
@pytest.mark.parametrize("tile", [0, 512, 1024])
def test_pairs_batched_matches_single_set_and_oracle(tile):
    """Batched launch with two particles per thread and tiles of 1, 2 or 4
    block-pairs: each particle equals, bit for bit, the two-particle push of
    its own set; per-set gamma sums match the oracle's."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(5)
    sets, counts = workloads.batch_sets(cfg)
    sets = sets[:7]
    counts = workloads.scaled_counts(counts[:7], 1400)
    counts[1] = 1
    counts[3] = 255
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    parts = workloads.particles_uniform(cfg["box"], int(off[-1]), workloads.seed_for(5))
    n_steps = 400
    with _lib.Handle(sets) as h:
        h.set_launch(block=128, pairs=1, tile=tile)
        dev = _lib.to_device(parts, "fp32")
        d_off = torch.as_tensor(off).cuda()
        ws = torch.zeros(_lib.ap_batch_workspace_bytes(h.h) // 4, dtype=torch.int32, device="cuda")
        diag = dict(set_sum=torch.zeros(len(sets), dtype=torch.float64, device="cuda"))
        _lib.ap_gather_push_batched(h.h, dev, d_off, None, cfg["t0"], cfg["dt"], n_steps, "fp32", diag, ws)
        assert h.status() == 0
        out = _lib.to_host(dev)
        sums = diag["set_sum"].cpu().numpy()
    refs = []
    for s in range(len(sets)):
        sl = slice(off[s], off[s + 1])
        sub = {k: v[sl] for k, v in parts.items()}
        one, _, _ = gpu_push(sets[s], sub, cfg["t0"], cfg["dt"], n_steps, "fp32", launch=PAIRS)
        for k in one:
            np.testing.assert_array_equal(out[k][sl], one[k])
        refs.append(oracle.push(sets[s], sub, cfg["t0"], cfg["dt"], n_steps, threads=THREADS))
    ref = {k: np.concatenate([r[k] for r in refs]) for k in refs[0]}
    _check(out, ref)
    np.testing.assert_allclose(sums, oracle.set_gamma_sums(off, ref["ux"], ref["uy"], ref["uz"]), rtol=1e-4)


@pytest.mark.gpu
def test_pairs_batched_tile_not_multiple_rejected():
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(5)
    sets, _ = workloads.batch_sets(cfg)
    sets = sets[:2]
    off = np.array([0, 10, 20], dtype=np.int64)
    parts = workloads.particles_uniform(cfg["box"], 20, 1)
    with _lib.Handle(sets) as h:
        h.set_launch(block=128, pairs=1, tile=384)  # not a multiple of 2 x 128
        dev = _lib.to_device(parts, "fp32")
        ws = torch.zeros(_lib.ap_batch_workspace_bytes(h.h) // 4, dtype=torch.int32, device="cuda")
        with pytest.raises(_lib.APError) as e:
            _lib.ap_gather_push_batched(h.h, dev, torch.as_tensor(off).cuda(), None, 0.0, 0.02, 5, "fp32",
                                        None, ws)
        assert e.value.status == _lib.AP_ERR_ARG


@pytest.mark.gpu
def test_pairs_plasma_pulse_push():
    """A circularly polarised plane wave in a plasma (Sec. 4: k, v_g, B0/E0
    and B's finite-duration terms) pushes 3001 electrons with two particles
    per thread as the oracle does."""
    pulse = dict(kind="plane", pol="cp", env="gauss", env_len=15.0, a0=0.8, omega_p=0.3, t_focus=30.0)
    rng = np.random.default_rng(21)
    n = 3001
    parts = dict(x=rng.uniform(-1, 1, n), y=rng.uniform(-1, 1, n), z=rng.uniform(-20.0, 20.0, n),
                 ux=rng.normal(0, 0.05, n), uy=rng.normal(0, 0.05, n), uz=rng.normal(0, 0.05, n))
    out, _, st = gpu_push(pulse, parts, 0.0, 0.05, 1200, "fp32", launch=PAIRS)
    assert st == 0
    idx = np.arange(0, n, 150)
    sub = {k: v[idx] for k, v in parts.items()}
    ref = oracle.push(pulse, sub, 0.0, 0.05, 1200)
    _check({k: v[idx] for k, v in out.items()}, ref)
    assert np.max(np.abs(ref["ux"])) > 0.3


@pytest.mark.gpu
def test_pairs_super_gaussian_and_lg_negative_l():
    """Two particles per thread through (a) a super-Gaussian (g = 3) plane
    wave and (b) an LG_{2,-3} beam with circular polarisation and
    longitudinal terms: the run-time loops of the envelope, the Laguerre
    recurrence and the (x - i y) powers in packed form, against the oracle."""
    rng = np.random.default_rng(29)
    n = 257
    pulses = [dict(kind="plane", pol="y", env="sgauss", sg_order=3, env_len=12.0, a0=2.0, t_focus=15.0),
              dict(kind="lg", pol="cm", env="gauss", env_len=20.0, a0=3.0, w0=2 * L, lg_p=2, lg_l=-3,
                   longitudinal=True, t_focus=20.0)]
    for pulse in pulses:
        parts = dict(x=rng.uniform(-1, 1, n) * 2 * L, y=rng.uniform(-1, 1, n) * 2 * L,
                     z=rng.uniform(-1, 1, n) * 2 * L, ux=np.zeros(n), uy=np.zeros(n), uz=np.zeros(n))
        out, _, st = gpu_push(pulse, parts, 0.0, 0.02, 2000, "fp32", launch=PAIRS)
        assert st == 0
        ref = oracle.push(pulse, parts, 0.0, 0.02, 2000, threads=THREADS)
        _check(out, ref)
        assert np.max(np.abs(ref["ux"]) + np.abs(ref["uy"])) > 0.5, pulse["kind"]


@pytest.mark.gpu
def test_pairs_one_d_sweep_holds_transverse_positions():
    """1D-3V sets (workload-6 shape, 30 lines x 41 electrons) in the batched
    launch with two particles per thread: transverse positions held to the
    float-float representation, momenta and per-line sums as the oracle's."""
    import torch
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(6)
    sets, parts, off = workloads.sweep_lines(cfg, per_set=41)
    n_steps = 2000
    with _lib.Handle(sets) as h:
        h.set_launch(block=64, pairs=1, tile=256)
        dev = _lib.to_device(parts, "fp32")
        d_off = torch.as_tensor(off).cuda()
        ws = torch.zeros(_lib.ap_batch_workspace_bytes(h.h) // 4, dtype=torch.int32, device="cuda")
        diag = dict(set_sum=torch.zeros(len(sets), dtype=torch.float64, device="cuda"))
        _lib.ap_gather_push_batched(h.h, dev, d_off, None, cfg["t0"], cfg["dt"], n_steps, "fp32", diag, ws)
        assert h.status() == 0
        out = _lib.to_host(dev)
        sums = diag["set_sum"].cpu().numpy()
    for k in ("x", "y"):
        assert np.all(np.abs(out[k] - parts[k]) <= 2.0 ** -46 * np.abs(parts[k])), k
    ref = oracle.push(sets[0], parts, cfg["t0"], cfg["dt"], n_steps, threads=THREADS)
    _check(out, ref)
    np.testing.assert_allclose(sums, oracle.set_gamma_sums(off, ref["ux"], ref["uy"], ref["uz"]), rtol=1e-5)


@pytest.mark.gpu
def test_launch_shape_arguments_checked():
    """ap_set_launch rejects particles-per-thread settings other than 0 or 1,
    cell placements other than 0, 1, 2, negative tiles and bad blocks; a
    rejected call leaves the handle usable."""
    from paper_2307_04843_gb300 import _lib
    cfg = workloads.config(2)
    with _lib.Handle(cfg["pulse"]) as h:
        for bad in (dict(pairs=2), dict(pairs=-1), dict(grid_cache=3), dict(tile=-1), dict(block=48),
                    dict(block=512), dict(blocks_per_sm=-1)):
            with pytest.raises(_lib.APError) as e:
                h.set_launch(**bad)
            assert e.value.status == _lib.AP_ERR_ARG, bad
        h.set_launch(block=96, pairs=1, grid_cache=2, tile=192)
        parts = workloads.particles(cfg, n=100)
        dev = _lib.to_device(parts, "fp32")
        h.push(dev, -5.0, 0.02, 50, precision="fp32")
        assert h.status() == 0
