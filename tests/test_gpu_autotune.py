"""Launch-shape autotuner: sweeps the candidates (block, residency, particles
per thread, cell placement; for the batched launch also the tile), caches
the fastest shape keyed by GPU, library build, kind, precision, grid and
size, reuses the cache, and the tuned shape gives the same particle states
as the default shape of the same particles-per-thread setting."""
import json

import numpy as np
import pytest

from paper_2307_04843_gb300 import workloads


@pytest.mark.gpu
def test_autotune_sweeps_caches_and_preserves_results(tmp_path):
    import torch
    from paper_2307_04843_gb300 import _lib, autotune
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=20000)
    cache = str(tmp_path / "tune.json")
    with _lib.Handle(cfg["pulse"]) as h:
        dev = _lib.to_device(parts, "fp32")
        snap = {k: v.clone() for k, v in dev.items()}
        r = autotune.tune(h, dev, -5.0, 0.02, "fp32", sample_n=20000, sample_steps=40,
                          candidates=((64, 0), (128, 0), (256, 1)), cache_path=cache)
        # one and two particles per thread, three shapes each
        assert not r["cached"] and len(r["sweep"]) == 6
        assert {s["pairs"] for s in r["sweep"]} == {0, 1}
        for k in dev:  # the caller's particles are not pushed
            assert torch.equal(dev[k], snap[k])
        data = json.load(open(cache))
        key = list(data)[0]
        assert len(data) == 1 and data[key]["block"] == r["block"]
        assert autotune.build_id() in key
        r2 = autotune.tune(h, dev, -5.0, 0.02, "fp32", cache_path=cache)
        assert r2["cached"] and r2["block"] == r["block"] and r2["pairs"] == r["pairs"]
        h.push(dev, -5.0, 0.02, 100, precision="fp32")
        tuned = _lib.to_host(dev)
    with _lib.Handle(cfg["pulse"]) as h:
        h.set_launch(pairs=r["pairs"])
        dev = _lib.to_device(parts, "fp32")
        h.push(dev, -5.0, 0.02, 100, precision="fp32")
        ref = _lib.to_host(dev)
    for k in ref:
        np.testing.assert_array_equal(tuned[k], ref[k])


@pytest.mark.gpu
def test_autotune_cells_grid_tries_every_cache_placement(tmp_path):
    """With a per-cell coefficient grid the sweep covers the cell in shared
    memory or registers (one particle per thread) and the three placements
    of two particles per thread."""
    import torch
    from paper_2307_04843_gb300 import _lib, autotune
    cfg = workloads.config(2)
    parts = workloads.particles(cfg, n=8000)
    lo, hi = workloads.grid_box(cfg)
    g = workloads.grid_field(cfg["box"], 33, torch_device="cuda")
    grid = _lib.pack_grid((g, lo, hi), layout="cells")
    with _lib.Handle(cfg["pulse"]) as h:
        dev = _lib.to_device(parts, "fp32")
        r = autotune.tune(h, dev, -5.0, 0.02, "fp32", grid, sample_n=8000, sample_steps=20,
                          candidates=((128, 0),), cache_path=str(tmp_path / "t.json"))
    modes = sorted((s["pairs"], s["grid_cache"]) for s in r["sweep"])
    assert modes == [(0, 0), (0, 1), (1, 0), (1, 1), (1, 2)]
    assert torch.cuda.is_available()


@pytest.mark.gpu
def test_autotune_batched_launch_bit_identical_and_cached(tmp_path):
    """The batched tuner sweeps block, residency, particles per thread and the
    tile over the caller's own sets; the tuned launch gives bit-identical
    states and per-set sums to the default shape of the same particles-per-
    thread setting, and is cached under its own key."""
    import torch
    from paper_2307_04843_gb300 import _lib, autotune
    cfg = workloads.config(5)
    sets, counts = workloads.batch_sets(cfg)
    sets = sets[:12]
    counts = workloads.scaled_counts(counts[:12], 6000)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    parts = workloads.particles_uniform(cfg["box"], int(off[-1]), workloads.seed_for(5))
    cache = str(tmp_path / "tune.json")
    d_off = torch.as_tensor(off).cuda()

    def run(h):
        dev = _lib.to_device(parts, "fp32")
        ws = torch.zeros(_lib.ap_batch_workspace_bytes(h.h) // 4, dtype=torch.int32, device="cuda")
        diag = dict(set_sum=torch.zeros(len(sets), dtype=torch.float64, device="cuda"))
        _lib.ap_gather_push_batched(h.h, dev, d_off, None, cfg["t0"], cfg["dt"], 150, "fp32", diag, ws)
        assert h.status() == 0
        return _lib.to_host(dev), diag["set_sum"].cpu().numpy()

    with _lib.Handle(sets) as h:
        dev = _lib.to_device(parts, "fp32")
        r = autotune.tune_batched(h, dev, d_off, cfg["t0"], cfg["dt"], "fp32", sample_steps=20,
                                  candidates=((64, 0), (128, 2)), tile_multiples=(1, 4), cache_path=cache)
        assert not r["cached"] and len(r["sweep"]) == 2 * 2 * 2
        assert all(s["tile"] % (s["block"] * (2 if s["pairs"] else 1)) == 0 for s in r["sweep"])
        tuned, tsum = run(h)
        r2 = autotune.tune_batched(h, dev, d_off, cfg["t0"], cfg["dt"], "fp32", cache_path=cache)
        assert r2["cached"] and (r2["block"], r2["tile"], r2["pairs"]) == (r["block"], r["tile"], r["pairs"])
    assert "batched" in list(json.load(open(cache)))[0]
    with _lib.Handle(sets) as h:
        h.set_launch(pairs=r["pairs"])
        ref, rsum = run(h)
    for k in ref:
        np.testing.assert_array_equal(tuned[k], ref[k])
    np.testing.assert_allclose(tsum, rsum, rtol=1e-13)
