"""Launch-shape autotuner: sweeps the candidates, caches the fastest shape
keyed by GPU, kind, precision, grid and size, reuses the cache, and the tuned
shape gives the same particle states as the default one."""
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
        assert not r["cached"] and len(r["sweep"]) == 3
        for k in dev:  # the caller's particles are not pushed
            assert torch.equal(dev[k], snap[k])
        data = json.load(open(cache))
        assert len(data) == 1 and list(data.values())[0]["block"] == r["block"]
        r2 = autotune.tune(h, dev, -5.0, 0.02, "fp32", cache_path=cache)
        assert r2["cached"] and r2["block"] == r["block"]
        h.push(dev, -5.0, 0.02, 100, precision="fp32")
        tuned = _lib.to_host(dev)
    with _lib.Handle(cfg["pulse"]) as h:
        dev = _lib.to_device(parts, "fp32")
        h.push(dev, -5.0, 0.02, 100, precision="fp32")
        ref = _lib.to_host(dev)
    for k in ref:
        np.testing.assert_array_equal(tuned[k], ref[k])
