"""Multi-rank path on CPU: two gloo ranks each push their shard (through the
oracle: no GPU here) and reduce the diagnostics; the result equals the
unsharded run.  Covers shard_range, shard_sets, reduce_sum/reduce_max and
scatter_set_sums."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2307_04843_gb300 import shard, workloads


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_shard_range_partitions():
    for n in (0, 1, 7, 100, 1001):
        for w in (1, 2, 3, 8):
            parts = [shard.shard_range(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            for a, b in zip(parts[:-1], parts[1:]):
                assert a[1] == b[0]
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def test_shard_sets_balanced_and_complete():
    counts = np.array([50, 7, 30, 30, 1, 90, 12, 44])
    owned = shard.shard_sets(counts, 3)
    flat = sorted(s for o in owned for s in o)
    assert flat == list(range(len(counts)))
    loads = [counts[o].sum() for o in owned]
    assert max(loads) - min(loads) <= counts.max()


def _worker(rank, world, port, result_path):
    import torch
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # workload-3 histogram on a particle shard
    cfg = workloads.config(3)
    parts = workloads.particles(cfg, n=64)
    a, b = shard.shard_range(64, rank, world)
    mine = {k: v[a:b] for k, v in parts.items()}
    out = oracle.push(cfg["pulse"], mine, cfg["t0"], cfg["dt"], 150)
    d = cfg["diag"]
    h = oracle.gamma_hist(out["ux"], out["uy"], out["uz"], d["hist_bins"], d["hist_lo"], d["hist_hi"])
    ht = torch.as_tensor(h.astype(np.int64))
    shard.reduce_sum(ht)
    # workload-5 per-set sums with whole sets per rank
    c5 = workloads.config(5)
    sets, counts = workloads.batch_sets(c5)
    sets, counts = sets[:5], workloads.scaled_counts(counts[:5], 40)
    off = np.concatenate([[0], np.cumsum(counts)])
    p5 = workloads.particles_uniform(c5["box"], int(off[-1]), workloads.seed_for(5))
    owned = shard.shard_sets(counts, world)[rank]
    local = []
    for s in owned:
        sub = {k: v[off[s]:off[s + 1]] for k, v in p5.items()}
        o = oracle.push(sets[s], sub, c5["t0"], c5["dt"], 100)
        local.append(oracle.set_gamma_sums(np.array([0, counts[s]]), o["ux"], o["uy"], o["uz"])[0])
    st = torch.as_tensor(shard.scatter_set_sums(np.array(local), owned, len(sets)))
    shard.reduce_sum(st)
    tm = torch.tensor([float(rank + 1)])
    shard.reduce_max(tm)
    if rank == 0:
        np.savez(result_path, hist=ht.numpy(), sums=st.numpy(), tmax=tm.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_unsharded(tmp_path):
    import oracle
    world = 2
    path = str(tmp_path / "res.npz")
    mp.start_processes(_worker, args=(world, _free_port(), path), nprocs=world, join=True,
                       start_method="spawn")
    res = np.load(path)
    cfg = workloads.config(3)
    parts = workloads.particles(cfg, n=64)
    out = oracle.push(cfg["pulse"], parts, cfg["t0"], cfg["dt"], 150)
    d = cfg["diag"]
    h = oracle.gamma_hist(out["ux"], out["uy"], out["uz"], d["hist_bins"], d["hist_lo"], d["hist_hi"])
    np.testing.assert_array_equal(res["hist"], h.astype(np.int64))
    c5 = workloads.config(5)
    sets, counts = workloads.batch_sets(c5)
    sets, counts = sets[:5], workloads.scaled_counts(counts[:5], 40)
    off = np.concatenate([[0], np.cumsum(counts)])
    p5 = workloads.particles_uniform(c5["box"], int(off[-1]), workloads.seed_for(5))
    ref = []
    for s in range(5):
        sub = {k: v[off[s]:off[s + 1]] for k, v in p5.items()}
        o = oracle.push(sets[s], sub, c5["t0"], c5["dt"], 100)
        ref.append(oracle.set_gamma_sums(np.array([0, counts[s]]), o["ux"], o["uy"], o["uz"])[0])
    np.testing.assert_allclose(res["sums"], ref, rtol=1e-14)
    assert res["tmax"][0] == 2.0
    assert not math.isnan(res["sums"].sum())
