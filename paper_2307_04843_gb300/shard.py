"""Host-side sharding of the push over ranks (one process per GPU).

The analytic field needs no communication (Sec. 2.3: each process evaluates
the pulse on its own, with no data from other processes), so the
particles -- or whole pulse sets of a batched run -- are split across ranks
and every rank pushes its shard independently.  The only exchange is one
final reduction of the diagnostics: histogram counts and per-set sums of
gamma (plain sums), done here with torch.distributed (NCCL on GPUs, gloo in
the CPU tests).  Nothing in this module touches the step loop.
"""
import numpy as np


def shard_range(n, rank, world):
    """Contiguous [start, stop) of n particles owned by `rank` (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(int(n), world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_sets(counts, world):
    """Assign whole pulse sets to ranks, balancing particle counts by the
    longest-processing-time rule (largest set to the least-loaded rank).
    Returns a list (per rank) of sorted set indices."""
    counts = np.asarray(counts, dtype=np.int64)
    order = np.argsort(-counts, kind="stable")
    load = np.zeros(world, dtype=np.int64)
    owned = [[] for _ in range(world)]
    for s in order:
        r = int(np.argmin(load))
        owned[r].append(int(s))
        load[r] += counts[s]
    return [sorted(o) for o in owned]


def shard_seed(base_seed, rank):
    """Seed of a rank's own shard in weak-scaling runs (independent streams)."""
    return int(base_seed) + 7919 * int(rank)


def reduce_sum(tensor, group=None):
    """In-place sum over ranks of a diagnostics tensor (counts or sums)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor


def reduce_max(tensor, group=None):
    """In-place max over ranks (the bench's timer: slowest rank)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.MAX, group=group)
    return tensor


def scatter_set_sums(local_sums, owned, n_sets):
    """Per-set sums of a rank's own sets placed into the global [n_sets]
    vector (zeros elsewhere), ready for reduce_sum."""
    out = np.zeros(n_sets)
    out[np.asarray(owned, dtype=np.int64)] = local_sums
    return out
