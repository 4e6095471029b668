"""Multi-rank helpers for the APRIL filter (one process per GPU).

Candidate pairs are independent, so ranks split them with no exchange on the
data path: each rank filters a contiguous shard on its own GPU, against its
own resident copy of both sets.  The only collectives are outside the timed
kernels: a gather of the verdict bytes to rank 0 and the max-over-ranks
reduction of step times.

Shards are balanced by an estimate of each pair's work, |A(r)| + |A(s)| (the
length of the AA merge, an upper bound of Algorithm 2's first join), so that
ranks finish together despite list lengths that differ by orders of
magnitude.
"""
from __future__ import annotations

import numpy as np


def balanced_shards(cost: np.ndarray, world: int) -> list[tuple[int, int]]:
    """Split range(len(cost)) into `world` contiguous [lo, hi) ranges of about
    equal total cost (each rank gets at least one pair when there are enough)."""
    n = len(cost)
    if world <= 1 or n == 0:
        return [(0, n)] + [(n, n)] * max(world - 1, 0)
    csum = np.cumsum(np.asarray(cost, dtype=np.float64))
    total = csum[-1]
    cuts = [0]
    for k in range(1, world):
        c = int(np.searchsorted(csum, total * k / world, side="left")) + 1
        c = min(max(c, cuts[-1]), n)
        cuts.append(c)
    cuts.append(n)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def pair_cost(a_len_r: np.ndarray, a_len_s: np.ndarray, pr: np.ndarray, ps: np.ndarray) -> np.ndarray:
    """Per-pair work estimate |A(r)| + |A(s)|."""
    return a_len_r[pr].astype(np.int64) + a_len_s[ps].astype(np.int64)


def gather_verdicts(local: np.ndarray, shards: list[tuple[int, int]], rank: int, world: int, group=None):
    """Rank 0 receives the concatenated verdicts of all shards (others get None)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return local
    n_max = max(hi - lo for lo, hi in shards)
    buf = torch.zeros(n_max, dtype=torch.uint8)
    buf[: len(local)] = torch.from_numpy(np.asarray(local, dtype=np.uint8))
    if rank == 0:
        parts = [torch.zeros(n_max, dtype=torch.uint8) for _ in range(world)]
        dist.gather(buf, parts, dst=0, group=group)
        return np.concatenate([parts[k][: hi - lo].numpy() for k, (lo, hi) in enumerate(shards)])
    dist.gather(buf, None, dst=0, group=group)
    return None


def sharded_filter(cost: np.ndarray, world: int, rank: int, run_shard, group=None):
    """The multi-rank filter of one pair list: split the pairs into `world`
    contiguous shards of about equal cost, run run_shard(lo, hi) -> this
    rank's verdicts of pairs [lo, hi), and gather every rank's verdicts to
    rank 0.  Returns (shards, all verdicts on rank 0 / None elsewhere); with
    one rank, (the one shard, its verdicts)."""
    shards = balanced_shards(cost, world)
    lo, hi = shards[rank]
    local = np.asarray(run_shard(lo, hi), dtype=np.uint8)
    if len(local) != hi - lo:
        raise ValueError("run_shard returned the wrong number of verdicts")
    return shards, gather_verdicts(local, shards, rank, world, group)


def max_over_ranks(x: float, world: int, device=None, group=None) -> float:
    """The maximum of a scalar over ranks (step times: the job is as slow as its slowest rank)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
