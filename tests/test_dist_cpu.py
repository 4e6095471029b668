"""The multi-rank path on CPU: two gloo ranks run dist.sharded_filter, the
function bench.py's multi-rank run uses -- the candidate pairs split by
estimated cost, each rank's shard filtered (here by Algorithm 2 on the host
over the same built sets, where the bench runs the GPU filter), the verdicts
gathered to rank 0 -- and rank 0's gathered verdicts equal the
single-process result; the max-over-ranks reduction returns the slowest
rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2307_01716_gb300 import dist as D


def test_balanced_shards_cover_and_balance():
    rng = np.random.default_rng(0)
    cost = np.exp(rng.normal(5, 2, 10_000))  # heavy-tailed like list lengths
    for world in (1, 2, 3, 8):
        sh = D.balanced_shards(cost, world)
        assert sh[0][0] == 0 and sh[-1][1] == len(cost)
        assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
        loads = [cost[lo:hi].sum() for lo, hi in sh]
        assert max(loads) <= cost.sum() / world + cost.max() + 1e-6
    assert D.balanced_shards(np.zeros(0), 4) == [(0, 0)] * 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from tests import _data
        from paper_2307_01716_gb300 import april as A
        w = _data.workload(1, 1.0)
        g = A.global_grid(w.order)
        R = A.april_build_sets(w.R.xy, w.R.off, g)
        S = A.april_build_sets(w.S.xy, w.S.off, g)
        a_r, _ = R.lengths()
        a_s, _ = S.lengths()
        assert a_r.tolist() == [R.list(i, 0).shape[0] for i in range(w.R.n)]
        def run_shard(lo, hi):
            return A.april_host_filter(R, S, w.pr[lo:hi], w.ps[lo:hi], n_threads=1)[0]

        shards, allv = D.sharded_filter(D.pair_cost(a_r, a_s, w.pr, w.ps), world, rank, run_shard)
        assert shards[0][0] == 0 and shards[-1][1] == len(w.pr) and shards[0][1] == shards[1][0]
        t = D.max_over_ranks(float(rank + 1), world)
        if rank == 0:
            full, _ = A.april_host_filter(R, S, w.pr, w.ps, n_threads=1)
            q.put((bool(np.array_equal(allv, full)), t, len(allv)))
        else:
            assert allv is None
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_shard_and_gather():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ok, t, n = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ok and t == 2.0 and n > 1000
