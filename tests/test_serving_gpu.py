"""Serving loop (GPU only): requests over resident sets, admitted by a memory
budget and stream slots, overlapping on the device.

* Every request's verdicts are the same when it runs alone and when it runs in
  the mix with others (bit-exact), and equal the oracle on a sample.
* A budget that fits only a few requests at once still completes every
  request, never exceeds the budget, and overlaps requests.
* Failure handling on the host: a request larger than the whole budget is
  refused, a queued request can be cancelled, a request with an out-of-range
  id fails alone, and shutting down with queued work neither hangs nor leaks.
"""
import time

import numpy as np
import pytest

from synth import serving
from tests import _data
from paper_2307_01716_gb300 import april as A

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def env(torch_cuda):
    w = _data.workload(5, 0.05)
    g = A.global_grid(w.order)
    R = A.april_build_sets(w.R.xy, w.R.off, g)
    S = A.april_build_sets(w.S.xy, w.S.off, g)
    dR, dS = A.april_upload(R), A.april_upload(S)
    ctx = A.Context(0)
    maker = serving.RequestMaker(w.R.mbr, w.S.mbr, w.pr, w.ps)
    reqs = maker.requests(seed=3, count=16, rate=0.0, lo=50, hi=20000)
    return w, ctx, dR, dS, reqs


def _host(torch, req):
    h_r = torch.from_numpy(req.pr.view(np.int32).copy()).pin_memory()
    h_s = torch.from_numpy(req.ps.view(np.int32).copy()).pin_memory()
    h_v = torch.full((len(req.pr),), 0xEE, dtype=torch.uint8).pin_memory()
    return h_r, h_s, h_v


def _serve(torch, ctx, dR, dS, reqs, max_inflight, arena_bytes, alone):
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    srv = A.Server(ctx, dR, dS, arena, max_inflight)
    outs = []
    try:
        if alone:
            for q in reqs:
                bufs = _host(torch, q)
                t = srv.april_submit(*bufs)
                assert srv.april_wait(t) is not None
                outs.append(bufs[2].numpy().copy())
        else:
            bufs = [_host(torch, q) for q in reqs]
            tickets = [srv.april_submit(*b) for b in bufs]
            for t in tickets:
                assert srv.april_wait(t) is not None
            outs = [b[2].numpy().copy() for b in bufs]
        info = srv.info()
    finally:
        srv.close()
    return outs, info


def test_alone_equals_mixed_equals_oracle(torch_cuda, env):
    w, ctx, dR, dS, reqs = env
    alone, _ = _serve(torch_cuda, ctx, dR, dS, reqs, 1, 1 << 28, alone=True)
    mixed, info = _serve(torch_cuda, ctx, dR, dS, reqs, 6, 1 << 28, alone=False)
    assert info.completed == len(reqs) and info.max_concurrent >= 2
    for a, m in zip(alone, mixed):
        assert np.array_equal(a, m)
    for q, v in zip(reqs[:4], alone[:4]):
        k = min(len(q.pr), 150)
        idx = np.sort(np.random.default_rng(1).choice(len(q.pr), k, replace=False))
        assert np.array_equal(v[idx], _data.oracle_sample_pairs(w, q.pr[idx], q.ps[idx]))


def test_budget_limits_admission(torch_cuda, env):
    w, ctx, dR, dS, reqs = env
    sizes = sorted(len(q.pr) for q in reqs)

    def need(n):  # a request's buffers: pairs, verdicts, the batched scratch, status (each 256-aligned)
        return 9 * n + ctx.scratch_bytes(A.MODE_BATCHED, n) + 8192
    budget = max(need(sizes[-1]), 3 * need(sizes[len(sizes) // 2]))
    budget = (budget + 255) // 256 * 256
    alone, _ = _serve(torch_cuda, ctx, dR, dS, reqs, 1, 1 << 28, alone=True)
    mixed, info = _serve(torch_cuda, ctx, dR, dS, reqs, 8, budget, alone=False)
    assert info.arena_peak_bytes <= info.arena_bytes <= budget
    assert info.completed == len(reqs)
    for a, m in zip(alone, mixed):
        assert np.array_equal(a, m)


def test_over_budget_cancel_bad_ids_and_shutdown(torch_cuda, env):
    torch = torch_cuda
    w, ctx, dR, dS, reqs = env
    arena = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    srv = A.Server(ctx, dR, dS, arena, 1)
    try:
        big = np.zeros(200_000, dtype=np.uint32)
        with pytest.raises(A.AprilError) as e:
            srv.april_submit(big, big, np.zeros(200_000, dtype=np.uint8))
        assert e.value.status == -3
        # a request with an out-of-range id fails on its own
        q = reqs[0]
        bad_r = q.pr.copy()
        bad_r[len(bad_r) // 2] = 10_000_000
        b_bad = (torch.from_numpy(bad_r.view(np.int32)).pin_memory(),
                 torch.from_numpy(q.ps.view(np.int32).copy()).pin_memory(),
                 torch.zeros(len(q.pr), dtype=torch.uint8).pin_memory())
        good = _host(torch, q)
        tickets = [srv.april_submit(*b_bad), srv.april_submit(*good)]
        # queue more behind one slot and cancel the last one before it runs
        extra = [_host(torch, reqs[i % len(reqs)]) for i in range(6)]
        et = [srv.april_submit(*b) for b in extra]
        cancelled = srv.april_cancel(et[-1])
        with pytest.raises(A.AprilError) as e:
            srv.april_wait(tickets[0])
        assert e.value.status == -2
        assert srv.april_wait(tickets[1]) is not None
        if cancelled == 0:
            with pytest.raises(A.AprilError) as e:
                srv.april_wait(et[-1])
            assert e.value.status == -6
    finally:
        t0 = time.time()
        srv.close()  # queued requests are cancelled, running ones finish
        assert time.time() - t0 < 60
