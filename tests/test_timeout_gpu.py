"""The filter kernels' error path for a bounded wait that runs out (GPU only).

Every wait of a filter kernel for its window copies is bounded.  The
diagnostic april_debug_set_wait_limit(0) makes each such wait give up at
once, with no fault: the kernel then waits (bounded) for the copies in
flight, marks the pairs it held as APRIL_VERDICT_ERROR, records the timeout
and stops.  These tests check that april_sync_status reports it for the warp
and batched modes and for the filter variants, and that the context works
again at the default limit.
"""
import numpy as np
import pytest

from tests import _data
from paper_2307_01716_gb300 import april as A

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = _data.workload(3, 0.01)
    g = A.global_grid(w.order)
    R = A.april_build_sets(w.R.xy, w.R.off, g)
    S = A.april_build_sets(w.S.xy, w.S.off, g)
    dR, dS = A.april_upload(R), A.april_upload(S)
    d_r = torch.from_numpy(w.pr.view(np.int32)).cuda()
    d_s = torch.from_numpy(w.ps.view(np.int32)).cuda()
    want, _ = A.april_host_filter(R, S, w.pr, w.ps)
    return torch, w, dR, dS, d_r, d_s, want


def _run(torch, ctx, call, n):
    out = torch.full((n,), 0xEE, dtype=torch.uint8, device="cuda")
    try:
        A.april_debug_set_wait_limit(0)
        call(out)
        torch.cuda.synchronize()
    finally:
        A.april_debug_set_wait_limit(A.WAIT_LIMIT_DEFAULT)
    with pytest.raises(A.AprilError) as e:
        ctx.april_sync_status()
    assert e.value.status == -5
    got = out.cpu().numpy()
    assert int((got == 0xFF).sum()) > 0
    return got


@pytest.mark.parametrize("mode", ["warp", "batched"])
@pytest.mark.parametrize("long_scope", ["warp", "cta"])
def test_timeout_reported_then_recovers(setup, mode, long_scope):
    torch, w, dR, dS, d_r, d_s, want = setup
    n = len(w.pr)
    ctx = A.Context(0)
    t = ctx.get_tune()
    t.cta_threshold = 2048  # long pairs go to the warp or CTA scope under test
    t.cta_window = 64 if long_scope == "warp" else 256
    ctx.set_tune(t)
    m = A.MODES[mode]
    sb = ctx.scratch_bytes(m, n)
    scratch = torch.empty(max(sb, 256), dtype=torch.uint8, device="cuda") if sb else None
    _run(torch, ctx, lambda out: ctx.april_filter_pairs(dR, dS, d_r, d_s, n, out, m, scratch), n)
    out = torch.full((n,), 0xEE, dtype=torch.uint8, device="cuda")
    ctx.april_filter_pairs(dR, dS, d_r, d_s, n, out, m, scratch)
    ctx.april_sync_status()
    assert np.array_equal(out.cpu().numpy(), want)


def test_timeout_in_variant_kernel(setup):
    torch, w, dR, dS, d_r, d_s, want = setup
    n = len(w.pr)
    ctx = A.Context(0)
    scratch = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device="cuda")
    _run(torch, ctx, lambda out: ctx.april_filter_pairs_ex(dR, dS, d_r, d_s, n, out, A.PREDICATE_INTERSECTS,
                                                           scratch), n)
    out = torch.full((n,), 0xEE, dtype=torch.uint8, device="cuda")
    ctx.april_filter_pairs_ex(dR, dS, d_r, d_s, n, out, A.PREDICATE_INTERSECTS, scratch)
    ctx.april_sync_status()
    assert np.array_equal(out.cpu().numpy(), want)
