"""Parity of the filter variants on the GPU (april_filter_pairs_ex) with the
oracle, bit-exact: intersects on equal orders (Algorithm 2), on grids of
different order with either side the finer one (Sec. 5.3), and the within
filter (Sec. 4.3.2); configs 1-3 at reduced sizes with every pair checked,
both execution paths (whole-CTA joins and warp joins), the coarse-grid
triage on and off, config 2 at full size
on a sampled subset plus agreement with the host execution on every pair,
and the argument checks."""
import numpy as np
import pytest

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
def ctx(torch_cuda):
    return A.Context(0)


def _sets(w, o_r, o_s):
    R = A.april_build_sets(w.R.xy, w.R.off, A.global_grid(o_r))
    S = A.april_build_sets(w.S.xy, w.S.off, A.global_grid(o_s))
    return R, S, A.april_upload(R), A.april_upload(S)


def run_ex(torch, ctx, dR, dS, pr, ps, pred):
    n = len(pr)
    d_r = torch.from_numpy(np.ascontiguousarray(pr, dtype=np.uint32).view(np.int32)).cuda()
    d_s = torch.from_numpy(np.ascontiguousarray(ps, dtype=np.uint32).view(np.int32)).cuda()
    out = torch.full((max(n, 1),), 0xEE, dtype=torch.uint8, device="cuda")
    scratch = torch.empty(max(ctx.scratch_bytes(A.MODE_BATCHED, n), 256), dtype=torch.uint8, device="cuda")
    ctx.april_filter_pairs_ex(dR, dS, d_r, d_s, n, out, pred, scratch)
    ctx.april_sync_status()
    return out[:n].cpu().numpy()


def _variants(order):
    return [((order, order), 0), ((order, order - 2), 0), ((order - 2, order), 0), ((order, order - 4), 0),
            ((order, order), 1)]


@pytest.mark.parametrize("cfg,scale", [(1, 1.0), (2, 0.01), (3, 0.01)])
def test_variants_equal_oracle(torch_cuda, ctx, cfg, scale):
    w = _data.workload(cfg, scale)
    for (o_r, o_s), pred in _variants(w.order):
        _, _, dR, dS = _sets(w, o_r, o_s)
        got = run_ex(torch_cuda, ctx, dR, dS, w.pr, w.ps, pred)
        want = _data.oracle_verdicts_ex(cfg, scale, o_r, o_s, pred)
        assert np.array_equal(got, want), ((o_r, o_s), pred, np.nonzero(got != want)[0][:10])
        if (o_r, o_s) == (w.order, w.order) and pred == 0:
            assert np.array_equal(got, _data.oracle_verdicts(cfg, scale))


@pytest.mark.parametrize("long_window", [64, 256])
@pytest.mark.parametrize("threshold", [0, 64, 0xFFFFFFFF])
def test_variants_both_paths(torch_cuda, ctx, threshold, long_window):
    """Threshold 0 makes every pair a long pair, the maximum none; long pairs
    are joined by one warp (first window 64) or by the whole CTA (256)."""
    if threshold == 0xFFFFFFFF and long_window != 256:
        pytest.skip("no long pairs: the long-pair scope is unused")
    w = _data.workload(2, 0.01)
    saved = ctx.get_tune()
    ctx.set_tune(A.april_tune(threshold, saved.group_lanes, saved.group_window, long_window, 0, 0.0))
    try:
        for (o_r, o_s), pred in _variants(w.order):
            _, _, dR, dS = _sets(w, o_r, o_s)
            got = run_ex(torch_cuda, ctx, dR, dS, w.pr, w.ps, pred)
            want = _data.oracle_verdicts_ex(2, 0.01, o_r, o_s, pred)
            assert np.array_equal(got, want), ((o_r, o_s), pred, threshold)
    finally:
        ctx.set_tune(saved)


def test_variants_coarse_triage_on_and_off(torch_cuda, ctx):
    """On different orders the default tuning runs the coarse-grid triage
    first (Sec. 5.3 coarsening on nested global grids); with triage_off the
    variant kernel joins every pair.  Both equal the oracle."""
    w = _data.workload(2, 0.01)
    saved = ctx.get_tune()
    try:
        for off in (0, 1):
            t = ctx.get_tune()
            t.triage_off = off
            ctx.set_tune(t)
            for o_r, o_s in [(w.order, w.order - 2), (w.order - 2, w.order), (w.order, w.order - 4)]:
                _, _, dR, dS = _sets(w, o_r, o_s)
                got = run_ex(torch_cuda, ctx, dR, dS, w.pr, w.ps, 0)
                want = _data.oracle_verdicts_ex(2, 0.01, o_r, o_s, 0)
                assert np.array_equal(got, want), ((o_r, o_s), off, np.nonzero(got != want)[0][:10])
    finally:
        ctx.set_tune(saved)


def test_variants_full_size_config2_sampled(torch_cuda, ctx):
    w = _data.workload(2, 1.0)
    rng = np.random.default_rng(91)
    idx = np.sort(rng.choice(len(w.pr), 800, replace=False))
    for (o_r, o_s), pred in [((w.order, w.order - 2), 0), ((w.order - 2, w.order), 0), ((w.order, w.order), 1)]:
        R, S, dR, dS = _sets(w, o_r, o_s)
        got = run_ex(torch_cuda, ctx, dR, dS, w.pr, w.ps, pred)
        want = _data.oracle_pairs_ex(w, w.pr[idx], w.ps[idx], o_r, o_s, pred)
        assert np.array_equal(got[idx], want)
        hv, _ = A.april_host_filter_ex(R, S, w.pr, w.ps, pred)
        assert np.array_equal(got, hv)


def test_variants_arguments(torch_cuda, ctx):
    torch = torch_cuda
    w = _data.workload(1, 1.0)
    _, _, dR, dS = _sets(w, w.order, w.order - 2)
    n = len(w.pr)
    d_r = torch.from_numpy(w.pr.view(np.int32)).cuda()
    d_s = torch.from_numpy(w.ps.view(np.int32)).cuda()
    out = torch.zeros(n, dtype=torch.uint8, device="cuda")
    scratch = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AprilError):  # within needs one grid
        ctx.april_filter_pairs_ex(dR, dS, d_r, d_s, n, out, A.PREDICATE_WITHIN, scratch)
    with pytest.raises(A.AprilError):
        ctx.april_filter_pairs_ex(dR, dS, d_r, d_s, n, out, 5, scratch)
    with pytest.raises(A.AprilError):
        ctx.april_filter_pairs_ex(dR, dS, d_r, d_s, n, out, 0, scratch[:256])
    # out-of-range ids: error verdicts and an OUT_OF_RANGE_ID status
    bad_r = torch.from_numpy(np.array([0, w.R.n, 1], np.uint32).view(np.int32)).cuda()
    bad_s = torch.from_numpy(np.array([0, 0, w.S.n + 5], np.uint32).view(np.int32)).cuda()
    ctx.april_filter_pairs_ex(dR, dS, bad_r, bad_s, 3, out, 0, scratch)
    with pytest.raises(A.AprilError) as e:
        ctx.april_sync_status()
    assert e.value.status == -2
    assert out[1:3].cpu().tolist() == [0xFF, 0xFF]
    # partitioned sets are refused
    w4 = _data.workload(4, 0.005)
    Rp, Sp = A.april_build_partitioned_sets(w4.R.xy, w4.R.off, w4.S.xy, w4.S.off, 16, 14)
    with pytest.raises(A.AprilError):
        ctx.april_filter_pairs_ex(A.april_upload(Rp), A.april_upload(Sp), d_r, d_s, n, out, 0, scratch)
