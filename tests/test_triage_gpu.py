"""The batched filter's triage (GPU only): before the lane groups, every pair
whose MBR-intersection centre cell lies in A(r) and F(s), or in F(r) and
A(s), is settled as a true hit (an AF or FA overlap, Sec. 4.2).  Verdicts
with the triage on must equal those with it off and host Algorithm 2 (which
the CPU tests pin to the oracle), on sets uploaded from the host builder and
on sets built on the GPU, with bad ids among the pairs."""
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


def _run(torch, ctx, dR, dS, pr, ps, triage_off, mode=A.MODE_BATCHED):
    n = len(pr)
    saved = ctx.get_tune()
    t = A.april_tune(0xFFFFFFFF, 4, 32, 128, 0, 0.0, 0, 0, triage_off)
    ctx.set_tune(t)
    try:
        d_r = torch.from_numpy(pr.view(np.int32)).cuda()
        d_s = torch.from_numpy(ps.view(np.int32)).cuda()
        out = torch.full((n,), 0xEE, dtype=torch.uint8, device="cuda")
        scratch = torch.empty(ctx.scratch_bytes(mode, n), dtype=torch.uint8, device="cuda")
        ctx.april_filter_pairs(dR, dS, d_r, d_s, n, out, mode, scratch)
        try:
            ctx.april_sync_status()
        except A.AprilError as e:
            assert e.status == -2  # the bad ids planted below
        return out.cpu().numpy()
    finally:
        ctx.set_tune(saved)


@pytest.mark.parametrize("packed", [False, True])
@pytest.mark.parametrize("cfg,scale", [(1, 1.0), (2, 0.05), (3, 0.02)])
def test_triage_keeps_the_verdicts(torch_cuda, ctx, cfg, scale, packed):
    w = _data.workload(cfg, scale)
    g = A.global_grid(w.order)
    R = A.april_build_sets(w.R.xy, w.R.off, g)
    S = A.april_build_sets(w.S.xy, w.S.off, g)
    want_sets = (A.april_build_sets(w.R.xy, w.R.off, g), A.april_build_sets(w.S.xy, w.S.off, g))
    mode = A.MODE_BATCHED
    if packed:
        R.compress()
        S.compress()
        mode = A.MODE_BATCHED_PACKED
    dR, dS = A.april_upload(R), A.april_upload(S)
    assert dR.c.grid_known == 1 and dS.c.grid_known == 1
    pr, ps = np.array(w.pr, dtype=np.uint32), np.array(w.ps, dtype=np.uint32)
    pr[::997] = 0xFFFFFFF0  # bad ids: error verdicts either way
    want, _ = A.april_host_filter(*want_sets, pr, ps)
    on = _run(torch_cuda, ctx, dR, dS, pr, ps, 0, mode)
    off = _run(torch_cuda, ctx, dR, dS, pr, ps, 1, mode)
    assert np.array_equal(off, want)
    bad = np.flatnonzero(on != want)
    assert len(bad) == 0, (len(bad), bad[:10])
    assert (np.bincount(want[want < 3], minlength=3) > 0).all()


def test_triage_on_gpu_built_sets(torch_cuda, ctx):
    torch = torch_cuda
    w = _data.workload(2, 0.05)
    g = A.global_grid(w.order)
    S = A.april_build_sets(w.S.xy, w.S.off, g)
    Rh = A.april_build_sets(w.R.xy, w.R.off, g)
    d_xy = torch.from_numpy(np.ascontiguousarray(w.R.xy, dtype=np.int32)).cuda()
    d_off = torch.from_numpy(np.ascontiguousarray(w.R.off, dtype=np.int64)).cuda()
    dR, _ = ctx.april_build_sets_device(d_xy, d_off, g)
    dS = A.april_upload(S)
    assert dR.c.grid_known == 1
    pr, ps = np.array(w.pr, dtype=np.uint32), np.array(w.ps, dtype=np.uint32)
    want, _ = A.april_host_filter(Rh, S, pr, ps)
    assert np.array_equal(_run(torch, ctx, dR, dS, pr, ps, 0), want)


@pytest.mark.parametrize("packed", [False, True])
def test_triage_on_partitioned_sets(torch_cuda, ctx, packed):
    """Partitioned sets (Sec. 5.2): each pair's probe cell is taken on the grid
    of the partition the routing picks, and looked up in the entries' lists,
    raw or compressed (Sec. 5.1)."""
    w = _data.workload(4, 0.05)
    R, S = A.april_build_partitioned_sets(w.R.xy, w.R.off, w.S.xy, w.S.off, w.partitions, w.order)
    mode = A.MODE_BATCHED
    if packed:
        R.compress()
        S.compress()
        mode = A.MODE_BATCHED_PACKED
    dR, dS = A.april_upload(R), A.april_upload(S)
    assert dR.c.grid_known == 1 and dR.c.grid_id == dS.c.grid_id and dR.c.part_grid
    pr, ps = np.array(w.pr, dtype=np.uint32), np.array(w.ps, dtype=np.uint32)
    pr[::1009] = 0xFFFFFFF0
    want, _ = A.april_host_filter(R, S, pr, ps)
    assert np.array_equal(_run(torch_cuda, ctx, dR, dS, pr, ps, 1, mode), want)
    bad = np.flatnonzero(_run(torch_cuda, ctx, dR, dS, pr, ps, 0, mode) != want)
    assert len(bad) == 0, (len(bad), bad[:10])


def test_no_triage_across_different_grids(torch_cuda, ctx):
    """Sets on grids of the same order but other origins have different
    fingerprints, so the triage stays off (a cell id means another cell on
    each side) and the verdicts are host Algorithm 2's over the given lists."""
    w = _data.workload(1, 1.0)
    R = A.april_build_sets(w.R.xy, w.R.off, A.global_grid(w.order))
    g2 = A.global_grid(w.order)
    g2.ox -= 1 << g2.log2_cell
    S = A.april_build_sets(w.S.xy, w.S.off, g2)
    dR, dS = A.april_upload(R), A.april_upload(S)
    assert dR.c.grid_id != dS.c.grid_id
    pr, ps = np.array(w.pr, dtype=np.uint32), np.array(w.ps, dtype=np.uint32)
    want, _ = A.april_host_filter(R, S, pr, ps)
    assert np.array_equal(_run(torch_cuda, ctx, dR, dS, pr, ps, 0), want)
