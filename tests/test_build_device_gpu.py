"""GPU construction (april_build_sets_device) against the host builder and
the oracle: every polygon's A- and F-list equals april_build_sets' list for
list (which test_builder pins to the oracle's cell sets), the MBRs match,
the filter over device-built sets gives the oracle's verdicts, and a
selection batch whose query lists were built on the GPU returns the same
pairs and verdicts as host-built ones.  Edge cases: a polygon on the last
Hilbert cell (end 2^32 stored as 0), a polygon holding the whole grid (no
touched cell), polygons that miss every cell or have < 3 vertices
(errors), and buffers that are too small (sizes reported)."""
import numpy as np
import pytest

import oracle
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


def _device_polys(torch, xy, off):
    d_xy = torch.from_numpy(np.ascontiguousarray(xy, dtype=np.int32)).cuda()
    d_off = torch.from_numpy(np.ascontiguousarray(off, dtype=np.int64)).cuda()
    return d_xy, d_off


def _read_lists(dev: A.DevSets, n):
    """Host copies of a device image's lists: [(A, F)] as (k, 2) uint32."""
    img = dev.buf.cpu().numpy()
    base = dev.buf.data_ptr()
    desc = img[dev.c.desc - base:dev.c.desc - base + 16 * n].view(np.uint32).reshape(n, 4)
    iv = img[dev.c.iv - base:].view(np.uint32)
    out = []
    for a_off, a_len, f_off, f_len in desc.tolist():
        out.append((iv[2 * a_off:2 * (a_off + a_len)].reshape(-1, 2), iv[2 * f_off:2 * (f_off + f_len)].reshape(-1, 2)))
    mbr = img[dev.c.mbr - base:dev.c.mbr - base + 16 * n].view(np.int32).reshape(n, 4)
    return out, mbr


def _check_equal_host(torch, ctx, xy, off, grd):
    n = len(off) - 1
    H = A.april_build_sets(xy, off, grd)
    dev, info = ctx.april_build_sets_device(*_device_polys(torch, xy, off), grd)
    torch.cuda.synchronize()
    lists, mbr = _read_lists(dev, n)
    for p in range(n):
        assert np.array_equal(lists[p][0], H.list(p, 0)), ("A", p)
        assert np.array_equal(lists[p][1], H.list(p, 1)), ("F", p)
    assert np.array_equal(mbr, H.mbrs())
    return H, dev, info


@pytest.mark.parametrize("cfg,scale", [(1, 1.0), (2, 0.01), (3, 0.01)])
def test_device_lists_equal_host(torch_cuda, ctx, cfg, scale):
    w = _data.workload(cfg, scale)
    g = A.global_grid(w.order)
    for P in (w.R, w.S):
        _, _, info = _check_equal_host(torch_cuda, ctx, P.xy, P.off, g)
        assert info.touched_cells > 0 and info.image_bytes > 0


def test_device_sets_filter_to_oracle(torch_cuda, ctx):
    torch = torch_cuda
    w = _data.workload(1, 1.0)
    g = A.global_grid(w.order)
    dR, _ = ctx.april_build_sets_device(*_device_polys(torch, w.R.xy, w.R.off), g)
    dS, _ = ctx.april_build_sets_device(*_device_polys(torch, w.S.xy, w.S.off), g)
    n = len(w.pr)
    d_r = torch.from_numpy(w.pr.view(np.int32)).cuda()
    d_s = torch.from_numpy(w.ps.view(np.int32)).cuda()
    out = torch.zeros(n, dtype=torch.uint8, device="cuda")
    scratch = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device="cuda")
    ctx.april_filter_pairs(dR, dS, d_r, d_s, n, out, A.MODE_BATCHED, scratch)
    ctx.april_sync_status()
    assert np.array_equal(out.cpu().numpy(), _data.oracle_verdicts(1, 1.0))


def _rect(x0, y0, x1, y1):
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], dtype=np.int64)


def _pack(polys):
    xy = np.concatenate(polys)
    off = np.zeros(len(polys) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(p) for p in polys])
    return xy, off


def test_device_edge_cases(torch_cuda, ctx):
    torch = torch_cuda
    # the last Hilbert cell at N=16 and polygons along grid lines and corners
    h = 1 << 8
    L = 1 << 24
    xy, off = _pack([_rect(L - 3 * h, 0, L, 3 * h), _rect(L - h, 0, L, h), _rect(0, 0, 2 * h, 2 * h),
                     _rect(10 * h, 10 * h, 20 * h, 30 * h), _rect(19 * h, 29 * h, 40 * h, 40 * h),
                     np.array([[5 * h, 5 * h], [9 * h, 5 * h], [5 * h, 9 * h]], dtype=np.int64)])
    _check_equal_host(torch, ctx, xy, off, A.global_grid(16))
    # a grid of 16 x 16 cells of side 4 inside a polygon that holds all of it
    small = A.april_grid(0, 0, 2, 4)
    xy, off = _pack([_rect(-10, -10, 100, 100), _rect(3, 3, 9, 9)])
    H, dev, info = _check_equal_host(torch, ctx, xy, off, small)
    assert H.list(0, 0).tolist() == [[0, 256]] and H.list(0, 1).tolist() == [[0, 256]]
    # an L around the grid that meets no cell, and a two-vertex polygon: errors
    ell = np.array([[-20, -20], [100, -20], [100, -10], [-10, -10], [-10, 100], [-20, 100]], dtype=np.int64)
    for bad in ([_rect(3, 3, 9, 9), ell], [_rect(3, 3, 9, 9), np.array([[1, 1], [5, 5]], dtype=np.int64)]):
        xy, off = _pack(bad)
        with pytest.raises(A.AprilError) as e:
            A.april_build_sets(xy, off, small)
        assert e.value.status == -8
        with pytest.raises(A.AprilError) as e:
            ctx.april_build_sets_device(*_device_polys(torch, xy, off), small)
        assert e.value.status == -8 and "polygon 1" in str(e.value)


def test_device_build_buffer_sizes(torch_cuda, ctx):
    torch = torch_cuda
    w = _data.workload(1, 0.3)
    d_xy, d_off = _device_polys(torch, w.R.xy, w.R.off)
    info = A.april_device_build_info()
    out = A.april_dev_sets()
    lib = A.load()
    g = A.global_grid(w.order)
    st = torch.cuda.current_stream().cuda_stream
    n = w.R.n
    assert lib.april_build_sets_device(ctx.handle, d_xy.data_ptr(), d_off.data_ptr(), n, g, None, 0, None, 0, out,
                                       info, st) == -3
    small = info.work_bytes
    work = torch.empty(small, dtype=torch.uint8, device="cuda")
    assert lib.april_build_sets_device(ctx.handle, d_xy.data_ptr(), d_off.data_ptr(), n, g, work.data_ptr(), small,
                                       None, 0, out, info, st) == -3
    assert info.work_bytes > small and info.image_bytes > 0 and info.touched_cells > 0
    work = torch.empty(info.work_bytes, dtype=torch.uint8, device="cuda")
    image = torch.empty(info.image_bytes, dtype=torch.uint8, device="cuda")
    assert lib.april_build_sets_device(ctx.handle, d_xy.data_ptr(), d_off.data_ptr(), n, g, work.data_ptr(),
                                       info.work_bytes, image.data_ptr(), info.image_bytes - 256, out, info, st) == -3
    assert lib.april_build_sets_device(ctx.handle, d_xy.data_ptr(), d_off.data_ptr(), n, g, work.data_ptr(),
                                       info.work_bytes, image.data_ptr(), info.image_bytes, out, info, st) == 0
    torch.cuda.synchronize()


def test_selection_with_device_built_queries(torch_cuda, ctx):
    torch = torch_cuda
    from synth import selection
    s = selection.make(0.05, 80)
    g = A.global_grid(s.order)
    R = A.april_build_sets(s.R.xy, s.R.off, g)
    dR = A.april_upload(R)
    dI = A.april_index_upload(A.april_index_build(R))
    Qh = A.april_upload(A.april_build_sets(s.Q.xy, s.Q.off, g))
    Qd, _ = ctx.april_build_sets_device(*_device_polys(torch, s.Q.xy, s.Q.off), g)
    res = []
    for Q in (Qh, Qd):
        cap = 100_000
        d_r = torch.empty(cap, dtype=torch.int32, device="cuda")
        d_q = torch.empty(cap, dtype=torch.int32, device="cuda")
        d_v = torch.empty(cap, dtype=torch.uint8, device="cuda")
        off = torch.empty(s.Q.n + 1, dtype=torch.int32, device="cuda")
        scratch = torch.empty(ctx.select_scratch_bytes(cap), dtype=torch.uint8, device="cuda")
        n = ctx.april_select(dI, dR, Q, cap, d_r, d_q, d_v, off, scratch)
        ctx.april_sync_status()
        res.append((d_r[:n].cpu().numpy(), d_q[:n].cpu().numpy(), d_v[:n].cpu().numpy()))
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)
    assert len(res[0][0]) > 300


def test_device_sets_variants_equal_host(torch_cuda, ctx):
    """The filter variants over GPU-built sets (within; S on a coarser grid)
    give the host execution's verdicts over host-built sets."""
    torch = torch_cuda
    w = _data.workload(2, 0.01)
    gR, gS2 = A.global_grid(w.order), A.global_grid(w.order - 2)
    R = A.april_build_sets(w.R.xy, w.R.off, gR)
    S = A.april_build_sets(w.S.xy, w.S.off, gR)
    S2 = A.april_build_sets(w.S.xy, w.S.off, gS2)
    dR, _ = ctx.april_build_sets_device(*_device_polys(torch, w.R.xy, w.R.off), gR)
    dS, _ = ctx.april_build_sets_device(*_device_polys(torch, w.S.xy, w.S.off), gR)
    dS2, _ = ctx.april_build_sets_device(*_device_polys(torch, w.S.xy, w.S.off), gS2)
    n = len(w.pr)
    d_r = torch.from_numpy(w.pr.view(np.int32)).cuda()
    d_s = torch.from_numpy(w.ps.view(np.int32)).cuda()
    scratch = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device="cuda")
    for host_S, dev_S, pred in ((S, dS, A.PREDICATE_WITHIN), (S2, dS2, A.PREDICATE_INTERSECTS)):
        out = torch.full((n,), 0xEE, dtype=torch.uint8, device="cuda")
        ctx.april_filter_pairs_ex(dR, dev_S, d_r, d_s, n, out, pred, scratch)
        ctx.april_sync_status()
        want, _ = A.april_host_filter_ex(R, host_S, w.pr, w.ps, pred)
        assert np.array_equal(out.cpu().numpy(), want), pred
