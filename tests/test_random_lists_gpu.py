"""Adversarial parity of the merge joins (GPU only): random sorted interval
lists imported with april_sets_from_lists (not derived from polygons, so
they reach shapes polygons rarely do), filtered on the GPU in every mode and
several tunings, and compared verdict for verdict with the host's sequential
Algorithm 2 (april_host_filter, which the CPU tests pin to the oracle), and
the filter variants likewise with april_host_filter_ex.  The lists include
heavy-tailed lengths (up to thousands of intervals against a few), single
cells, intervals ending at the last cell of order 16 (end 2^32 written as
0), empty F-lists, and pairs of an object with itself; F-lists are random
sub-intervals of the A-lists, as every approximation's Full cells are among
the cells it meets."""
import numpy as np
import pytest

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


def _random_list(rng, order, k, hot):
    """k intervals with strictly increasing endpoints inside a random span
    (a hot region for most lists so that lists of different objects meet)."""
    top = 1 << (2 * order)
    if k == 0:
        return np.zeros((0, 2), np.uint64)
    span = int(min(top, max(4 * k, rng.integers(4 * k, 64 * k + 8))))
    lo = int(min(max(0, hot + rng.integers(-span, span)), top - span))
    pts = np.sort(rng.choice(span, 2 * k, replace=False)).astype(np.uint64) + np.uint64(lo)
    if rng.random() < 0.05:  # reach the very last cell
        pts = pts - pts[-1] + np.uint64(top - 1)
        pts[-1] = np.uint64(top)
        if pts[0] >= np.uint64(top) or np.any(np.diff(pts.astype(np.int64)) <= 0):
            return np.array([[top - 1, top]], np.uint64)
    return pts.reshape(-1, 2)


def _inner_list(rng, a):
    """Random F intervals inside the A intervals of `a` (an approximation's
    Full cells are among the cells it meets): for a random subset of A's
    intervals, one random sub-interval each."""
    if len(a) == 0 or rng.random() < 0.2:
        return np.zeros((0, 2), np.uint64)
    pick = np.flatnonzero(rng.random(len(a)) < rng.uniform(0.1, 0.9))
    out = []
    for st, en in a[pick].astype(np.int64).tolist():
        lo = int(rng.integers(st, en))
        hi = int(rng.integers(lo + 1, en + 1))
        out.append((lo, hi))
    return np.array(out, np.uint64).reshape(-1, 2)


def _random_sets(rng, n, order, hot):
    A_, F_ = [], []
    for _ in range(n):
        ka = int(min(6000, rng.pareto(1.2) * 8 + 1))
        a = _random_list(rng, order, ka, hot)
        A_.append(a)
        F_.append(_inner_list(rng, a))
    return A.april_sets_from_lists(order, A_, F_)


@pytest.fixture(scope="module")
def data():
    rng = np.random.default_rng(2024)
    hot = 1 << 30
    R = _random_sets(rng, 1500, 16, hot)
    S = _random_sets(rng, 1500, 16, hot)
    S14 = _random_sets(np.random.default_rng(7), 1500, 14, hot >> 4)
    n = 60_000
    pr = rng.integers(0, 1500, n).astype(np.uint32)
    ps = rng.integers(0, 1500, n).astype(np.uint32)
    pr[:1500] = np.arange(1500)  # every object with itself's counterpart index
    ps[:1500] = np.arange(1500)
    return R, S, S14, pr, ps


def _run(torch, ctx, dR, dS, pr, ps, fn):
    n = len(pr)
    d_r = torch.from_numpy(pr.view(np.int32)).cuda()
    d_s = torch.from_numpy(ps.view(np.int32)).cuda()
    out = torch.full((n,), 0xEE, dtype=torch.uint8, device="cuda")
    fn(d_r, d_s, out, n)
    ctx.april_sync_status()
    return out.cpu().numpy()


@pytest.mark.parametrize("mode,tune", [("plain", None), ("warp", None), ("warp", (2048, 4, 16, 64, 1)),
                                       ("batched", None), ("batched", (2048, 4, 16, 64)), ("batched", (0, 8, 32, 64)),
                                       ("batched", (64, 16, 32, 256)), ("batched", (0xFFFFFFFF, 32, 64, 256)),
                                       ("batched", (512, 4, 4, 2048)), ("batched", (2048, 4, 16, 64, 1)),
                                       ("batched", (0, 8, 32, 256, 1)), ("batched", (0xFFFFFFFF, 16, 32, 64, 1))])
def test_random_lists_equal_host(torch_cuda, ctx, data, mode, tune):
    torch = torch_cuda
    R, S, _, pr, ps = data
    want, _ = A.april_host_filter(R, S, pr, ps)
    assert np.bincount(want, minlength=3).min() > 100
    dR, dS = A.april_upload(R), A.april_upload(S)
    m = A.MODES[mode]
    saved = ctx.get_tune()
    if tune:
        ctx.set_tune(A.april_tune(*tune[:4], 0, 0.0, tune[4] if len(tune) > 4 else 0))
    try:
        def fn(d_r, d_s, out, n):
            sb = ctx.scratch_bytes(m, n)
            scratch = torch.empty(max(sb, 256), dtype=torch.uint8, device="cuda") if sb else None
            ctx.april_filter_pairs(dR, dS, d_r, d_s, n, out, m, scratch)
        got = _run(torch, ctx, dR, dS, pr, ps, fn)
    finally:
        ctx.set_tune(saved)
    bad = np.flatnonzero(got != want)
    assert len(bad) == 0, (len(bad), bad[:10])


@pytest.mark.parametrize("join_order", [0, 1])
@pytest.mark.parametrize("which", ["within", "coarser S", "coarser R"])
def test_random_lists_variants_equal_host(torch_cuda, ctx, data, which, join_order):
    torch = torch_cuda
    R, S, S14, pr, ps = data
    if which == "within":
        X, Y, pred = R, S, A.PREDICATE_WITHIN
    elif which == "coarser S":
        X, Y, pred = R, S14, A.PREDICATE_INTERSECTS
    else:
        X, Y, pred = S14, R, A.PREDICATE_INTERSECTS
    want, _ = A.april_host_filter_ex(X, Y, pr, ps, pred)
    assert np.bincount(want, minlength=3).min() > 10
    dX, dY = A.april_upload(X), A.april_upload(Y)
    for long_window in (64, 256):
        saved = ctx.get_tune()
        ctx.set_tune(A.april_tune(1024, saved.group_lanes, saved.group_window, long_window, 0, 0.0, join_order))
        try:
            def fn(d_r, d_s, out, n):
                scratch = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device="cuda")
                ctx.april_filter_pairs_ex(dX, dY, d_r, d_s, n, out, pred, scratch)
            got = _run(torch, ctx, dX, dY, pr, ps, fn)
        finally:
            ctx.set_tune(saved)
        bad = np.flatnonzero(got != want)
        assert len(bad) == 0, (which, long_window, len(bad), bad[:10])


@pytest.mark.parametrize("tune", [None, (2048, 4, 16, 64), (0, 8, 8, 64), (512, 16, 128, 256), (0xFFFFFFFF, 32, 64, 256),
                                  (2048, 4, 16, 64, 1)])
def test_random_lists_packed_equal_host(torch_cuda, ctx, data, tune):
    """The compressed form of random lists (per-block uint16/uint32 gaps)
    filters to the same verdicts as the host over the raw lists, with lane
    groups of every size and long pairs by warps or CTAs."""
    torch = torch_cuda
    _, _, _, pr, ps = data
    Rc = _random_sets(np.random.default_rng(11), 1500, 16, 1 << 30)
    Sc = _random_sets(np.random.default_rng(12), 1500, 16, 1 << 30)
    want, _ = A.april_host_filter(Rc, Sc, pr, ps)
    Rc.compress()
    Sc.compress()
    dR, dS = A.april_upload(Rc), A.april_upload(Sc)

    def fn(d_r, d_s, out, n):
        scratch = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED_PACKED, n), dtype=torch.uint8, device="cuda")
        ctx.april_filter_pairs(dR, dS, d_r, d_s, n, out, A.MODE_BATCHED_PACKED, scratch)
    saved = ctx.get_tune()
    if tune:
        ctx.set_tune(A.april_tune(*tune[:4], 0, 0.0, tune[4] if len(tune) > 4 else 0))
    try:
        got = _run(torch, ctx, dR, dS, pr, ps, fn)
    finally:
        ctx.set_tune(saved)
    assert np.array_equal(got, want), np.flatnonzero(got != want)[:10]


_BAND = 1 << 20  # galloping lists hold cells of q in [0, _BAND): 8 q .. 8 q + 7
_COMMON = np.linspace(1000, _BAND - 1000, 64).astype(np.int64)  # q's every dense list holds


def _gallop_list(rng, k, dense, cross):
    """A dense list: intervals [8 q, 8 q + 4) for k random q and every q of
    _COMMON.  A sparse list: intervals [8 q + 5, 8 q + 7) for k random q (they
    meet no dense interval), and, if cross, the one at a random q = c of
    _COMMON replaced by [8 c + 2, 8 c + 6), which meets every dense list."""
    q = np.sort(rng.choice(_BAND, k, replace=False)).astype(np.int64)
    if dense:
        q = np.union1d(q, _COMMON)
        iv = np.stack([8 * q, 8 * q + 4], axis=1)
    else:
        iv = np.stack([8 * q + 5, 8 * q + 7], axis=1)
        if cross:
            c = int(rng.choice(_COMMON))
            iv = np.concatenate([iv[q != c], [[8 * c + 2, 8 * c + 6]]])
            iv = iv[np.argsort(iv[:, 0])]
    return iv.astype(np.uint64)


def _gallop_sets(rng, n, dense):
    """Objects on order 16 whose A-lists are dense (500 to 20,000 intervals)
    or sparse (1 to 40, a third of them crossing); F-lists are random
    sub-intervals, as for _random_sets."""
    A_, F_ = [], []
    for _ in range(n):
        if dense:
            a = _gallop_list(rng, int(rng.integers(500, 20000)), True, False)
        else:
            a = _gallop_list(rng, int(rng.integers(1, 40)), False, rng.random() < 0.35)
        A_.append(a)
        F_.append(_inner_list(rng, a))
    return A.april_sets_from_lists(16, A_, F_)


@pytest.fixture(scope="module")
def gallop_data():
    """A set of objects with a few intervals each spread over the whole curve
    and a set of objects with thousands, where a merge join spends nearly all
    its steps on the long list and the kernels gallop over it; pairs in both
    roles (the short list as X and as Y)."""
    rng = np.random.default_rng(77)
    Sp = _gallop_sets(rng, 300, False)
    De = _gallop_sets(rng, 300, True)
    n = 12_000
    pr = rng.integers(0, 300, n).astype(np.uint32)
    ps = rng.integers(0, 300, n).astype(np.uint32)
    return Sp, De, pr, ps


@pytest.mark.parametrize("mode,tune", [("batched", None), ("batched", (0, 4, 32, 128)), ("batched", (0, 4, 32, 256)),
                                       ("batched", (2048, 8, 64, 64, 1)), ("batched", (0xFFFFFFFF, 16, 128, 256)),
                                       ("batched", (0xFFFFFFFF, 32, 256, 256)), ("batched", (0xFFFFFFFF, 4, 8, 64, 1)),
                                       ("warp", None), ("packed", None), ("packed", (0, 8, 64, 128))])
@pytest.mark.parametrize("roles", ["sparse X", "sparse Y"])
def test_galloping_equals_host(torch_cuda, ctx, gallop_data, mode, tune, roles):
    """Joins of a few intervals against thousands, with and without one
    planted overlap, in every scope that gallops (lane groups, warps, CTAs,
    compressed lists), equal host Algorithm 2 verdict for verdict."""
    torch = torch_cuda
    Sp, De, pr, ps = gallop_data
    R, S = (Sp, De) if roles == "sparse X" else (De, Sp)
    want, _ = A.april_host_filter(R, S, pr, ps)
    assert np.bincount(want, minlength=3)[:2].min() > 100  # true negatives and true hits both occur
    m = A.MODE_BATCHED_PACKED if mode == "packed" else A.MODES[mode]
    if mode == "packed":
        R = A.april_sets_from_lists(16, *_lists_of(R))
        S = A.april_sets_from_lists(16, *_lists_of(S))
        R.compress()
        S.compress()
    dR, dS = A.april_upload(R), A.april_upload(S)
    saved = ctx.get_tune()
    if tune:
        ctx.set_tune(A.april_tune(*tune[:4], 0, 0.0, tune[4] if len(tune) > 4 else 0))
    try:
        def fn(d_r, d_s, out, n):
            sb = ctx.scratch_bytes(m, n)
            scratch = torch.empty(max(sb, 256), dtype=torch.uint8, device="cuda") if sb else None
            ctx.april_filter_pairs(dR, dS, d_r, d_s, n, out, m, scratch)
        got = _run(torch, ctx, dR, dS, pr, ps, fn)
    finally:
        ctx.set_tune(saved)
    bad = np.flatnonzero(got != want)
    assert len(bad) == 0, (len(bad), bad[:10])


def _lists_of(sets):
    """The A- and F-lists of every object of `sets` (a fresh copy to compress)."""
    n = sets.info().n_objects
    return [sets.list(i, 0) for i in range(n)], [sets.list(i, 1) for i in range(n)]
