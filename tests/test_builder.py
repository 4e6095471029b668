"""Host logic of libapril (CPU only): april_build_sets produces exactly the
oracle's A/F cell sets as maximal Hilbert intervals, and the host execution
of Algorithm 2 over those lists gives the oracle's verdicts."""
import numpy as np
import pytest

import oracle
from synth import configs
from paper_2307_01716_gb300 import april as A


def _compare_lists(S, P, order, idx):
    g = oracle.Grid(order)
    for i in idx:
        La, Lf = oracle.cell_lists(P.poly(int(i)), g)
        ba = S.list(int(i), 0).astype(np.uint64)
        bf = S.list(int(i), 1).astype(np.uint64)
        # the device format stores end mod 2^32
        La[:, 1] %= np.uint64(1 << 32)
        Lf[:, 1] %= np.uint64(1 << 32)
        assert np.array_equal(La, ba), f"A-list of polygon {i}"
        assert np.array_equal(Lf, bf), f"F-list of polygon {i}"


@pytest.fixture(scope="module")
def cfg1():
    w = configs.make(1)
    g = A.global_grid(w.order)
    return w, A.april_build_sets(w.R.xy, w.R.off, g), A.april_build_sets(w.S.xy, w.S.off, g)


def test_lists_equal_oracle_config1(cfg1):
    w, R, S = cfg1
    _compare_lists(R, w.R, w.order, range(w.R.n))
    _compare_lists(S, w.S, w.order, range(0, w.S.n, 3))


@pytest.mark.parametrize("cfg", [2, 3])
def test_lists_equal_oracle_sampled(cfg):
    w = configs.make(cfg, scale=0.004)
    g = A.global_grid(w.order)
    R = A.april_build_sets(w.R.xy, w.R.off, g)
    rng = np.random.default_rng(cfg)
    _compare_lists(R, w.R, w.order, rng.choice(w.R.n, 150, replace=False))


def test_host_filter_equals_oracle_config1(cfg1):
    w, R, S = cfg1
    v, used = A.april_host_filter(R, S, w.pr, w.ps)
    ov = oracle.verdicts(w.R.xy, w.R.off, w.S.xy, w.S.off, w.pr, w.ps, oracle.Grid(w.order))
    assert np.array_equal(v, ov)
    assert np.all(used >= 2)
    counts = np.bincount(ov, minlength=3)
    assert counts.min() > 0


def _rect(x0, y0, x1, y1):
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], dtype=np.int64)


def test_degenerate_and_corner_polygons():
    """Grid-line edges, grid-corner vertices, and the last Hilbert cell
    (id 2^32-1 at N=16, whose interval end 2^32 is stored as 0)."""
    order = 16
    h = 1 << (24 - order)
    L = 1 << 24
    polys = [
        _rect(L - 3 * h, 0, L, 3 * h),                     # covers the last cell (2^16-1, 0)
        _rect(L - h, 0, L, h),                             # exactly the last cell
        _rect(0, 0, 2 * h, 2 * h),                         # covers cell 0
        _rect(10 * h, 10 * h, 20 * h, 30 * h),             # grid-aligned
        np.array([[5 * h, 5 * h], [9 * h, 5 * h + 7], [7 * h, 9 * h]]),
        np.array([[100 * h, 100 * h], [103 * h, 101 * h], [101 * h, 104 * h + h // 2]]),
    ]
    xy = np.concatenate(polys)
    off = np.zeros(len(polys) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(p) for p in polys])
    S = A.april_build_sets(xy, off, A.global_grid(order))

    class P:
        def poly(self, i):
            return polys[i]
    _compare_lists(S, P(), order, range(len(polys)))
    a0 = S.list(0, 0)
    assert a0[-1, 1] == 0, "end of the interval holding the last cell wraps to 0"
    n = len(polys)
    pr, ps = np.meshgrid(np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32), indexing="ij")
    pr, ps = pr.ravel(), ps.ravel()
    v, _ = A.april_host_filter(S, S, pr, ps)
    ov = oracle.verdicts(xy, off, xy, off, pr, ps, oracle.Grid(order))
    assert np.array_equal(v, ov)
    assert ov[0 * n + 1] == 1 and ov[0 * n + 2] == 0  # shares the last cell; far apart


def test_build_errors():
    bad = np.array([[0, 0], [5, 5]], dtype=np.int64)
    with pytest.raises(A.AprilError) as e:
        A.april_build_sets(bad, np.array([0, 2]), A.global_grid(12))
    assert e.value.status == -8
    with pytest.raises(A.AprilError) as e:
        A.april_build_sets(_rect(0, 0, 10, 10), np.array([0, 4]), A.grid(17, log2_cell=1))
    assert e.value.status == -1


def test_empty_set():
    S = A.april_build_sets(np.zeros((0, 2), np.int64), np.array([0]), A.global_grid(12))
    assert S.info().n_objects == 0


@pytest.mark.parametrize("cfg,scale", [(1, 1.0), (3, 0.01)])
def test_searched_host_filter(cfg, scale):
    """The kernels' reading (joins in the order AF, AA, FA, each from its
    searched start, galloping) keeps Algorithm 2's verdicts; per pair it
    reads no more than a full scan of the three joins plus the probes of the
    start searches and of at most one jump per 16 intervals read (each at
    most 32 probes), and in total less than sequential Algorithm 2."""
    from tests import _data
    w = _data.workload(cfg, scale)
    g = A.global_grid(w.order)
    R = A.april_build_sets(w.R.xy, w.R.off, g)
    S = A.april_build_sets(w.S.xy, w.S.off, g)
    v0, c0 = A.april_host_filter(R, S, w.pr, w.ps)
    v1, c1 = A.april_host_filter(R, S, w.pr, w.ps, searched=True)
    assert np.array_equal(v0, v1)
    a_r, f_r = R.lengths()
    a_s, f_s = S.lengths()
    bw = lambda v: np.floor(np.log2(np.maximum(v, 1))).astype(np.int64) + (v > 0)
    probes = 3 * (bw(np.maximum(a_r, f_r)[w.pr]) + bw(np.maximum(a_s, f_s)[w.ps]))
    full = 2 * a_r[w.pr].astype(np.int64) + 2 * a_s[w.ps] + f_r[w.pr] + f_s[w.ps]
    assert np.all(c1.astype(np.int64) <= full + probes + 2 * full)
    assert c1.sum() < c0.sum()


def test_searched_host_filter_partitioned():
    """The kernels' reading over partitioned sets (Sec. 5.2): the triage takes
    each pair's probe cell on the grid of the partition the routing picks; the
    verdicts stay Algorithm 2's, and the searched reading reads less than
    sequential Algorithm 2."""
    from tests import _data
    w = _data.workload(4, 0.02)
    R, S = A.april_build_partitioned_sets(w.R.xy, w.R.off, w.S.xy, w.S.off, w.partitions, w.order)
    v0, c0 = A.april_host_filter(R, S, w.pr, w.ps)
    v1, c1 = A.april_host_filter(R, S, w.pr, w.ps, searched=True)
    assert np.array_equal(v0, v1)
    assert c1.sum() < c0.sum()


def test_quantize_polygons():
    """Reading C3: x -> nearest integer of x * 2^24 (ties to even), clamped to
    [0, 2^24], consecutive and closing duplicates dropped; checked against
    numpy's rint (ties to even) on random and hand-made inputs."""
    rng = np.random.default_rng(4)
    polys = [rng.random((int(k), 2)) * 1.2 - 0.1 for k in rng.integers(3, 40, 50)]
    half = (np.array([[0.5, 1.5], [2.5, 3.5], [4.5, 4.5], [4.5, 4.5], [0.5, 1.5]]) / (1 << 24))
    polys.append(half)  # ties, a duplicate and a closing copy of the first vertex
    off = np.zeros(len(polys) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(p) for p in polys])
    q, qoff = A.april_quantize_polygons(np.concatenate(polys), off)
    for i, p in enumerate(polys):
        want = np.clip(np.rint(p * (1 << 24)), 0, 1 << 24).astype(np.int64)
        keep = [0] + [k for k in range(1, len(want)) if not np.array_equal(want[k], want[k - 1])]
        want = want[keep]
        while len(want) > 1 and np.array_equal(want[-1], want[0]):
            want = want[:-1]
        assert np.array_equal(q[qoff[i]:qoff[i + 1]], want), i
    assert q[qoff[-2]:qoff[-1]].tolist() == [[0, 2], [2, 4], [4, 4]]
    with pytest.raises(A.AprilError):
        A.april_quantize_polygons(np.array([[0.1, np.nan], [0.2, 0.2], [0.3, 0.1]]), [0, 3])
    # quantized polygons build
    ok = np.array([[0.1, 0.1], [0.2, 0.1], [0.15, 0.2]])
    qq, qo = A.april_quantize_polygons(ok, [0, 3])
    S = A.april_build_sets(qq, qo.astype(np.int64), A.global_grid(10))
    assert S.list(0, 0).shape[0] > 0
