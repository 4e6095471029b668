"""Pins of the filter variants (CPU only) and the host execution against them.

* Different granularity (Sec. 5.3): a polygon's A-cells on a fine grid,
  lifted to the coarse grid that nests it, are exactly its A-cells on the
  coarse grid (a closed coarse cell that meets the polygon contains a closed
  fine cell that meets it at the same point, and conversely).  So the
  mixed-order verdicts must equal the cell-table rule evaluated directly on
  the coarse grid with A(fine side) read there: no common A cell -> true
  negative; an A cell of the fine side in F of the coarse side -> true hit.
  Also sound against exact geometry, and equal to the plain filter when the
  orders agree.
* Within (Sec. 4.3.2): a true hit needs A(r) inside F(s), so r lies in s;
  checked against necessary conditions of containment computed exactly
  (every vertex of r in closed s, no proper edge crossing), against the
  closed form for axis-parallel rectangles, and the special case r within r
  (boundary cells are never full, so always inconclusive).
"""
import numpy as np
import pytest

import oracle
from tests import _brute as B
from tests.test_oracle_pins import _rect, _small_sets


def _all_pairs(n):
    pr, ps = np.meshgrid(np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32), indexing="ij")
    return pr.ravel(), ps.ravel()


def _table_on_coarse(polys, pr, ps, order, fine_side):
    """The Sec. 5.3 rule on the coarse grid of `order`, from oracle.cells
    (direct classification there, no lifting)."""
    g = oracle.Grid(order)
    cells = [oracle.cells(p, g) for p in polys]
    out = np.zeros(len(pr), dtype=np.uint8)
    for k, (r, s) in enumerate(zip(pr, ps)):
        Ar, Fr = cells[r]
        As, Fs = cells[s]
        if not (Ar & As):
            out[k] = 0
        elif (fine_side == "r" and Ar & Fs) or (fine_side == "s" and Fr & As):
            out[k] = 1
        else:
            out[k] = 2
    return out


@pytest.mark.parametrize("orders", [(6, 4), (4, 6), (7, 4), (5, 5)])
def test_mixed_granularity_equals_coarse_table(orders):
    polys, xy, off, _ = _small_sets(31, 24, 4)
    pr, ps = _all_pairs(len(polys))
    o_r, o_s = orders
    v = oracle.verdicts_ex(xy, off, xy, off, pr, ps, o_r, o_s)
    if o_r == o_s:
        want = oracle.verdicts(xy, off, xy, off, pr, ps, oracle.Grid(o_r))
    else:
        want = _table_on_coarse(polys, pr, ps, min(orders), "r" if o_r > o_s else "s")
    assert np.array_equal(v, want)
    assert np.bincount(v, minlength=3).min() > 0


def test_mixed_granularity_sound_against_exact_geometry():
    polys, xy, off, _ = _small_sets(37, 30, 4)
    pr, ps = _all_pairs(len(polys))
    for o_r, o_s in ((7, 5), (5, 7)):
        v = oracle.verdicts_ex(xy, off, xy, off, pr, ps, o_r, o_s)
        for k in np.flatnonzero(v != 2):
            inter = B.polygons_intersect(polys[pr[k]].tolist(), polys[ps[k]].tolist())
            assert inter == (v[k] == 1), (o_r, o_s, pr[k], ps[k])


def _contained_necessary(P, Q):
    """Exact necessary conditions for closed P inside closed Q: every vertex
    of P in closed Q, and no edge of P crosses an edge of Q properly."""
    P, Q = P.tolist(), Q.tolist()
    if not all(B.point_in_or_on(p, Q) for p in P):
        return False
    for i in range(len(P)):
        a, b = P[i], P[(i + 1) % len(P)]
        for j in range(len(Q)):
            c, d = Q[j], Q[(j + 1) % len(Q)]
            o1, o2 = B.orient(a, b, c), B.orient(a, b, d)
            o3, o4 = B.orient(c, d, a), B.orient(c, d, b)
            if o1 * o2 < 0 and o3 * o4 < 0:
                return False
    return True


def test_within_sound_against_exact_geometry():
    rng = np.random.default_rng(5)
    polys, _, _, g = _small_sets(41, 24, 5)
    # add small polygons inside larger ones so that true hits occur
    for k in range(24):
        P = polys[k]
        c = P.mean(0).astype(np.int64)
        d = int(g.h * rng.uniform(0.2, 1.5))
        polys.append(_rect(c[0] - d, c[1] - d, c[0] + d, c[1] + d))
    xy = np.concatenate(polys)
    off = np.zeros(len(polys) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(p) for p in polys])
    pr, ps = _all_pairs(len(polys))
    for order in (5, 7):
        v = oracle.verdicts_ex(xy, off, xy, off, pr, ps, order, order, oracle.WITHIN)
        assert (v == 1).sum() > 0 and (v == 0).sum() > 0
        inter = oracle.verdicts(xy, off, xy, off, pr, ps, oracle.Grid(order))
        assert np.all(inter[v == 1] == 1), "r within s implies r meets s"
        assert np.array_equal(v == 0, inter == 0)
        for k in np.flatnonzero(v == 1):
            assert _contained_necessary(polys[pr[k]], polys[ps[k]]), (order, pr[k], ps[k])
        for k in np.flatnonzero(v == 0):
            assert not B.polygons_intersect(polys[pr[k]].tolist(), polys[ps[k]].tolist())


def test_within_self_is_inconclusive():
    polys, xy, off, _ = _small_sets(43, 20, 5)
    idx = np.arange(len(polys), dtype=np.uint32)
    v = oracle.verdicts_ex(xy, off, xy, off, idx, idx, 6, 6, oracle.WITHIN)
    assert np.all(v == 2)


def _cell_range_meets(lo, hi, h, G):
    return max(-(-lo // h) - 1, 0), min(hi // h, G - 1)


def _cell_range_full(lo, hi, h):
    return -(-lo // h), hi // h - 1


def test_within_rectangles_closed_form():
    """For axis-parallel rectangles the A range of r per axis is the cells
    [ceil(lo/h) - 1, floor(hi/h)] (closed cells touching the closed side)
    and the F range of s is [ceil(lo/h), floor(hi/h) - 1]; r within s is a
    true hit iff r's A box lies in s's F box on both axes."""
    rng = np.random.default_rng(9)
    g = oracle.Grid(5)
    h, G = g.h, g.G
    rects = []
    for _ in range(60):
        x0, y0 = (int(v) for v in rng.integers(2 * h, (G - 10) * h, 2))
        w_, h_ = (int(v) for v in rng.integers(h // 3, 6 * h, 2))
        if rng.random() < 0.4:  # snap to grid lines
            x0, w_ = x0 // h * h, max(1, w_ // h) * h
        rects.append(_rect(x0, y0, x0 + w_, y0 + h_))
    for k in range(30):  # rectangles inside others, some a hair from the F box edge
        B_ = rects[k]
        bx0, by0, bx1, by1 = int(B_[0, 0]), int(B_[0, 1]), int(B_[2, 0]), int(B_[2, 1])
        if bx1 - bx0 < 4 or by1 - by0 < 4:
            continue
        x0 = int(rng.integers(bx0, (bx0 + bx1) // 2))
        y0 = int(rng.integers(by0, (by0 + by1) // 2))
        x1 = int(rng.integers((bx0 + bx1) // 2 + 1, bx1 + 1))
        y1 = int(rng.integers((by0 + by1) // 2 + 1, by1 + 1))
        rects.append(_rect(x0, y0, x1, y1))
    big = _rect(4 * h, 4 * h, 20 * h, 20 * h)
    rects += [big, _rect(5 * h, 5 * h, 19 * h, 19 * h), _rect(5 * h + 1, 5 * h + 1, 19 * h - 1, 19 * h - 1),
              _rect(5 * h - 1, 6 * h, 10 * h, 10 * h)]
    xy = np.concatenate(rects)
    off = np.arange(0, 4 * len(rects) + 1, 4, dtype=np.int64)
    pr, ps = _all_pairs(len(rects))
    v = oracle.verdicts_ex(xy, off, xy, off, pr, ps, 5, 5, oracle.WITHIN)
    n_hit = 0
    for k, (r, s) in enumerate(zip(pr, ps)):
        R, S = rects[r], rects[s]
        ok = True
        for ax in (0, 1):
            a0, a1 = _cell_range_meets(int(R[0, ax]), int(R[2, ax]), h, G)
            f0, f1 = _cell_range_full(int(S[0, ax]), int(S[2, ax]), h)
            ok &= f0 <= a0 and a1 <= f1
        if ok:
            assert v[k] == 1, (r, s)
            n_hit += 1
        else:
            assert v[k] != 1, (r, s)
    assert n_hit > 0


# ------------------------------------------------------------ host execution
@pytest.fixture(scope="module")
def tiny():
    from tests import _data
    return _data.workload(1, 1.0)


@pytest.mark.parametrize("orders,pred", [((12, 12), 0), ((12, 10), 0), ((10, 12), 0), ((13, 9), 0),
                                         ((12, 12), 1), ((10, 10), 1)])
def test_host_variants_equal_oracle(tiny, orders, pred):
    from paper_2307_01716_gb300 import april as A
    w = tiny
    R = A.april_build_sets(w.R.xy, w.R.off, A.global_grid(orders[0]))
    S = A.april_build_sets(w.S.xy, w.S.off, A.global_grid(orders[1]))
    v, used = A.april_host_filter_ex(R, S, w.pr, w.ps, pred)
    o = oracle.verdicts_ex(w.R.xy, w.R.off, w.S.xy, w.S.off, w.pr, w.ps, orders[0], orders[1], pred)
    assert np.array_equal(v, o)
    assert np.all(used > 0)
    if orders[0] == orders[1] and pred == 0:
        base, used0 = A.april_host_filter(R, S, w.pr, w.ps)
        assert np.array_equal(v, base) and np.array_equal(used, used0)


def test_host_variants_reject_bad_arguments(tiny):
    from paper_2307_01716_gb300 import april as A
    w = tiny
    R = A.april_build_sets(w.R.xy, w.R.off, A.global_grid(12))
    S = A.april_build_sets(w.S.xy, w.S.off, A.global_grid(10))
    with pytest.raises(A.AprilError):
        A.april_host_filter_ex(R, S, w.pr, w.ps, 1)  # within needs equal orders
    with pytest.raises(A.AprilError):
        A.april_host_filter_ex(R, S, w.pr, w.ps, 7)
    v, _ = A.april_host_filter_ex(R, S, np.array([w.R.n], np.uint32), np.array([0], np.uint32), 0)
    assert v[0] == 0xFF
