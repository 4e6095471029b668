"""Pins of the oracle to things other than itself (CPU only).

* Hilbert order: the order-1 visiting order (reading of Sec. 3.2), bijection,
  4-adjacency of consecutive ids, start/end cells, and nesting (the property
  the different-granularity rule of Sec. 5.3 relies on), exhaustive for small
  orders and sampled at N=16.
* Cell classes: the closed form for axis-parallel rectangles; for star
  polygons on small grids, brute force from the paper's coverage definition
  (Sec. 4.1: Full = 100% covered) by exact rational areas, and A = cells that
  meet the polygon by separating axes; hand-built degenerate contacts.
* Verdicts: soundness against exact polygon intersection (a true hit
  intersects, a true negative does not), the cell-matching table of Sec. 4.1,
  special cases, symmetry, and granularity monotonicity.
* Intervals: the worked values printed in the paper (tests/golden).
"""
import json
import os

import numpy as np
import pytest

import oracle
from synth import polygons as SP
from tests import _brute as B

GOLD = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


# ----------------------------------------------------------------- Hilbert
def test_hilbert_order1_visits():
    d = oracle.hilbert(1, [0, 0, 1, 1], [0, 1, 1, 0])
    assert list(d) == [0, 1, 2, 3]


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6, 7, 8])
def test_hilbert_bijection_adjacency_nesting(order):
    G = 1 << order
    yy, xx = np.mgrid[0:G, 0:G]
    d = oracle.hilbert(order, xx.ravel(), yy.ravel())
    assert np.array_equal(np.sort(d), np.arange(G * G, dtype=np.uint64))
    inv = np.empty((G * G, 2), dtype=np.int64)
    inv[d.astype(np.int64)] = np.stack([xx.ravel(), yy.ravel()], 1)
    step = np.abs(np.diff(inv, axis=0)).sum(1)
    assert np.all(step == 1), "consecutive cells must share an edge"
    assert tuple(inv[0]) == (0, 0) and tuple(inv[-1]) == (G - 1, 0)
    if order > 1:
        parent = oracle.hilbert(order - 1, xx.ravel() >> 1, yy.ravel() >> 1)
        assert np.array_equal(d >> np.uint64(2), parent)


def test_hilbert_sampled_order16():
    rng = np.random.default_rng(5)
    x = rng.integers(0, 1 << 16, 4000)
    y = rng.integers(0, 1 << 16, 4000)
    d = oracle.hilbert(16, x, y)
    for k in (1, 3, 8):
        parent = oracle.hilbert(16 - k, x >> k, y >> k)
        assert np.array_equal(d >> np.uint64(2 * k), parent)
    # among the 4 neighbours of an interior cell, d-1 and d+1 appear
    G = 1 << 16
    ok = (x > 0) & (x < G - 1) & (y > 0) & (y < G - 1) & (d > 0) & (d < np.uint64(G * G - 1))
    x, y, d = x[ok], y[ok], d[ok]
    nb = np.stack([oracle.hilbert(16, x + 1, y), oracle.hilbert(16, x - 1, y),
                   oracle.hilbert(16, x, y + 1), oracle.hilbert(16, x, y - 1)], 1)
    assert np.all((nb == (d - np.uint64(1))[:, None]).any(1))
    assert np.all((nb == (d + np.uint64(1))[:, None]).any(1))
    assert oracle.hilbert(16, [G - 1], [0])[0] == np.uint64(G * G - 1)


# -------------------------------------------------------------- intervals
def test_intervalization_worked_examples():
    gold = json.load(open(GOLD))
    for ex in gold["intervalization"]:
        got = oracle.intervalize(np.array(ex["cells"]))
        assert got.tolist() == ex["intervals"], ex["cite"]
    for ex in gold["interval_overlap"]:
        xs = set(range(*ex["x"]))
        ys = set(range(*ex["y"]))
        assert sorted(xs & ys) == ex["common_cells"], ex["cite"]
        # and the half-open lists of those cell sets are the printed intervals
        assert oracle.intervalize(np.array(sorted(xs))).tolist() == [ex["x"]]


# ------------------------------------------------------ cell classification
def _rect(x0, y0, x1, y1):
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], dtype=np.int64)


def _axis_ranges(lo, hi, o, h, G):
    a0 = max(-(-(lo - o) // h) - 1, 0)
    a1 = min((hi - o) // h, G - 1)
    f0 = -(-(lo - o) // h)
    f1 = (hi - o) // h - 1
    return (a0, a1), (max(f0, 0), min(f1, G - 1))


def test_rectangles_closed_form():
    """A closed rectangle meets the closed cell i on an axis iff
    i in [ceil(lo/h)-1, floor(hi/h)]; it contains it iff
    i in [ceil(lo/h), floor(hi/h)-1]; a cell is in A (F) iff both axes are."""
    rng = np.random.default_rng(11)
    for trial in range(300):
        order = int(rng.integers(2, 7))
        g = oracle.Grid(order)
        h, G = g.h, g.G
        if trial % 3 == 0:  # grid-aligned corners
            c = np.sort(rng.integers(0, G + 1, 4).reshape(2, 2), axis=1) * h
        else:
            c = np.sort(rng.integers(0, G * h + 1, 4).reshape(2, 2), axis=1)
        x0, x1 = c[0]
        y0, y1 = c[1]
        if x0 == x1 or y0 == y1:
            continue
        A, F = oracle.cells(_rect(x0, y0, x1, y1), g)
        (ax, fx), (ay, fy) = _axis_ranges(x0, x1, 0, h, G), _axis_ranges(y0, y1, 0, h, G)
        eA = {(i, j) for i in range(ax[0], ax[1] + 1) for j in range(ay[0], ay[1] + 1)}
        eF = {(i, j) for i in range(fx[0], fx[1] + 1) for j in range(fy[0], fy[1] + 1)}
        assert A == eA
        assert F == eF


def _star(rng, G, h, nv_max=12):
    """A small lattice star polygon on a grid of G cells of side h."""
    side = G * h
    c = rng.integers(side // 4, 3 * side // 4, 2)
    R = int(rng.integers(h, max(h + 1, side // 3)))
    nv = int(rng.integers(3, nv_max + 1))
    ang = np.sort(rng.random(nv)) * 2 * np.pi
    rad = R * rng.uniform(0.4, 1.2, nv)
    xy = np.stack([c[0] + rad * np.cos(ang), c[1] + rad * np.sin(ang)], 1)
    # snap some vertices onto grid corners, and some single coordinates onto
    # grid lines, to exercise degenerate contacts
    snap = rng.random(nv) < 0.2
    xy[snap] = np.round(xy[snap] / h) * h
    for axis in (0, 1):
        s1 = rng.random(nv) < 0.2
        xy[s1, axis] = np.round(xy[s1, axis] / h) * h
    xy = np.clip(np.rint(xy), 0, side).astype(np.int64)
    keep = [0]
    for k in range(1, nv):
        if tuple(xy[k]) != tuple(xy[keep[-1]]):
            keep.append(k)
    xy = xy[keep]
    if len(xy) >= 3 and SP.is_simple_star(xy, c):
        return xy, c
    return None


def test_star_polygons_against_coverage_brute_force():
    rng = np.random.default_rng(3)
    done = 0
    while done < 80:
        order = int(rng.integers(3, 6))
        g = oracle.Grid(order)
        got = _star(rng, g.G, g.h)
        if got is None:
            continue
        poly, cen = got
        A, F = oracle.cells(poly, g)
        bA, bF = B.brute_cells(poly.tolist(), tuple(int(v) for v in cen), 0, 0, g.h, g.G)
        assert A == bA, f"A mismatch poly={poly.tolist()} order={order}"
        assert F == bF, f"F mismatch poly={poly.tolist()} order={order}"
        assert F <= A and len(A) > 0
        done += 1


def test_degenerate_contacts():
    g = oracle.Grid(4)
    h = g.h
    # an edge along a grid line: the cells on both sides are in A
    A, F = oracle.cells(_rect(2 * h, 2 * h, 5 * h, 6 * h), g)
    assert (1, 3) in A and (5, 3) in A and (2, 3) in F and (1, 3) not in F
    # a vertex on a grid corner touches all four cells around it
    tri = np.array([[3 * h, 3 * h], [3 * h + h // 2, 5 * h + h // 3], [5 * h + h // 3, 3 * h + h // 2]])
    A, _ = oracle.cells(tri, g)
    assert {(2, 2), (3, 2), (2, 3), (3, 3)} <= A
    # an edge passing through a grid corner touches the diagonal neighbour
    # cell at that single point: the cell is in A but not in F
    tri2 = np.array([[h, h], [3 * h, h], [h, 3 * h]])
    A, F = oracle.cells(tri2, g)
    assert (2, 2) in A and (2, 2) not in F and (1, 1) in F
    bA, bF = B.brute_cells(tri2.tolist(), (4 * h // 3, 4 * h // 3), 0, 0, h, g.G)
    assert (A, F) == (bA, bF)
    # vertex order does not matter (clockwise input)
    assert oracle.cells(tri2[::-1].copy(), g) == (A, F)


def test_reflex_vertex_on_cell_border():
    """A reflex vertex on the bottom border of a cell that the polygon
    otherwise covers: the cell is Full (its open square meets no edge)."""
    g = oracle.Grid(4)
    h = g.h
    notch = np.array([[h, h], [5 * h // 2, 2 * h], [4 * h, h], [4 * h, 4 * h], [h, 4 * h]])
    A, F = oracle.cells(notch, g)
    assert (2, 2) in F
    bA, bF = B.brute_cells(notch.tolist(), (5 * h // 2, 3 * h), 0, 0, h, g.G)
    assert (A, F) == (bA, bF)
    # the same with the vertex on a left border
    notch2 = np.array([[h, h], [4 * h, h], [3 * h, 5 * h // 2], [4 * h, 4 * h], [h, 4 * h]])
    A, F = oracle.cells(notch2, g)
    assert (2, 2) in F and (3, 2) in A and (3, 2) not in F


def _v(P, Q, g):
    xy = np.concatenate([P, Q])
    off = np.array([0, len(P)])
    offs = np.array([0, len(P), len(P) + len(Q)])
    return int(oracle.verdicts(xy, offs, xy, offs, [0], [1], g)[0])


def test_touching_polygons_are_never_true_negatives():
    g = oracle.Grid(4)
    h = g.h
    # two squares sharing an edge on a grid line
    assert _v(_rect(2 * h, 2 * h, 4 * h, 4 * h), _rect(4 * h, 2 * h, 6 * h, 4 * h), g) != 0
    # sharing only a corner on a grid corner
    assert _v(_rect(2 * h, 2 * h, 4 * h, 4 * h), _rect(4 * h, 4 * h, 6 * h, 6 * h), g) != 0
    # sharing only a corner inside a cell
    q = h // 2
    assert _v(_rect(2 * h, 2 * h, 4 * h + q, 4 * h + q), _rect(4 * h + q, 4 * h + q, 6 * h, 6 * h), g) != 0


def test_cell_matching_table():
    """Sec. 4.1 table: Partial x Partial is inconclusive; Full with anything
    non-empty is a sure hit; no common cell is a sure non-result."""
    gold = json.load(open(GOLD))["cell_matching"]
    g = oracle.Grid(4)
    h = g.h
    q = h // 4
    inner = _rect(2 * h + q, 2 * h + q, 3 * h - q, 3 * h - q)  # Partial in cell (2,2) only
    big = _rect(h + 2 * q, h + 2 * q, 4 * h - 2 * q, 4 * h - 2 * q)  # (2,2) Full, neighbours Partial
    corner = _rect(h + 2 * q, h + 2 * q, 2 * h + 2 * q, 2 * h + 2 * q)  # Partial only, ends inside (2,2)
    A, F = oracle.cells(big, g)
    assert (2, 2) in F
    assert _v(inner, corner, g) == 2 and gold["Partial,Partial"] == "inconclusive"
    assert _v(big, inner, g) == 1 and gold["Full,Partial"] == "yes"
    assert _v(inner, big, g) == 1 and gold["Partial,Full"] == "yes"
    assert _v(big, big, g) == 1 and gold["Full,Full"] == "yes"
    assert _v(inner, _rect(10 * h, 10 * h, 12 * h, 12 * h), g) == 0


def _small_sets(seed, n, order):
    rng = np.random.default_rng(seed)
    g = oracle.Grid(order)
    polys = []
    while len(polys) < n:
        got = _star(rng, g.G, g.h, nv_max=10)
        if got is not None:
            polys.append(got[0])
    xy = np.concatenate(polys)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(p) for p in polys])
    return polys, xy, off, g


def test_verdicts_sound_against_exact_geometry():
    polys, xy, off, g = _small_sets(7, 40, 5)
    pr, ps = np.meshgrid(np.arange(40), np.arange(40), indexing="ij")
    pr = pr.ravel().astype(np.uint32)
    ps = ps.ravel().astype(np.uint32)
    v = oracle.verdicts(xy, off, xy, off, pr, ps, g)
    counts = np.bincount(v, minlength=3)
    assert counts[0] > 0 and counts[1] > 0 and counts[2] > 0
    for k in range(len(pr)):
        inter = B.polygons_intersect(polys[pr[k]].tolist(), polys[ps[k]].tolist())
        if v[k] == 1:
            assert inter, (pr[k], ps[k])
        if v[k] == 0:
            assert not inter, (pr[k], ps[k])


def test_verdict_special_cases_and_symmetry():
    polys, xy, off, g = _small_sets(9, 30, 5)
    n = len(polys)
    idx = np.arange(n, dtype=np.uint32)
    self_v = oracle.verdicts(xy, off, xy, off, idx, idx, g)
    for k in range(n):
        _, F = oracle.cells(polys[k], g)
        assert self_v[k] == (1 if F else 2)
    pr, ps = np.meshgrid(idx, idx, indexing="ij")
    v = oracle.verdicts(xy, off, xy, off, pr.ravel(), ps.ravel(), g).reshape(n, n)
    assert np.array_equal(v, v.T)


def test_granularity_monotonicity():
    """Going from order N to N+1 over the same space never turns a decisive
    verdict into another verdict (children of A cells cover A, children of F
    cells are F)."""
    polys, xy, off, _ = _small_sets(13, 30, 4)
    n = len(polys)
    idx = np.arange(n, dtype=np.uint32)
    pr, ps = np.meshgrid(idx, idx, indexing="ij")
    prev = None
    for order in range(4, 9):
        v = oracle.verdicts(xy, off, xy, off, pr.ravel(), ps.ravel(), oracle.Grid(order))
        if prev is not None:
            dec = prev != 2
            assert np.array_equal(v[dec], prev[dec])
        prev = v


def test_cell_lists_cover_cell_sets():
    polys, _, _, g = _small_sets(21, 20, 6)
    for p in polys:
        A, F = oracle.cells(p, g)
        La, Lf = oracle.cell_lists(p, g)
        for L, S in ((La, A), (Lf, F)):
            assert int(sum(int(e) - int(s) for s, e in L)) == len(S)
            if len(L) > 1:
                assert np.all(L[1:, 0] > L[:-1, 1]), "lists must be maximal and disjoint"
            ids = set(int(d) for s, e in L for d in range(int(s), int(e)))
            want = set(int(d) for d in oracle.hilbert(g.order, [c[0] for c in S], [c[1] for c in S])) if S else set()
            assert ids == want


def test_partition_areas_cover_members():
    from synth import configs
    w = configs.make(4, scale=0.005)
    grids = oracle.partition_areas(w.R.mbr, w.S.mbr, 16, 14)
    for mbr in (w.R.mbr, w.S.mbr):
        for m, pids in zip(mbr, oracle.partitions_met(mbr, 16)):
            for p in pids:
                g = grids[p]
                side = g.h * g.G
                assert g.ox <= m[0] and g.oy <= m[1] and m[2] <= g.ox + side and m[3] <= g.oy + side
                assert g.ox % g.h == 0 and g.oy % g.h == 0 and g.h >= 2
    part = oracle.route_pairs(w.R.mbr, w.S.mbr, w.pr, w.ps, 16)
    # the routed partition is met by both objects
    met_r = oracle.partitions_met(w.R.mbr, 16)
    met_s = oracle.partitions_met(w.S.mbr, 16)
    for k in range(len(w.pr)):
        assert part[k] in met_r[w.pr[k]] and part[k] in met_s[w.ps[k]]


def _smallest_area_brute(lo, hi, order):
    """Reading C11 enumerated: the smallest power-of-two side 2^k (cell side
    2^k >> order of at least 2) such that SOME origin that is a multiple of
    the cell side, at or below the MBR's lower corner, covers the closed MBR;
    among the origins that work at that side, the largest (the snap of the
    lower corner down to the cell lattice)."""
    for k in range(order + 1, 26):
        size = 1 << k
        h = size >> order
        ok = []
        for ox in range(0, lo[0] + 1, h):
            for oy in range(0, lo[1] + 1, h):
                if ox + size >= hi[0] and oy + size >= hi[1]:
                    ok.append((ox, oy))
        if ok:
            return size, max(o[0] for o in ok), max(o[1] for o in ok)
    raise AssertionError("no area")


@pytest.mark.parametrize("lo,hi,order,size,origin", [
    # a 4x4 grid (order 2): cell side 2 at side 8
    ((0, 0), (8, 8), 2, 8, (0, 0)),      # exactly 2^3 lattice units: side 8
    ((0, 0), (9, 8), 2, 16, (0, 0)),     # one unit wider: must step to 2^4
    ((5, 5), (12, 12), 2, 8, (4, 4)),    # origin snaps down to the cell lattice (4), 4 + 8 reaches 12
    ((5, 5), (13, 12), 2, 16, (4, 4)),   # 4 + 8 misses 13: side 16 with cell side 4, origin 4
    ((7, 3), (14, 10), 2, 8, (6, 2)),    # snaps to (6, 2) at cell side 2; 6 + 8 and 2 + 8 just reach
    ((7, 3), (15, 10), 2, 16, (4, 0)),   # one unit wider: side 16, cell side 4, origin (4, 0)
    ((100, 36), (224, 160), 3, 128, (96, 32)),  # order 3: cell side 16 at side 128
    ((100, 36), (225, 160), 3, 256, (96, 32)),  # one unit wider in x: side 256, cell side 32
])
def test_partition_areas_minimal_square(lo, hi, order, size, origin):
    """partition_areas picks the smallest admissible square (reading C11),
    pinned by hand-computed cases and by brute force over all origins."""
    mbr_r = np.array([[lo[0], lo[1], hi[0], hi[1]]], dtype=np.int64)
    mbr_s = np.array([[lo[0], lo[1], lo[0], lo[1]]], dtype=np.int64)  # a point inside: does not grow the MBR
    g = oracle.partition_areas(mbr_r, mbr_s, 1, order)[0]
    assert (g.h * g.G, g.ox, g.oy) == (size, origin[0], origin[1])
    assert (size, origin[0], origin[1]) == _smallest_area_brute(lo, hi, order)


def test_partition_areas_minimal_square_random():
    """Brute force on random small MBRs of two objects (one partition)."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        order = int(rng.integers(1, 4))
        a = rng.integers(0, 300, 4)
        b = rng.integers(0, 300, 4)
        ma = [min(a[0], a[2]), min(a[1], a[3]), max(a[0], a[2]), max(a[1], a[3])]
        mb = [min(b[0], b[2]), min(b[1], b[3]), max(b[0], b[2]), max(b[1], b[3])]
        g = oracle.partition_areas(np.array([ma]), np.array([mb]), 1, order)[0]
        lo = (min(ma[0], mb[0]), min(ma[1], mb[1]))
        hi = (max(ma[2], mb[2]), max(ma[3], mb[3]))
        assert (g.h * g.G, g.ox, g.oy) == _smallest_area_brute(lo, hi, order)
