"""Curve independence (the verdicts are a property of the cell sets, Sec. 4.1;
the curve only orders them, Sec. 3.2): the oracle's A- and F-cell sets of
every polygon, written as maximal intervals under the Hilbert order, the
Z-order (bit interleaving) and row-major order, imported with
april_sets_from_lists, give the same verdicts under Algorithm 2, equal to the
oracle's curve-free verdicts.  The Hilbert import also equals the builder's
lists.  Plus the import's argument checks."""
import functools

import numpy as np
import pytest

import oracle
from tests import _data
from paper_2307_01716_gb300 import april as A


def _morton(order, x, y):
    d = np.zeros(len(x), dtype=np.uint64)
    for b in range(order):
        d |= ((x >> b) & 1).astype(np.uint64) << np.uint64(2 * b)
        d |= ((y >> b) & 1).astype(np.uint64) << np.uint64(2 * b + 1)
    return d


CURVES = {
    "hilbert": lambda order, x, y: oracle.hilbert(order, x, y).astype(np.uint64),
    "zorder": _morton,
    "rowmajor": lambda order, x, y: (y.astype(np.uint64) << np.uint64(order)) | x.astype(np.uint64),
}


def _lists(cellset, order, curve):
    if not cellset:
        return np.zeros((0, 2), np.uint64)
    c = np.array(sorted(cellset), dtype=np.int64)
    return oracle.intervalize(np.sort(CURVES[curve](order, c[:, 0], c[:, 1])))


@functools.lru_cache(maxsize=None)
def _cells(side: str):
    w = _data.workload(1, 1.0)
    P = w.R if side == "R" else w.S
    g = oracle.Grid(w.order)
    return [oracle.cells(P.poly(i), g) for i in range(P.n)]


@functools.lru_cache(maxsize=None)
def imported(curve: str):
    w = _data.workload(1, 1.0)
    out = []
    for side in ("R", "S"):
        cs = _cells(side)
        out.append(A.april_sets_from_lists(w.order, [_lists(a, w.order, curve) for a, _ in cs],
                                           [_lists(f, w.order, curve) for _, f in cs]))
    return tuple(out)


def test_hilbert_import_equals_builder():
    w = _data.workload(1, 1.0)
    R, _ = imported("hilbert")
    B = A.april_build_sets(w.R.xy, w.R.off, A.global_grid(w.order))
    for i in range(0, w.R.n, 7):
        for which in (0, 1):
            assert np.array_equal(R.list(i, which), B.list(i, which)), (i, which)


def test_verdicts_do_not_depend_on_the_curve():
    w = _data.workload(1, 1.0)
    want = _data.oracle_verdicts(1, 1.0)
    for curve in CURVES:
        R, S = imported(curve)
        v, _ = A.april_host_filter(R, S, w.pr, w.ps)
        assert np.array_equal(v, want), curve


def test_import_rejects_bad_lists():
    ok = [np.array([[1, 3], [5, 6]], np.uint64)]
    A.april_sets_from_lists(4, ok, ok)
    for bad in ([[3, 3]], [[1, 4], [3, 6]], [[5, 6], [1, 2]], [[0, 1 << 8 | 1]]):
        with pytest.raises(A.AprilError):
            A.april_sets_from_lists(4, [np.array(bad, np.uint64)], ok)
    with pytest.raises(A.AprilError):
        A.april_sets_from_lists(17, ok, ok)
    with pytest.raises(A.AprilError):  # an F interval outside the A intervals
        A.april_sets_from_lists(4, ok, [np.array([[2, 4]], np.uint64)])
    A.april_sets_from_lists(4, ok, [np.array([[1, 2], [5, 6]], np.uint64)])
    # an end of 2^32 at order 16 is written as 0 and accepted
    top = [np.array([[0xFFFFFFF0, 1 << 32]], np.uint64)]
    S = A.april_sets_from_lists(16, top, top)
    assert S.list(0, 0).tolist() == [[0xFFFFFFF0, 0]]
