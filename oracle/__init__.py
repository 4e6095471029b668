"""APRIL oracle -- TEST INFRASTRUCTURE ONLY.

Plain CPU statement of the APRIL intermediate filter (paper Sec. 4.1, Table
"APRIL: do two objects intersect in a common cell?", Algorithm 2), used by the
test suite, the smoke check and the benchmark's CPU-baseline leg to check the
CUDA path.  The product path must never import this package.

* `april_oracle.c` classifies cells and computes per-pair verdicts by cell-set
  intersection (no curve, no intervals), plus the Hilbert index.
* This module wraps it with ctypes and adds:
  - `cell_lists`: a polygon's A- and F-cell sets written as maximal
    Hilbert-order intervals (Sec. 3.2 intervalization: sort the cell ids and
    merge consecutive ids), used to compare a builder's lists list-for-list;
  - `partition_areas` / `route_pairs`: the partition raster areas and the
    partition each pair is evaluated in (Sec. 5.2), per the readings stated
    in the functions.

Parity status: cell classes, verdicts, Hilbert order, intervalization and the
partition raster areas are pinned by tests (closed forms, brute force,
invariants, hand-computed minimal squares).  The figure-based
worked examples of Sec. 3.2 and Sec. 6.2 are parity unpinned: their polygons
exist only in figures that are missing from the paper's text.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "april_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
_lib_lock = threading.Lock()

LATTICE_BITS = 24

CLS_A = 1
CLS_F = 2

TRUE_NEGATIVE = 0
TRUE_HIT = 1
INCONCLUSIVE = 2


def build(force: bool = False) -> str:
    """Compile the oracle's C source into liboracle.so (plain gcc -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        return _load()


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        p64 = ctypes.POINTER(ctypes.c_int64)
        L.oracle_window.restype = ctypes.c_int64
        L.oracle_window.argtypes = [p64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int64, p64]
        L.oracle_classify.restype = ctypes.c_int
        L.oracle_classify.argtypes = [p64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_int64, p64, ctypes.c_void_p]
        L.oracle_verdicts.restype = ctypes.c_int
        L.oracle_verdicts.argtypes = [p64, p64, p64, p64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_void_p]
        L.oracle_verdicts_ex.restype = ctypes.c_int
        L.oracle_verdicts_ex.argtypes = [p64, p64, p64, p64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
        L.oracle_hilbert_d.restype = ctypes.c_uint64
        L.oracle_hilbert_d.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_hilbert_many.restype = None
        L.oracle_hilbert_many.argtypes = [ctypes.c_int, p64, p64, ctypes.c_int64, ctypes.c_void_p]
        _lib = L
    return _lib


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


class Grid:
    """A 2^order x 2^order grid of square cells of side h lattice units whose
    lower-left corner is (ox, oy).  The global grid of order N over the unit
    square has ox = oy = 0 and h = 2^(24-N)."""

    def __init__(self, order: int, ox: int = 0, oy: int = 0, h: int | None = None):
        self.order = order
        self.G = 1 << order
        self.ox = int(ox)
        self.oy = int(oy)
        self.h = int(h if h is not None else 1 << (LATTICE_BITS - order))
        if self.h < 2 or self.h % 2:
            raise ValueError("cell side must be an even number of lattice units")

    def args(self):
        return self.ox, self.oy, self.h, self.G


def raster(poly: np.ndarray, grid: Grid):
    """Classify the cells of one polygon.

    Returns (win, cls): win = (i0, j0, i1, j1) is the inclusive cell window of
    the polygon's MBR, cls is a (j1-j0+1, i1-i0+1) uint8 array of CLS_A|CLS_F
    bits (row j, column i)."""
    xy = np.ascontiguousarray(poly, dtype=np.int64).reshape(-1)
    nv = len(xy) // 2
    win = np.zeros(4, dtype=np.int64)
    n = lib().oracle_window(_p64(xy), nv, *grid.args(), _p64(win))
    if n <= 0:
        return win, np.zeros((0, 0), dtype=np.uint8)
    cls = np.zeros(int(n), dtype=np.uint8)
    rc = lib().oracle_classify(_p64(xy), nv, *grid.args(), _p64(win), cls.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_classify failed ({rc})")
    return win, cls.reshape(int(win[3] - win[1] + 1), int(win[2] - win[0] + 1))


def cells(poly: np.ndarray, grid: Grid):
    """(A, F) as sets of (i, j) cell coordinates."""
    win, cls = raster(poly, grid)
    jj, ii = np.nonzero(cls & CLS_A)
    A = {(int(i + win[0]), int(j + win[1])) for i, j in zip(ii, jj)}
    jj, ii = np.nonzero(cls & CLS_F)
    F = {(int(i + win[0]), int(j + win[1])) for i, j in zip(ii, jj)}
    return A, F


def _serial_verdicts(rxy, roff, sxy, soff, pr, ps, grid: Grid) -> np.ndarray:
    out = np.zeros(len(pr), dtype=np.uint8)
    rc = lib().oracle_verdicts(_p64(rxy), _p64(roff), _p64(sxy), _p64(soff), pr.ctypes.data, ps.ctypes.data,
                               len(pr), *grid.args(), out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_verdicts failed ({rc})")
    return out


def _in_chunks(fn, pr, ps, threads: int, min_chunk: int = 16) -> np.ndarray:
    """fn over contiguous chunks of the pairs on `threads` host threads (the
    C calls release the GIL); every pair is still computed on its own by the
    same plain code, so the result does not depend on the chunking."""
    n = len(pr)
    if threads <= 1 or n <= min_chunk:
        return fn(pr, ps)
    from concurrent.futures import ThreadPoolExecutor
    bounds = np.linspace(0, n, min(4 * threads, n // min_chunk) + 1).astype(np.int64)
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda ab: fn(pr[ab[0]:ab[1]], ps[ab[0]:ab[1]]), zip(bounds[:-1], bounds[1:])))
    return np.concatenate(parts)


def verdicts(R_xy, R_off, S_xy, S_off, pr, ps, grid: Grid, threads: int = 1) -> np.ndarray:
    """Per-pair verdicts (0 true negative, 1 true hit, 2 inconclusive);
    `threads` > 1 evaluates contiguous chunks of the pairs concurrently."""
    rxy = np.ascontiguousarray(R_xy, dtype=np.int64).reshape(-1)
    sxy = np.ascontiguousarray(S_xy, dtype=np.int64).reshape(-1)
    roff = np.ascontiguousarray(R_off, dtype=np.int64)
    soff = np.ascontiguousarray(S_off, dtype=np.int64)
    pr = np.ascontiguousarray(pr, dtype=np.uint32)
    ps = np.ascontiguousarray(ps, dtype=np.uint32)
    return _in_chunks(lambda a, b: _serial_verdicts(rxy, roff, sxy, soff, a, b, grid), pr, ps, threads)


INTERSECTS = 0
WITHIN = 1


def verdicts_ex(R_xy, R_off, S_xy, S_off, pr, ps, order_r: int, order_s: int, pred: int = INTERSECTS) -> np.ndarray:
    """Verdicts of the filter variants on global grids of orders order_r and
    order_s (Sec. 5.3 when they differ) for the intersects predicate, or of
    the within-join filter (Sec. 4.3.2; equal orders)."""
    rxy = np.ascontiguousarray(R_xy, dtype=np.int64).reshape(-1)
    sxy = np.ascontiguousarray(S_xy, dtype=np.int64).reshape(-1)
    roff = np.ascontiguousarray(R_off, dtype=np.int64)
    soff = np.ascontiguousarray(S_off, dtype=np.int64)
    pr = np.ascontiguousarray(pr, dtype=np.uint32)
    ps = np.ascontiguousarray(ps, dtype=np.uint32)
    out = np.zeros(len(pr), dtype=np.uint8)
    gr, gs = Grid(order_r), Grid(order_s)
    rc = lib().oracle_verdicts_ex(_p64(rxy), _p64(roff), _p64(sxy), _p64(soff), pr.ctypes.data, ps.ctypes.data,
                                  len(pr), 0, 0, gr.h, gr.G, gs.h, gs.G, pred, out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_verdicts_ex failed ({rc})")
    return out


def select_candidates(mbr_r, mbr_q):
    """The MBR step of a selection query (Sec. 4.3.1): every pair (r, q) whose
    closed MBRs meet, by a direct test of each query against every data MBR.
    Returns (r, q) sorted by q, then r."""
    mbr_r = np.asarray(mbr_r, dtype=np.int64)
    out_r, out_q = [], []
    for q, (x0, y0, x1, y1) in enumerate(np.asarray(mbr_q, dtype=np.int64)):
        hit = np.flatnonzero((mbr_r[:, 0] <= x1) & (x0 <= mbr_r[:, 2]) & (mbr_r[:, 1] <= y1) & (y0 <= mbr_r[:, 3]))
        out_r.append(hit)
        out_q.append(np.full(len(hit), q))
    if not out_r:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    return np.concatenate(out_r).astype(np.uint32), np.concatenate(out_q).astype(np.uint32)


def hilbert(order: int, x, y) -> np.ndarray:
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.int64)
    y = np.ascontiguousarray(np.atleast_1d(y), dtype=np.int64)
    d = np.zeros(len(x), dtype=np.uint64)
    lib().oracle_hilbert_many(order, _p64(x), _p64(y), len(x), d.ctypes.data)
    return d


def intervalize(ids: np.ndarray) -> np.ndarray:
    """Sorted cell ids -> maximal half-open intervals [st, end) (Sec. 3.2:
    sort the ids and merge consecutive ids).  Returns (n, 2) uint64."""
    ids = np.sort(np.asarray(ids, dtype=np.uint64))
    if len(ids) == 0:
        return np.zeros((0, 2), dtype=np.uint64)
    brk = np.nonzero(np.diff(ids) != 1)[0]
    starts = np.concatenate([[ids[0]], ids[brk + 1]])
    ends = np.concatenate([ids[brk] + 1, [ids[-1] + 1]])
    return np.stack([starts, ends], 1)


def cell_lists(poly: np.ndarray, grid: Grid):
    """A- and F-lists of one polygon as (n, 2) uint64 arrays of [st, end)
    Hilbert intervals on `grid` (end may equal 4^order)."""
    win, cls = raster(poly, grid)
    out = []
    for bit in (CLS_A, CLS_F):
        jj, ii = np.nonzero(cls & bit)
        d = hilbert(grid.order, ii + win[0], jj + win[1])
        out.append(intervalize(d))
    return out[0], out[1]


# ---------------------------------------------------------------------------
# Partitioning (Sec. 5.2).
#
# Reading of the paper: the data space is split into p x p equal disjoint
# partitions; every object is approximated once for every partition its MBR
# meets, on that partition's own grid of order n_part; the "raster area" of a
# partition is the smallest square whose side is a power of two (in lattice
# units) and whose corner is a multiple of its cell side, that covers the MBR
# of all objects (of both inputs) whose MBRs meet the partition; a candidate
# pair is evaluated only in the partition that holds the lower-left corner of
# MBR(r) n MBR(s).
# ---------------------------------------------------------------------------

def partition_of_point(x, y, parts: int):
    side = (1 << LATTICE_BITS) // parts
    px = np.minimum(np.asarray(x) // side, parts - 1)
    py = np.minimum(np.asarray(y) // side, parts - 1)
    return py * parts + px


def partitions_met(mbr: np.ndarray, parts: int):
    """List of partition ids whose closed square meets each closed MBR."""
    side = (1 << LATTICE_BITS) // parts
    out = []
    for x0, y0, x1, y1 in np.asarray(mbr, dtype=np.int64):
        # closed partition [k*side, (k+1)*side] meets [x0, x1]
        kx0 = max(-(-x0 // side) - 1, 0)
        kx1 = min(x1 // side, parts - 1)
        ky0 = max(-(-y0 // side) - 1, 0)
        ky1 = min(y1 // side, parts - 1)
        out.append([ky * parts + kx for ky in range(ky0, ky1 + 1) for kx in range(kx0, kx1 + 1)])
    return out


def partition_areas(mbr_r: np.ndarray, mbr_s: np.ndarray, parts: int, order: int):
    """Grid of every partition: a dict pid -> Grid (order `order`)."""
    side = (1 << LATTICE_BITS) // parts
    lo = {}
    hi = {}
    for mbr in (mbr_r, mbr_s):
        for m, pids in zip(np.asarray(mbr, dtype=np.int64), partitions_met(mbr, parts)):
            for p in pids:
                if p in lo:
                    lo[p] = (min(lo[p][0], m[0]), min(lo[p][1], m[1]))
                    hi[p] = (max(hi[p][0], m[2]), max(hi[p][1], m[3]))
                else:
                    lo[p] = (m[0], m[1])
                    hi[p] = (m[2], m[3])
    grids = {}
    for p in lo:
        k = order + 1  # smallest side 2^k with a cell side of at least 2
        while True:
            size = 1 << k
            h = size >> order
            ox = (lo[p][0] // h) * h
            oy = (lo[p][1] // h) * h
            if ox + size >= hi[p][0] and oy + size >= hi[p][1]:
                break
            k += 1
        grids[p] = Grid(order, ox, oy, h)
    return grids


def route_pairs(mbr_r: np.ndarray, mbr_s: np.ndarray, pr, ps, parts: int) -> np.ndarray:
    """Partition each pair is evaluated in: the one holding the lower-left
    corner of MBR(r) n MBR(s)."""
    mr = np.asarray(mbr_r, dtype=np.int64)[np.asarray(pr, dtype=np.int64)]
    ms = np.asarray(mbr_s, dtype=np.int64)[np.asarray(ps, dtype=np.int64)]
    return partition_of_point(np.maximum(mr[:, 0], ms[:, 0]), np.maximum(mr[:, 1], ms[:, 1]), parts)


def partitioned_verdicts(R_xy, R_off, mbr_r, S_xy, S_off, mbr_s, pr, ps, parts: int, order: int,
                         threads: int = 1):
    """Verdicts of the partitioned filter: each pair on its routed partition's grid."""
    grids = partition_areas(mbr_r, mbr_s, parts, order)
    part = route_pairs(mbr_r, mbr_s, pr, ps, parts)
    out = np.zeros(len(pr), dtype=np.uint8)
    pr = np.asarray(pr)
    ps = np.asarray(ps)
    for p in np.unique(part):
        sel = np.nonzero(part == p)[0]
        out[sel] = verdicts(R_xy, R_off, S_xy, S_off, pr[sel], ps[sel], grids[int(p)], threads)
    return out
