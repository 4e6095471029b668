"""Seeded synthetic star-polygon generator on the integer lattice.

This module only draws inputs.  It holds none of the APRIL method's
arithmetic (no cell classification, no curve, no interval logic): it produces
simple polygons whose vertices are integer lattice points, plus their MBRs.

Coordinate model.  The data space is the unit square [0,1]^2, represented by
the integer lattice {0, ..., 2^24}^2 (one data unit = 2^24 lattice units).  A
2^N x 2^N grid over the data space has cells of 2^(24-N) lattice units, so for
every N <= 16 the cell corners and centres are lattice points and all
geometric predicates used downstream are exact in int64 arithmetic.

Polygon recipe (star-shaped, after the workloads of Sec. 7 of the paper, whose
real datasets are not available here): a centre c, a mean radius R, k vertex
angles sorted uniformly in [0, 2pi), and per-vertex radius R * U[0.6, 1.4].
Vertices that would leave [0,1]^2 are pulled radially towards c.  After
rounding to the lattice, consecutive duplicates are dropped and any vertex that
breaks the strict counter-clockwise angular order around the (rounded) centre
is dropped, so each output polygon is simple and strictly star-shaped around
its centre (a polygon whose consecutive vertex angles strictly increase by
less than pi and wind once around the centre cannot self-intersect).
"""
from __future__ import annotations

import numpy as np

LATTICE_BITS = 24
LATTICE = 1 << LATTICE_BITS  # lattice units per data-space unit


def _segment_ids(counts: np.ndarray) -> np.ndarray:
    return np.repeat(np.arange(len(counts), dtype=np.int64), counts)


def _cyclic_prev(off: np.ndarray) -> np.ndarray:
    """Index of the cyclic predecessor of every element of a segmented array."""
    n = int(off[-1])
    idx = np.arange(n, dtype=np.int64) - 1
    starts = off[:-1]
    ends = off[1:]
    nonempty = ends > starts
    idx[starts[nonempty]] = ends[nonempty] - 1
    return idx


def _compact(xy: np.ndarray, off: np.ndarray, keep: np.ndarray):
    counts = np.add.reduceat(keep.astype(np.int64), off[:-1]) if len(off) > 1 else np.zeros(0, np.int64)
    # reduceat on empty segments returns the element at the start; all our
    # segments are non-empty when this is called.
    new_off = np.zeros(len(off), dtype=np.int64)
    np.cumsum(counts, out=new_off[1:])
    return xy[keep], new_off


def _bad_mask(xy, off, cen):
    seg = _segment_ids(np.diff(off))
    prev = _cyclic_prev(off)
    c = cen[seg]
    ax = xy[prev, 0] - c[:, 0]
    ay = xy[prev, 1] - c[:, 1]
    bx = xy[:, 0] - c[:, 0]
    by = xy[:, 1] - c[:, 1]
    bad = (ax * by - ay * bx) <= 0
    bad |= (bx == 0) & (by == 0)          # a vertex on the centre is invalid too
    bad &= np.diff(off)[seg] > 3          # the winding check handles tiny ones
    # drop at most every other offender in a run, so that both ends of a
    # valid edge are never removed together
    drop = bad.copy()
    drop[1:] &= ~bad[:-1] | (seg[1:] != seg[:-1])
    return drop, seg


def _cleanup(xy: np.ndarray, off: np.ndarray, cen: np.ndarray):
    """Drop duplicates and angular-order violations (vectorised over polygons).

    One pass over all polygons, then repeated passes over only the polygons
    that still changed: a polygon's mask depends on its own vertices alone,
    so one that had nothing to drop in a pass keeps its vertices for good.
    """
    drop, seg = _bad_mask(xy, off, cen)
    if not drop.any():
        return xy, off
    touched = np.unique(seg[drop])
    xy, off = _compact(xy, off, ~drop)
    # iterate on the affected polygons only, retiring each once it is stable
    counts = np.diff(off)
    sub_cnt = counts[touched]
    sub_off = np.zeros(len(touched) + 1, dtype=np.int64)
    np.cumsum(sub_cnt, out=sub_off[1:])
    gather = np.repeat(off[touched] - sub_off[:-1], sub_cnt) + np.arange(int(sub_off[-1]))
    sub_xy = xy[gather]
    sub_cen = cen[touched]
    ids = touched
    done_ids, done_cnt, done_xy = [], [], []
    for _ in range(256):
        d, s = _bad_mask(sub_xy, sub_off, sub_cen)
        if not d.any():
            break
        changing = np.zeros(len(ids), dtype=bool)
        changing[np.unique(s[d])] = True
        keep_v = changing[s]
        cnt = np.diff(sub_off)
        if not changing.all():
            done_ids.append(ids[~changing])
            done_cnt.append(cnt[~changing])
            done_xy.append(sub_xy[~keep_v])
        ch_off = np.zeros(int(changing.sum()) + 1, dtype=np.int64)
        np.cumsum(cnt[changing], out=ch_off[1:])
        sub_xy, sub_off = _compact(sub_xy[keep_v], ch_off, ~d[keep_v])
        ids = ids[changing]
        sub_cen = sub_cen[changing]
    done_ids.append(ids)
    done_cnt.append(np.diff(sub_off))
    done_xy.append(sub_xy)
    all_ids = np.concatenate(done_ids)
    all_cnt = np.concatenate(done_cnt)
    all_xy = np.concatenate(done_xy)
    # the retired polygons back in id order
    order = np.argsort(all_ids, kind="stable")
    src_off = np.zeros(len(all_cnt) + 1, dtype=np.int64)
    np.cumsum(all_cnt, out=src_off[1:])
    dst_cnt = all_cnt[order]
    dst_off = np.zeros(len(dst_cnt) + 1, dtype=np.int64)
    np.cumsum(dst_cnt, out=dst_off[1:])
    sub_xy = all_xy[np.repeat(src_off[:-1][order] - dst_off[:-1], dst_cnt) + np.arange(int(dst_off[-1]))]
    counts[all_ids[order]] = dst_cnt
    new_off = np.zeros(len(off), dtype=np.int64)
    np.cumsum(counts, out=new_off[1:])
    new_xy = np.empty((int(new_off[-1]), 2), dtype=np.int64)
    keep_seg = np.ones(len(counts), dtype=bool)
    keep_seg[touched] = False
    src_seg = _segment_ids(np.diff(off))
    dst_seg = _segment_ids(counts)
    new_xy[keep_seg[dst_seg]] = xy[keep_seg[src_seg]]
    new_xy[~keep_seg[dst_seg]] = sub_xy
    return new_xy, new_off


def _winding_ok(xy: np.ndarray, off: np.ndarray, cen: np.ndarray) -> np.ndarray:
    counts = np.diff(off)
    seg = _segment_ids(counts)
    prev = _cyclic_prev(off)
    c = cen[seg]
    ax = xy[prev, 0] - c[:, 0]
    ay = xy[prev, 1] - c[:, 1]
    bx = xy[:, 0] - c[:, 0]
    by = xy[:, 1] - c[:, 1]
    cross = ax * by - ay * bx
    pos = np.ones(len(counts), dtype=bool)
    if len(xy):
        allpos = np.minimum.reduceat((cross > 0).astype(np.int8), off[:-1]).astype(bool)
        pos &= allpos
    # Counter-clockwise crossings of the ray {c + t*(1,0), t>0}: the edge goes
    # from below the ray's line to on/above it with positive cross product.
    crossing = ((ay < 0) & (by >= 0) & (cross > 0)).astype(np.int64)
    wind = np.add.reduceat(crossing, off[:-1]) if len(xy) else np.zeros(0, np.int64)
    return pos & (wind == 1) & (counts >= 3)


def _square(c: np.ndarray, half: np.ndarray) -> np.ndarray:
    x0 = np.maximum(c[:, 0] - half, 0)
    y0 = np.maximum(c[:, 1] - half, 0)
    x1 = np.minimum(c[:, 0] + half, LATTICE)
    y1 = np.minimum(c[:, 1] + half, LATTICE)
    sq = np.stack([np.stack([x0, y0], 1), np.stack([x1, y0], 1),
                   np.stack([x1, y1], 1), np.stack([x0, y1], 1)], 1)
    return sq


def star_polygons(rng: np.random.Generator, centers: np.ndarray, radii: np.ndarray,
                  nverts: np.ndarray, jitter=(0.6, 1.4)):
    """Build lattice star polygons.

    centers: (n,2) float in [0,1]; radii: (n,) float (data units);
    nverts: (n,) int >= 3.  Returns (xy int64 (V,2), off int64 (n+1,)).
    """
    n = len(centers)
    centers = np.clip(centers, 1e-6, 1 - 1e-6)
    nverts = np.asarray(nverts, dtype=np.int64)
    # Cap the vertex count so neighbouring vertices stay a few lattice units
    # apart (rounding would otherwise collapse them).
    cap = np.maximum(8, (2 * np.pi * radii * LATTICE / 16.0).astype(np.int64))
    nverts = np.clip(np.minimum(nverts, cap), 3, None)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(nverts, out=off[1:])
    seg = _segment_ids(nverts)
    total = int(off[-1])
    # Sorted uniform angles per polygon without a sort: the normalised
    # partial sums of k+1 i.i.d. exponentials are the order statistics of k
    # uniforms.  Each polygon draws k+1 values; the last closes the circle.
    e = rng.exponential(size=total + n)
    eoff = off + np.arange(n + 1)
    cs = np.cumsum(e)
    seg_e = _segment_ids(nverts + 1)
    base = np.concatenate([[0.0], cs[eoff[1:-1] - 1]]) if n else np.zeros(0)
    tot = cs[eoff[1:] - 1] - base
    last = np.zeros(total + n, dtype=bool)
    last[eoff[1:] - 1] = True
    part = (cs - base[seg_e]) / tot[seg_e]
    ang = (part[~last] * (2 * np.pi))
    ang = (ang + rng.random(n)[seg] * 2 * np.pi) % (2 * np.pi)
    rad = radii[seg] * rng.uniform(jitter[0], jitter[1], size=total)
    c = centers[seg]
    dx = np.cos(ang) * rad
    dy = np.sin(ang) * rad
    # pull towards the centre so that c + t*(dx,dy) stays inside [0,1]^2
    t = np.ones(total)
    with np.errstate(divide="ignore", invalid="ignore"):
        for d, cc in ((dx, c[:, 0]), (dy, c[:, 1])):
            lim_hi = np.where(d > 0, (1.0 - cc) / d, np.inf)
            lim_lo = np.where(d < 0, (0.0 - cc) / d, np.inf)
            t = np.minimum(t, np.minimum(lim_hi, lim_lo))
    px = c[:, 0] + t * dx
    py = c[:, 1] + t * dy
    xy = np.stack([np.rint(px * LATTICE), np.rint(py * LATTICE)], 1).astype(np.int64)
    np.clip(xy, 0, LATTICE, out=xy)
    cen = np.rint(centers * LATTICE).astype(np.int64)
    xy, off = _cleanup(xy, off, cen)
    ok = _winding_ok(xy, off, cen)
    if not ok.all():
        # Replace degenerate polygons by an axis-aligned square around the centre.
        bad = np.nonzero(~ok)[0]
        half = np.maximum(8, (radii[bad] * LATTICE * 0.5).astype(np.int64))
        sq = _square(cen[bad], half)
        counts = np.diff(off)
        counts[bad] = 4
        new_off = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(counts, out=new_off[1:])
        new_xy = np.empty((int(new_off[-1]), 2), dtype=np.int64)
        keep_seg = np.ones(n, dtype=bool)
        keep_seg[bad] = False
        src_seg = _segment_ids(np.diff(off))
        src_keep = keep_seg[src_seg]
        dst_seg = _segment_ids(counts)
        dst_keep = keep_seg[dst_seg]
        new_xy[dst_keep] = xy[src_keep]
        new_xy[~dst_keep] = sq.reshape(-1, 2)
        xy, off = new_xy, new_off
    return xy, off


def mbrs(xy: np.ndarray, off: np.ndarray) -> np.ndarray:
    """Closed MBR (x0, y0, x1, y1) of every polygon, lattice units, int64."""
    s = off[:-1]
    return np.stack([np.minimum.reduceat(xy[:, 0], s), np.minimum.reduceat(xy[:, 1], s),
                     np.maximum.reduceat(xy[:, 0], s), np.maximum.reduceat(xy[:, 1], s)], 1)


def is_simple_star(xy: np.ndarray, cen: np.ndarray) -> bool:
    """Exact check that a single polygon is strictly star-shaped around cen."""
    a = xy - cen
    b = np.roll(a, -1, axis=0)
    cross = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
    wind = int(np.sum((a[:, 1] < 0) & (b[:, 1] >= 0) & (cross > 0)))
    return bool(np.all(cross > 0) and wind == 1 and len(xy) >= 3)
