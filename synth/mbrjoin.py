"""Candidate pairs from an MBR intersection join (the filter step that precedes
the APRIL intermediate filter, Sec. 2 of the paper).

This is input generation, not the method under test: the paper takes its
candidate pairs from an external MBR-join.  Closed rectangles are used, so
MBRs that only touch are candidates.  Pairs are produced by a uniform-grid
partitioned join; each pair is reported once, by the grid tile that holds the
lower-left corner of MBR(r) n MBR(s) (reference-point duplicate avoidance).
The output is ordered by that tile (row-major), then by r, then by s, which is
the order a tile-by-tile MBR join emits.
"""
from __future__ import annotations

import numpy as np

from .polygons import LATTICE_BITS


def _overlap(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return (a[:, 0] <= b[:, 2]) & (b[:, 0] <= a[:, 2]) & (a[:, 1] <= b[:, 3]) & (b[:, 1] <= a[:, 3])


def _expand(mbr: np.ndarray, idx: np.ndarray, tb: int):
    """Replicate objects idx into every tile (of 2^tb lattice units) they meet."""
    m = mbr[idx]
    tx0 = m[:, 0] >> tb
    ty0 = m[:, 1] >> tb
    tx1 = m[:, 2] >> tb
    ty1 = m[:, 3] >> tb
    nx = tx1 - tx0 + 1
    ny = ty1 - ty0 + 1
    cnt = nx * ny
    rep = np.repeat(np.arange(len(idx)), cnt)
    start = np.zeros(len(idx) + 1, dtype=np.int64)
    np.cumsum(cnt, out=start[1:])
    k = np.arange(int(start[-1]), dtype=np.int64) - start[rep]
    tx = tx0[rep] + k % nx[rep]
    ty = ty0[rep] + k // nx[rep]
    ntiles = 1 << (LATTICE_BITS + 1 - tb)
    tile = ty * ntiles + tx
    return idx[rep], tile


def mbr_join(mbr_r: np.ndarray, mbr_s: np.ndarray, tile_bits: int | None = None,
             big_tiles: int = 16, chunk: int = 1 << 24):
    """Return (pr, ps, tile) uint32/uint32/int64 arrays of candidate pairs."""
    mbr_r = np.asarray(mbr_r, dtype=np.int64)
    mbr_s = np.asarray(mbr_s, dtype=np.int64)
    if tile_bits is None:
        ext = np.concatenate([mbr_r[:, 2] - mbr_r[:, 0], mbr_r[:, 3] - mbr_r[:, 1],
                              mbr_s[:, 2] - mbr_s[:, 0], mbr_s[:, 3] - mbr_s[:, 1]])
        p90 = max(int(np.percentile(ext, 90)) if len(ext) else 1, 1)
        tile_bits = max(int(np.ceil(np.log2(p90))) + 1, 10)
        tile_bits = min(tile_bits, LATTICE_BITS)
    tb = tile_bits
    ntiles_side = 1 << (LATTICE_BITS + 1 - tb)

    def spans(m):
        return np.maximum((m[:, 2] >> tb) - (m[:, 0] >> tb), (m[:, 3] >> tb) - (m[:, 1] >> tb)) + 1

    big_r = spans(mbr_r) > big_tiles
    big_s = spans(mbr_s) > big_tiles
    out_r, out_s, out_t = [], [], []

    # small x small through the tile grid
    ri, rt = _expand(mbr_r, np.nonzero(~big_r)[0], tb)
    si, st = _expand(mbr_s, np.nonzero(~big_s)[0], tb)
    ro = np.argsort(rt, kind="stable")
    ri, rt = ri[ro], rt[ro]
    so = np.argsort(st, kind="stable")
    si, st = si[so], st[so]
    ut_r, r_start, r_cnt = np.unique(rt, return_index=True, return_counts=True)
    ut_s, s_start, s_cnt = np.unique(st, return_index=True, return_counts=True)
    common, ir, is_ = np.intersect1d(ut_r, ut_s, assume_unique=True, return_indices=True)
    a = r_cnt[ir]
    b = s_cnt[is_]
    ab = a * b
    # process tiles in chunks bounded by `chunk` generated pairs
    csum = np.cumsum(ab)
    lo = 0
    while lo < len(common):
        base = csum[lo - 1] if lo else 0
        hi = int(np.searchsorted(csum, base + chunk, side="right"))
        hi = max(hi, lo + 1)
        sl = slice(lo, hi)
        cnt = ab[sl]
        rep = np.repeat(np.arange(hi - lo), cnt)
        start = np.zeros(hi - lo + 1, dtype=np.int64)
        np.cumsum(cnt, out=start[1:])
        k = np.arange(int(start[-1]), dtype=np.int64) - start[rep]
        bb = b[sl][rep]
        pr = ri[r_start[ir[sl]][rep] + k // bb]
        ps = si[s_start[is_[sl]][rep] + k % bb]
        tile = common[sl][rep]
        mr = mbr_r[pr]
        ms = mbr_s[ps]
        keep = _overlap(mr, ms)
        refx = np.maximum(mr[:, 0], ms[:, 0]) >> tb
        refy = np.maximum(mr[:, 1], ms[:, 1]) >> tb
        keep &= (refy * ntiles_side + refx) == tile
        out_r.append(pr[keep])
        out_s.append(ps[keep])
        out_t.append(tile[keep])
        lo = hi

    # pairs involving a big object: brute force against the other side
    def brute(big_idx, other_mbr, other_mask, swap):
        for i in big_idx:
            m = (mbr_r if not swap else mbr_s)[i]
            cand = np.nonzero(other_mask)[0]
            o = other_mbr[cand]
            keep = (o[:, 0] <= m[2]) & (m[0] <= o[:, 2]) & (o[:, 1] <= m[3]) & (m[1] <= o[:, 3])
            c = cand[keep]
            if not len(c):
                continue
            refx = np.maximum(o[keep, 0], m[0]) >> tb
            refy = np.maximum(o[keep, 1], m[1]) >> tb
            t = refy * ntiles_side + refx
            if swap:
                out_r.append(c)
                out_s.append(np.full(len(c), i, dtype=np.int64))
            else:
                out_r.append(np.full(len(c), i, dtype=np.int64))
                out_s.append(c)
            out_t.append(t)

    brute(np.nonzero(big_r)[0], mbr_s, np.ones(len(mbr_s), dtype=bool), swap=False)
    brute(np.nonzero(big_s)[0], mbr_r, ~big_r, swap=True)

    pr = np.concatenate(out_r) if out_r else np.zeros(0, np.int64)
    ps = np.concatenate(out_s) if out_s else np.zeros(0, np.int64)
    pt = np.concatenate(out_t) if out_t else np.zeros(0, np.int64)
    order = np.lexsort((ps, pr, pt))
    return pr[order].astype(np.uint32), ps[order].astype(np.uint32), pt[order]


def mbr_join_bruteforce(mbr_r: np.ndarray, mbr_s: np.ndarray):
    """All (r, s) with closed MBR overlap, by an O(|R||S|) scan (tiny inputs)."""
    out = []
    for i in range(len(mbr_r)):
        m = mbr_r[i]
        keep = (mbr_s[:, 0] <= m[2]) & (m[0] <= mbr_s[:, 2]) & (mbr_s[:, 1] <= m[3]) & (m[1] <= mbr_s[:, 3])
        for j in np.nonzero(keep)[0]:
            out.append((i, int(j)))
    return out
