"""Seeded join requests for the serving workload (config 5).

A request is a spatial query window over the join R x S: the candidate pairs
whose reference point (the lower-left corner of MBR(r) n MBR(s)) lies in the
window.  Its size target is drawn log-uniformly from [lo, hi] pairs; the
window is a square around the reference point of a random candidate and grows
until it holds at least the target number of reference points.  Arrival times
form a Poisson process of a given rate.  Input generation only: nothing here
evaluates the filter.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .polygons import LATTICE_BITS

GRID_BITS = 11  # reference points are counted on a 2048 x 2048 histogram


@dataclass
class Request:
    pr: np.ndarray    # uint32 object ids into R
    ps: np.ndarray    # uint32 object ids into S
    idx: np.ndarray   # positions of these pairs in the workload's candidate list
    arrival: float    # seconds after the start of the stream
    window: tuple     # (cx0, cy0, cx1, cy1) histogram cells, inclusive


class RequestMaker:
    def __init__(self, mbr_r: np.ndarray, mbr_s: np.ndarray, pr: np.ndarray, ps: np.ndarray):
        mr = np.asarray(mbr_r, dtype=np.int64)[pr.astype(np.int64)]
        ms = np.asarray(mbr_s, dtype=np.int64)[ps.astype(np.int64)]
        shift = LATTICE_BITS - GRID_BITS
        G = 1 << GRID_BITS
        self.cx = np.minimum(np.maximum(mr[:, 0], ms[:, 0]) >> shift, G - 1).astype(np.int32)
        self.cy = np.minimum(np.maximum(mr[:, 1], ms[:, 1]) >> shift, G - 1).astype(np.int32)
        hist = np.zeros((G, G), dtype=np.int64)
        np.add.at(hist, (self.cy, self.cx), 1)
        self.cum = np.zeros((G + 1, G + 1), dtype=np.int64)
        self.cum[1:, 1:] = hist.cumsum(0).cumsum(1)
        self.pr, self.ps = pr, ps
        self.G = G

    def count(self, cx0, cy0, cx1, cy1) -> int:
        c = self.cum
        return int(c[cy1 + 1, cx1 + 1] - c[cy0, cx1 + 1] - c[cy1 + 1, cx0] + c[cy0, cx0])

    def window_for(self, k: int, target: int):
        """Smallest square window (in histogram cells) around candidate k's
        reference point holding >= target reference points."""
        x, y = int(self.cx[k]), int(self.cy[k])
        lo, hi = 0, self.G
        while lo < hi:
            a = (lo + hi) // 2
            w = (max(x - a, 0), max(y - a, 0), min(x + a, self.G - 1), min(y + a, self.G - 1))
            if self.count(*w) >= target:
                hi = a
            else:
                lo = a + 1
        a = lo
        return (max(x - a, 0), max(y - a, 0), min(x + a, self.G - 1), min(y + a, self.G - 1))

    def pairs_in(self, w):
        m = (self.cx >= w[0]) & (self.cx <= w[2]) & (self.cy >= w[1]) & (self.cy <= w[3])
        idx = np.nonzero(m)[0]
        return self.pr[idx], self.ps[idx], idx

    def requests(self, seed: int, count: int, rate: float, lo: int = 1_000, hi: int = 2_000_000):
        """`count` requests with log-uniform size targets in [lo, hi] (capped
        by the number of candidates) and Poisson arrivals of `rate` per second."""
        rng = np.random.default_rng(np.random.SeedSequence([seed, 5000]))
        hi = min(hi, len(self.pr))
        lo = min(lo, hi)
        targets = np.exp(rng.uniform(np.log(lo), np.log(hi), count)).astype(np.int64)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, count)) if rate > 0 else np.zeros(count)
        out = []
        for t, at in zip(targets, arrivals):
            k = int(rng.integers(0, len(self.pr)))
            w = self.window_for(k, int(t))
            pr, ps, idx = self.pairs_in(w)
            out.append(Request(pr=pr, ps=ps, idx=idx, arrival=float(at), window=w))
        return out
