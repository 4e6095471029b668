"""Selection-query workload (seeded), standing in for the paper's experiment
of Sec. 7 on polygonal range queries: polygons sampled from a county data set
used as selection queries over a landmark or water data set (Sec. 4.3.1).

  data:    the R side of config 2 (200k polygons at scale 1, N=16).
  queries: `n_queries` county-like star polygons, seed 10 / stream 20:
           centres U[0,1]^2, radius log-normal (median 0.005, sigma 0.6)
           capped at 0.03, vertices log-normal (median 400, sigma 0.8)
           clipped to [32, 5000].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import configs as C
from . import polygons as P


@dataclass
class SelectionWorkload:
    name: str
    order: int
    R: C.PolySet        # data polygons
    Q: C.PolySet        # query polygons


def make(scale: float = 1.0, n_queries: int = 1000) -> SelectionWorkload:
    w = C.make(2, scale)
    rng = C._rng(10, 20)
    c = rng.random((n_queries, 2))
    r = np.minimum(C._lognormal(rng, 0.005, 0.6, n_queries), 0.03)
    nv = np.clip(np.rint(C._lognormal(rng, 400, 0.8, n_queries)), 32, 5000).astype(np.int64)
    Q = C._polyset(*P.star_polygons(rng, c, r, nv))
    return SelectionWorkload(name=f"selection-{n_queries}-queries-on-{w.R.n}", order=w.order, R=w.R, Q=Q)
