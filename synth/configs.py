"""The five synthetic workloads (seeded), standing in for the paper's
SpatialHadoop TIGER/OSM datasets (Sec. 7.1), which are not available here.

Each workload is two polygon sets R and S drawn by `synth.polygons`, a grid
order N, and the candidate pairs of their MBR join.  Config k uses seed k-1;
R draws from stream 2*seed and S from stream 2*seed+1; shared hotspot centres
draw from stream 1000+seed.

  1  tiny:         1,000 + 1,000 polygons, N=12, log-normal radius
                   (median 0.005, sigma 0.8), 20-200 vertices.
  2  paper scale:  200k + 200k polygons, N=16, vertices log-normal (median 60,
                   sigma 1.0, clipped to [8, 20000]), radius log-normal (median
                   2e-4, sigma 1.2), 5% of centres in 32 Gaussian hotspots.
  3  skewed:       as 2 but radius Pareto(alpha=1.3, x_m=1.17e-4) capped at
                   RADIUS_CAP_SKEWED (A-lists up to ~10^5 intervals); the
                   polygon count is grown from 200k to 340k per side so that
                   the join yields >= 10M candidates, which are then sampled
                   (seeded) to exactly 10M.
  4  partitioned:  the config-2 polygons on a 16x16 partition grid, each
                   partition rasterised at its own 2^14 grid.
  5  serving:      300k + 300k polygons from the config-3 generator, N=16.

`scale` shrinks the polygon counts (tests use small scales); the
distributions are unchanged.
"""
from __future__ import annotations

import os
import tempfile
from dataclasses import dataclass, field

import numpy as np

from . import polygons as P
from .mbrjoin import mbr_join

HOTSPOT_FRAC = 0.05
HOTSPOTS = 32
HOTSPOT_SIGMA = 2.5e-4  # tuned so that the full config-2 join yields 2-5M candidates
RADIUS_CAP_SKEWED = 0.04
PARETO_ALPHA = 1.3
PARETO_XM = 2e-4 / 2 ** (1 / 1.3)


@dataclass
class PolySet:
    xy: np.ndarray          # (V,2) int64 lattice coordinates
    off: np.ndarray         # (n+1,) int64 vertex offsets
    mbr: np.ndarray         # (n,4) int64 closed MBRs (x0,y0,x1,y1)

    @property
    def n(self) -> int:
        return len(self.off) - 1

    def poly(self, i: int) -> np.ndarray:
        return self.xy[self.off[i]:self.off[i + 1]]


@dataclass
class Workload:
    name: str
    order: int                      # grid order N (2^N x 2^N cells)
    R: PolySet
    S: PolySet
    pr: np.ndarray                  # candidate pairs (uint32)
    ps: np.ndarray
    partitions: int = 0             # partitions per dimension (config 4), 0 = global grid
    meta: dict = field(default_factory=dict)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([seed, stream]))


def _lognormal(rng, median, sigma, n):
    return median * np.exp(sigma * rng.standard_normal(n))


def _centers(rng, n, hot_centers):
    c = rng.random((n, 2))
    if hot_centers is not None and len(hot_centers):
        nh = int(round(HOTSPOT_FRAC * n))
        which = rng.integers(0, len(hot_centers), nh)
        pick = rng.choice(n, nh, replace=False)
        c[pick] = hot_centers[which] + HOTSPOT_SIGMA * rng.standard_normal((nh, 2))
    return np.clip(c, 1e-6, 1 - 1e-6)


def _polyset(xy, off) -> PolySet:
    return PolySet(xy=xy, off=off, mbr=P.mbrs(xy, off))


def tiny_side(seed: int, stream: int, n: int) -> PolySet:
    rng = _rng(seed, stream)
    c = rng.random((n, 2))
    r = _lognormal(rng, 0.005, 0.8, n)
    nv = rng.integers(20, 201, n)
    return _polyset(*P.star_polygons(rng, c, r, nv))


def paper_side(seed: int, stream: int, n: int, hot, skewed: bool) -> PolySet:
    rng = _rng(seed, stream)
    c = _centers(rng, n, hot)
    if skewed:
        r = PARETO_XM * (1.0 + rng.pareto(PARETO_ALPHA, n))
        r = np.minimum(r, RADIUS_CAP_SKEWED)
    else:
        r = _lognormal(rng, 2e-4, 1.2, n)
    nv = np.clip(np.rint(_lognormal(rng, 60, 1.0, n)), 8, 20000).astype(np.int64)
    return _polyset(*P.star_polygons(rng, c, r, nv))


def _hot(seed):
    return 0.1 + 0.8 * _rng(seed, 1000).random((HOTSPOTS, 2))


RECIPE_VERSION = 5


def _cache_path(cfg, scale, max_pairs):
    d = os.environ.get("APRIL_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "april_synth_cache"))
    return os.path.join(d, f"cfg{cfg}_s{scale:g}_m{max_pairs}_v{RECIPE_VERSION}.npz")


def make(cfg: int, scale: float = 1.0, max_pairs: int | None = None, cache: bool = True) -> Workload:
    """Build (or load from the on-disk cache) workload `cfg` at `scale`."""
    if cfg == 4:  # the config-2 polygons and candidates, on 16x16 partitions of order 14
        w = make(2, scale, max_pairs, cache)
        return Workload(name="partitioned-16x16-n14", order=14, R=w.R, S=w.S, pr=w.pr, ps=w.ps, partitions=16,
                        meta=dict(w.meta))
    use_cache = cache and scale >= 0.05
    if use_cache:
        path = _cache_path(cfg, scale, max_pairs)
        if os.path.exists(path):
            try:
                z = np.load(path)
                R = PolySet(z["rxy"].astype(np.int64), z["roff"], z["rmbr"])
                S = PolySet(z["sxy"].astype(np.int64), z["soff"], z["smbr"])
                return Workload(name=str(z["name"]), order=int(z["order"]), R=R, S=S, pr=z["pr"], ps=z["ps"],
                                partitions=int(z["parts"]), meta=dict(zip(z["mk"].tolist(), z["mv"].tolist())))
            except Exception:
                pass
    w = _make(cfg, scale, max_pairs)
    if use_cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".tmp{os.getpid()}.npz"
            np.savez(tmp, rxy=w.R.xy.astype(np.int32), roff=w.R.off, rmbr=w.R.mbr,
                     sxy=w.S.xy.astype(np.int32), soff=w.S.off, smbr=w.S.mbr, pr=w.pr, ps=w.ps,
                     name=w.name, order=w.order, parts=w.partitions,
                     mk=np.array(list(w.meta.keys())), mv=np.array(list(w.meta.values())))
            os.replace(tmp, path)
        except OSError:
            pass
    return w


def _make(cfg: int, scale: float, max_pairs: int | None) -> Workload:
    seed = cfg - 1
    if cfg == 1:
        n = max(int(round(1000 * scale)), 2)
        R = tiny_side(seed, 2 * seed, n)
        S = tiny_side(seed, 2 * seed + 1, n)
        order = 12
    elif cfg in (2, 4):
        n = max(int(round(200_000 * scale)), 2)
        hot = _hot(1)  # config 4 reuses the config-2 generator (seed 1)
        sd = 1
        R = paper_side(sd, 2 * sd, n, hot, skewed=False)
        S = paper_side(sd, 2 * sd + 1, n, hot, skewed=False)
        order = 16 if cfg == 2 else 14
    elif cfg in (3, 5):
        base = 340_000 if cfg == 3 else 300_000  # config 3 grown from 200k until the join yields >= 10M
        n = max(int(round(base * scale)), 2)
        hot = _hot(2)
        sd = 2 if cfg == 3 else 4
        R = paper_side(sd, 2 * sd, n, hot, skewed=True)
        S = paper_side(sd, 2 * sd + 1, n, hot, skewed=True)
        order = 16
    else:
        raise ValueError(f"unknown config {cfg}")
    pr, ps, _ = mbr_join(R.mbr, S.mbr)
    meta = {"candidates_joined": int(len(pr))}
    if cfg == 3 and max_pairs is None:
        max_pairs = int(round(10_000_000 * scale))
    if max_pairs is not None and len(pr) > max_pairs:
        keep = np.sort(_rng(seed, 2000).choice(len(pr), max_pairs, replace=False))
        pr, ps = pr[keep], ps[keep]
        meta["sampled_to"] = int(max_pairs)
    names = {1: "tiny-plain-1k", 2: "paper-scale-200k", 3: "skewed-pareto-340k-10M",
             4: "partitioned-16x16-n14", 5: "serving-300k"}
    return Workload(name=names[cfg], order=order, R=R, S=S, pr=pr, ps=ps,
                    partitions=16 if cfg == 4 else 0, meta=meta)
