"""Cached workloads for the tests: synthetic inputs, built sets, oracle
verdicts.  Expected values come only from the oracle.  The oracle's C calls
release the GIL, so long runs are split into contiguous chunks (keeping its
per-side raster cache useful) evaluated on a thread pool."""
from __future__ import annotations

import functools
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle
from synth import configs


@functools.lru_cache(maxsize=None)
def workload(cfg: int, scale: float):
    return configs.make(cfg, scale)


def _chunked(fn, pr, ps, min_chunk=16):
    pr = np.ascontiguousarray(pr, dtype=np.uint32)
    ps = np.ascontiguousarray(ps, dtype=np.uint32)
    n = len(pr)
    workers = max(1, os.cpu_count() or 1)
    if n <= min_chunk or workers == 1:
        return fn(pr, ps)
    bounds = np.linspace(0, n, min(4 * workers, n // min_chunk) + 1).astype(np.int64)
    with ThreadPoolExecutor(workers) as ex:
        parts = list(ex.map(lambda ab: fn(pr[ab[0]:ab[1]], ps[ab[0]:ab[1]]), zip(bounds[:-1], bounds[1:])))
    return np.concatenate(parts)


def oracle_pairs(w, pr, ps):
    """Oracle verdicts of the given pairs of workload w on its own grid."""
    g = oracle.Grid(w.order)
    return _chunked(lambda a, b: oracle.verdicts(w.R.xy, w.R.off, w.S.xy, w.S.off, a, b, g), pr, ps)


def oracle_pairs_ex(w, pr, ps, order_r, order_s, pred):
    """Oracle verdicts of a filter variant (global grids of the given orders)."""
    return _chunked(lambda a, b: oracle.verdicts_ex(w.R.xy, w.R.off, w.S.xy, w.S.off, a, b, order_r, order_s, pred),
                    pr, ps)


@functools.lru_cache(maxsize=None)
def oracle_verdicts(cfg: int, scale: float):
    w = workload(cfg, scale)
    return oracle_pairs(w, w.pr, w.ps)


@functools.lru_cache(maxsize=None)
def oracle_verdicts_ex(cfg: int, scale: float, order_r: int, order_s: int, pred: int):
    w = workload(cfg, scale)
    return oracle_pairs_ex(w, w.pr, w.ps, order_r, order_s, pred)


def oracle_sample(w, idx):
    idx = np.asarray(idx)
    return oracle_pairs(w, w.pr[idx], w.ps[idx])


def oracle_sample_pairs(w, pr, ps):
    return oracle_pairs(w, pr, ps)
