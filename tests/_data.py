"""Cached workloads for the tests: synthetic inputs, built sets, oracle
verdicts.  Expected values come only from the oracle."""
from __future__ import annotations

import functools

import numpy as np

import oracle
from synth import configs


@functools.lru_cache(maxsize=None)
def workload(cfg: int, scale: float):
    return configs.make(cfg, scale)


@functools.lru_cache(maxsize=None)
def oracle_verdicts(cfg: int, scale: float):
    w = workload(cfg, scale)
    return oracle.verdicts(w.R.xy, w.R.off, w.S.xy, w.S.off, w.pr, w.ps, oracle.Grid(w.order))


def oracle_sample(w, idx):
    idx = np.asarray(idx)
    return oracle.verdicts(w.R.xy, w.R.off, w.S.xy, w.S.off, w.pr[idx], w.ps[idx], oracle.Grid(w.order))


def oracle_sample_pairs(w, pr, ps):
    return oracle.verdicts(w.R.xy, w.R.off, w.S.xy, w.S.off, np.asarray(pr), np.asarray(ps), oracle.Grid(w.order))
