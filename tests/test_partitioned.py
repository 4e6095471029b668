"""Partitioned sets (paper Sec. 5.2) and compressed lists (Sec. 5.1), host
side (CPU only).

* The builder's partition raster areas equal the oracle's, which are computed
  independently from the same reading of Sec. 5.2.
* Every entry's A/F lists equal the oracle's cell sets on that partition's grid.
* Routing plus Algorithm 2 on the host equals the partitioned oracle.
* Codec: a decoder written here from the format's definition (anchor plus
  running sum of 31 gaps per 32-endpoint block) gives back every raw list.
"""
import numpy as np
import pytest

import oracle
from tests import _data
from paper_2307_01716_gb300 import april as A


@pytest.fixture(scope="module")
def cfg4():
    w = _data.workload(4, 0.005)
    R, S = A.april_build_partitioned_sets(w.R.xy, w.R.off, w.S.xy, w.S.off, 16, 14)
    return w, R, S


def test_partition_areas_equal_oracle(cfg4):
    w, R, S = cfg4
    grids = oracle.partition_areas(w.R.mbr, w.S.mbr, 16, 14)
    met = oracle.partitions_met(w.R.mbr, 16)
    seen = 0
    for obj in range(w.R.n):
        first, count = R.entries(obj)
        assert count == len(met[obj])
        for e in range(first, first + count):
            pid, g = R.entry_grid(e)
            assert pid == met[obj][e - first]
            og = grids[pid]
            assert (g.ox, g.oy, 1 << g.log2_cell, g.order) == (og.ox, og.oy, og.h, og.order)
            seen += 1
    assert seen >= w.R.n


def test_entry_lists_equal_oracle(cfg4):
    w, R, S = cfg4
    grids = oracle.partition_areas(w.R.mbr, w.S.mbr, 16, 14)
    rng = np.random.default_rng(4)
    for obj in rng.choice(w.S.n, 120, replace=False):
        first, count = S.entries(int(obj))
        for e in range(first, first + count):
            pid, _ = S.entry_grid(e)
            La, Lf = oracle.cell_lists(w.S.poly(int(obj)), grids[pid])
            assert np.array_equal(La, S.list(e, 0).astype(np.uint64))
            assert np.array_equal(Lf, S.list(e, 1).astype(np.uint64))


def test_host_routing_filter_equals_partitioned_oracle():
    w = _data.workload(4, 0.02)
    R, S = A.april_build_partitioned_sets(w.R.xy, w.R.off, w.S.xy, w.S.off, 16, 14)
    v, _ = A.april_host_filter(R, S, w.pr, w.ps)
    want = oracle.partitioned_verdicts(w.R.xy, w.R.off, w.R.mbr, w.S.xy, w.S.off, w.S.mbr, w.pr, w.ps, 16, 14)
    assert len(want) > 500
    assert np.array_equal(v, want)


def decode_list(n, blocks):
    """Endpoints of a compressed list, decoded from the format's definition:
    per block, the anchor and then a running sum of the 31 gaps (mod 2^32)."""
    out = []
    for anchor, wide, raw in blocks:
        slots = raw.view(np.uint32 if wide else np.uint16).astype(np.uint64)
        v = anchor
        for k in range(32):
            if k:
                v = (v + int(slots[k])) % (1 << 32)
            out.append(v)
    return np.array(out[:2 * n], dtype=np.uint64).reshape(-1, 2)


def _check_codec(S, entries, smaller=True):
    S.compress()
    inf = S.info()
    assert inf.packed == 1
    if smaller:
        assert inf.packed_list_bytes < 0.7 * inf.raw_list_bytes
    for e in entries:
        for which in (0, 1):
            n, blocks = S.packed_list(e, which)
            raw = S.list(e, which).astype(np.uint64)
            assert n == len(raw)
            assert np.array_equal(decode_list(n, blocks), raw)


def test_codec_round_trip_partitioned(cfg4):
    w, R, S = cfg4
    _check_codec(R, range(0, R.info().n_entries, 7))


def test_codec_round_trip_global_grid_with_wide_gaps_and_last_cell():
    """A global 2^16 grid: far-apart intervals need uint32 gaps, and a list
    holding the last cell ends with the wrapped end 0."""
    order = 16
    h = 1 << (24 - order)
    L = 1 << 24
    polys = [np.array([[L - 3 * h, 0], [L, 0], [L, 3 * h], [L - 3 * h, 3 * h]]),
             np.array([[100, 100], [L - 100, 200], [L // 2, L - 100]]),
             np.array([[5 * h, 5 * h], [9 * h, 5 * h + 7], [7 * h, 9 * h]])]
    xy = np.concatenate(polys)
    off = np.zeros(len(polys) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(p) for p in polys])
    S = A.april_build_sets(xy, off, A.global_grid(order))
    _check_codec(S, range(len(polys)), smaller=False)  # uint32 gaps do not shrink
    assert any(wide for _, wide, _ in S.packed_list(1, 0)[1])  # the big triangle has gaps >= 2^16
    assert S.list(0, 0)[-1, 1] == 0


def test_partitioned_errors():
    with pytest.raises(A.AprilError):
        A.april_build_partitioned_sets(np.zeros((3, 2)), [0, 3], np.zeros((3, 2)), [0, 3], 3, 14)


def test_route_pairs_equals_oracle_routing(cfg4):
    """april_route_pairs names, for every pair, each object's entry for the
    partition the oracle routes the pair to; on one global grid the objects
    themselves; out-of-range ids give UINT32_MAX."""
    w, R, S = cfg4
    er, es = A.april_route_pairs(R, S, w.pr, w.ps)
    part = oracle.route_pairs(w.R.mbr, w.S.mbr, w.pr, w.ps, 16)
    for k in range(len(w.pr)):
        assert R.entry_grid(int(er[k]))[0] == part[k] and S.entry_grid(int(es[k]))[0] == part[k]
        fr, cr = R.entries(int(w.pr[k]))
        fs, cs = S.entries(int(w.ps[k]))
        assert fr <= er[k] < fr + cr and fs <= es[k] < fs + cs
    g = A.global_grid(w.order)
    Rg = A.april_build_sets(w.R.xy, w.R.off, g)
    Sg = A.april_build_sets(w.S.xy, w.S.off, g)
    pr = np.array([0, 1, w.R.n], dtype=np.uint32)
    ps = np.array([2, 3, 0], dtype=np.uint32)
    er, es = A.april_route_pairs(Rg, Sg, pr, ps)
    assert er.tolist() == [0, 1, 0xFFFFFFFF] and es.tolist() == [2, 3, 0xFFFFFFFF]
