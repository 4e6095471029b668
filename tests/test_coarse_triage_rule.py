"""The rule of the different-granularity triage (CPU, against the oracle).

On global grids of orders N_f > N_c over the same space, let c be the cell of
the coarse grid under the centre of MBR(r) n MBR(s).  The triage declares a
true hit when c is a Full cell of the coarse side and some Partial-or-Full
cell of the fine side lies inside c.  On nested grids the fine cells inside
c are those whose Hilbert ids, shifted right by 2 (N_f - N_c), give c's id
(the nesting is pinned in test_oracle_pins.py), so this is the id-range test
the kernel makes.  Stated here on cell coordinates, the rule must only ever
fire on pairs the oracle's variant filter (Sec. 5.3) calls true hits, and it
must fire on a fair share of them."""
import numpy as np
import pytest

import oracle
from tests import _data


def _mbr(xy, off, k):
    p = xy[off[k]:off[k + 1]]
    return p[:, 0].min(), p[:, 1].min(), p[:, 0].max(), p[:, 1].max()


@pytest.mark.parametrize("o_r,o_s", [(12, 10), (10, 12), (12, 8)])
def test_coarse_triage_rule_is_sound(o_r, o_s):
    w = _data.workload(1, 1.0)
    fine_is_r = o_r > o_s
    o_f, o_c = max(o_r, o_s), min(o_r, o_s)
    d = o_f - o_c
    g_f, g_c = oracle.Grid(o_f), oracle.Grid(o_c)
    want = _data.oracle_pairs_ex(w, w.pr, w.ps, o_r, o_s, 0)
    cache = {}

    def cells(side, k, g):
        key = (side, k, g.order)
        if key not in cache:
            xy, off = (w.R.xy, w.R.off) if side == "r" else (w.S.xy, w.S.off)
            cache[key] = oracle.cells(xy[off[k]:off[k + 1]], g)
        return cache[key]

    fired = 0
    for r, s, v in zip(w.pr.tolist(), w.ps.tolist(), want.tolist()):
        a, b = _mbr(w.R.xy, w.R.off, r), _mbr(w.S.xy, w.S.off, s)
        x0, y0, x1, y1 = max(a[0], b[0]), max(a[1], b[1]), min(a[2], b[2]), min(a[3], b[3])
        if x0 > x1 or y0 > y1:
            continue
        cx, cy = ((x0 + x1) // 2) // g_c.h, ((y0 + y1) // 2) // g_c.h
        if not (0 <= cx < g_c.G and 0 <= cy < g_c.G):
            continue
        fine, coarse = ("r", r), ("s", s)
        if not fine_is_r:
            fine, coarse = coarse, fine
        _, F_c = cells(coarse[0], coarse[1], g_c)
        if (cx, cy) not in F_c:
            continue
        A_f, _ = cells(fine[0], fine[1], g_f)
        if any((i >> d, j >> d) == (cx, cy) for i, j in A_f):
            fired += 1
            assert v == 1, (r, s, v)
    true_hits = int((want == 1).sum())
    assert true_hits > 100
    assert fired > 0.3 * true_hits, (fired, true_hits)
