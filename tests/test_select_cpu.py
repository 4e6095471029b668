"""Selection queries on the CPU: the oracle's MBR step against hand-built
cases (touching MBRs are candidates, Sec. 4.3.1 with closed regions) and a
pure-Python double loop, and the host index (entry counts from the bucket
spans of every MBR; the C ABI rejects bad arguments)."""
import numpy as np
import pytest

import oracle
from paper_2307_01716_gb300 import april as A


def test_select_candidates_hand_cases():
    data = np.array([[0, 0, 10, 10], [10, 10, 20, 20], [11, 0, 20, 9], [30, 30, 40, 40], [5, 5, 6, 6]])
    queries = np.array([[10, 10, 10, 10],   # a point on two corners
                        [21, 21, 29, 29],   # in the gap
                        [0, 0, 40, 40]])    # everything
    r, q = oracle.select_candidates(data, queries)
    assert list(zip(q.tolist(), r.tolist())) == [(0, 0), (0, 1), (2, 0), (2, 1), (2, 2), (2, 3), (2, 4)]


def test_select_candidates_equal_double_loop():
    rng = np.random.default_rng(3)
    lo = rng.integers(0, 1000, (300, 2))
    data = np.concatenate([lo, lo + rng.integers(0, 80, (300, 2))], 1)
    lo = rng.integers(0, 1000, (40, 2))
    queries = np.concatenate([lo, lo + rng.integers(0, 200, (40, 2))], 1)
    want = [(qi, ri) for qi, Q in enumerate(queries.tolist()) for ri, M in enumerate(data.tolist())
            if M[0] <= Q[2] and Q[0] <= M[2] and M[1] <= Q[3] and Q[1] <= M[3]]
    r, q = oracle.select_candidates(data, queries)
    assert list(zip(q.tolist(), r.tolist())) == want


@pytest.mark.parametrize("bits", [0, 1, 6, 12])
def test_index_entry_counts(bits):
    from synth import selection
    s = selection.make(0.01, 20)
    R = A.april_build_sets(s.R.xy, s.R.off, A.global_grid(s.order))
    assert np.array_equal(R.mbrs(), s.R.mbr.astype(np.int32))
    inf = A.april_index_build(R, bits).info()
    b = inf.bucket_bits
    assert b == bits or (bits == 0 and 4 ** b >= s.R.n and 4 ** (b - 1) < s.R.n)
    cell = 24 - b
    m = s.R.mbr.astype(np.int64)
    span = lambda lo, hi: np.minimum(hi >> cell, (1 << b) - 1) - np.minimum(lo >> cell, (1 << b) - 1) + 1
    assert inf.n_entries == int((span(m[:, 0], m[:, 2]) * span(m[:, 1], m[:, 3])).sum())
    assert inf.n_objects == s.R.n and inf.device_bytes > 0


def test_index_rejects_bad_arguments():
    from synth import configs
    w = configs.make(4, scale=0.005)
    Rp, _ = A.april_build_partitioned_sets(w.R.xy, w.R.off, w.S.xy, w.S.off, 16, 14)
    with pytest.raises(A.AprilError):
        A.april_index_build(Rp)
    from synth import selection
    s = selection.make(0.005, 5)
    R = A.april_build_sets(s.R.xy, s.R.off, A.global_grid(s.order))
    with pytest.raises(A.AprilError):
        A.april_index_build(R, 13)
