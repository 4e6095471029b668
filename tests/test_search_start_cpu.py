"""The reading behind every join's searched start (CPU only, pure Python).

The merge join of Algorithm 2 asks whether some interval of X meets some
interval of Y.  The kernels start it past a prefix of each list: X from its
first interval whose last cell reaches Y's first start, Y likewise.  The
lane-group engine over raw lists stops its search early and starts at any
position up to that exact one.  These tests check, on random sorted
disjoint interval lists (half-open [st, end) of 32-bit cells, an end of 2^32
included), that a merge started at any positions up to the exact starts
returns the full merge's answer, and that starting past the exact start can
miss an overlap (so the bound is tight).  The kernels also gallop: at a
merge state (i, j) a list that lags may jump ahead to its first interval whose
last cell reaches the other list's current start; the last test checks that
jumps up to that position, taken at any state, keep the answer."""
import numpy as np
import pytest

TOP = 1 << 32


def _lists(rng, k, span):
    """k sorted, disjoint, non-adjacent half-open intervals inside [lo, lo + span)."""
    lo = int(rng.integers(0, TOP - span))
    pts = np.sort(rng.choice(span, 2 * k, replace=False)).astype(np.int64) + lo
    if rng.random() < 0.1:  # one list reaches the last cell (end 2^32)
        pts = pts - pts[-1] + TOP
    return [(int(a), int(b)) for a, b in pts.reshape(-1, 2)]


def _merge(X, Y, i, j):
    """Algorithm 2's merge join from positions (i, j): True iff it finds an overlap."""
    while i < len(X) and j < len(Y):
        (xs, xe), (ys, ye) = X[i], Y[j]
        if xs < ye and ys < xe:
            return True
        if xe <= ys:
            i += 1
        else:
            j += 1
    return False


def _exact_start(X, key):
    """First index whose last cell (end - 1) is >= key."""
    return next((q for q, (_, e) in enumerate(X) if e - 1 >= key), len(X))


def _any_overlap(X, Y):
    return any(xs < ye and ys < xe for xs, xe in X for ys, ye in Y)


@pytest.mark.parametrize("seed", range(6))
def test_start_anywhere_up_to_the_exact_start(seed):
    rng = np.random.default_rng(seed)
    for _ in range(400):
        span = int(rng.integers(64, 4000))
        X = _lists(rng, int(rng.integers(1, 24)), span)
        Y = _lists(rng, int(rng.integers(1, 24)), span)
        want = _any_overlap(X, Y)
        assert _merge(X, Y, 0, 0) == want
        sx, sy = _exact_start(X, Y[0][0]), _exact_start(Y, X[0][0])
        for _ in range(6):
            i, j = int(rng.integers(0, sx + 1)), int(rng.integers(0, sy + 1))
            assert _merge(X, Y, i, j) == want, (X, Y, i, j)


def test_exact_start_is_tight():
    # X's first interval ends before Y starts; its second meets Y's first:
    # starting X one past its exact start misses the only overlap
    X = [(0, 5), (10, 20), (30, 40)]
    Y = [(15, 16)]
    assert _exact_start(X, Y[0][0]) == 1
    assert _merge(X, Y, 1, 0) and not _merge(X, Y, 2, 0)


def _galloping_merge(X, Y, rng):
    """The merge of _merge from (0, 0), except that at random states the
    list whose current interval ends first jumps to a random position up to
    its first interval whose last cell reaches the other's current start."""
    i = j = 0
    while i < len(X) and j < len(Y):
        (xs, xe), (ys, ye) = X[i], Y[j]
        if xs < ye and ys < xe:
            return True
        if rng.random() < 0.3:
            if xe <= ye:
                e = i + _exact_start(X[i:], ys)
                i = int(rng.integers(i, e + 1))
            else:
                e = j + _exact_start(Y[j:], xs)
                j = int(rng.integers(j, e + 1))
            continue
        if xe <= ys:
            i += 1
        else:
            j += 1
    return False


@pytest.mark.parametrize("seed", range(6))
def test_galloping_jumps_keep_the_answer(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(400):
        span = int(rng.integers(256, 4000))
        # lists of very different lengths, where galloping pays
        X = _lists(rng, int(rng.integers(1, 6)), span)
        Y = _lists(rng, int(rng.integers(1, 60)), span)
        if rng.random() < 0.5:
            X, Y = Y, X
        want = _any_overlap(X, Y)
        for _ in range(4):
            assert _galloping_merge(X, Y, rng) == want, (X, Y)
