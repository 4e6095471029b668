"""Selection queries on the GPU (Sec. 4.3.1): april_select's candidate pairs
equal the oracle's MBR step exactly (as sets, grouped by query, no
duplicates, the same order on every call), for several bucket sizes; its
verdicts equal the oracle's cell-set verdicts bit for bit; the count-only
and over-capacity paths; and the full 1000-query workload with every
verdict equal to the host execution of Algorithm 2 and a sample equal to the
oracle."""
import numpy as np
import pytest

import oracle
from tests import _data
from paper_2307_01716_gb300 import april as A

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    return A.Context(0)


def _setup(s, bits=0):
    g = A.global_grid(s.order)
    R = A.april_build_sets(s.R.xy, s.R.off, g)
    Q = A.april_build_sets(s.Q.xy, s.Q.off, g)
    I = A.april_index_build(R, bits)
    return R, Q, A.april_upload(R), A.april_upload(Q), A.april_index_upload(I)


def run_select(torch, ctx, dI, dR, dQ, nq, capacity):
    d_r = torch.empty(max(capacity, 1), dtype=torch.int32, device="cuda")
    d_q = torch.empty(max(capacity, 1), dtype=torch.int32, device="cuda")
    d_v = torch.full((max(capacity, 1),), 0xEE, dtype=torch.uint8, device="cuda")
    off = torch.empty(nq + 1, dtype=torch.int32, device="cuda")
    scratch = torch.empty(ctx.select_scratch_bytes(capacity), dtype=torch.uint8, device="cuda")
    n = ctx.april_select(dI, dR, dQ, capacity, d_r, d_q, d_v, off, scratch)
    ctx.april_sync_status()
    cpu = lambda t: t[:n].cpu().numpy().view(np.uint32)
    return cpu(d_r), cpu(d_q), d_v[:n].cpu().numpy(), off.cpu().numpy().view(np.uint32)


def _check_grouping(r, q, off, nq):
    assert off[0] == 0 and off[nq] == len(r) and np.all(np.diff(off.astype(np.int64)) >= 0)
    assert np.array_equal(q, np.repeat(np.arange(nq, dtype=np.uint32), np.diff(off.astype(np.int64))))
    key = q.astype(np.uint64) << 32 | r
    assert len(np.unique(key)) == len(key), "duplicate pairs"


class _Join:
    """The oracle helper's view of (data, queries) as a join workload."""

    def __init__(self, s):
        self.order, self.R, self.S = s.order, s.R, s.Q


@pytest.fixture(scope="module")
def small():
    from synth import selection
    s = selection.make(0.05, 80)
    want_r, want_q = oracle.select_candidates(s.R.mbr, s.Q.mbr)
    want_v = _data.oracle_pairs(_Join(s), want_r, want_q)
    assert len(want_r) > 300 and np.bincount(want_v, minlength=3).min() > 0
    return s, want_r, want_q, want_v


@pytest.mark.parametrize("bits", [0, 1, 5, 12])
def test_select_equals_oracle(torch_cuda, ctx, small, bits):
    s, want_r, want_q, want_v = small
    R, Q, dR, dQ, dI = _setup(s, bits)
    r, q, v, off = run_select(torch_cuda, ctx, dI, dR, dQ, s.Q.n, len(want_r) + 7)
    _check_grouping(r, q, off, s.Q.n)
    order = np.lexsort((r, q))
    assert np.array_equal(r[order], want_r) and np.array_equal(q[order], want_q)
    assert np.array_equal(v[order], want_v)
    # the same pairs in the same order on a second call
    r2, q2, v2, _ = run_select(torch_cuda, ctx, dI, dR, dQ, s.Q.n, len(want_r))
    assert np.array_equal(r, r2) and np.array_equal(q, q2) and np.array_equal(v, v2)


def test_select_count_only_and_capacity(torch_cuda, ctx):
    torch = torch_cuda
    from synth import selection
    s = selection.make(0.05, 30)
    R, Q, dR, dQ, dI = _setup(s)
    want = len(oracle.select_candidates(s.R.mbr, s.Q.mbr)[0])
    off = torch.empty(s.Q.n + 1, dtype=torch.int32, device="cuda")
    scratch = torch.empty(ctx.select_scratch_bytes(0), dtype=torch.uint8, device="cuda")
    assert ctx.april_select(dI, dR, dQ, 0, None, None, None, off, scratch) == want
    assert int(off[-1].item()) == want
    small = max(want // 2, 1)
    d_r = torch.empty(small, dtype=torch.int32, device="cuda")
    d_v = torch.empty(small, dtype=torch.uint8, device="cuda")
    scratch = torch.empty(ctx.select_scratch_bytes(small), dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AprilError) as e:
        ctx.april_select(dI, dR, dQ, small, d_r, d_r.clone(), d_v, off, scratch)
    assert e.value.status == -3
    # a query set on another grid is refused
    Q2 = A.april_upload(A.april_build_sets(s.Q.xy, s.Q.off, A.global_grid(s.order - 1)))
    with pytest.raises(A.AprilError):
        ctx.april_select(dI, dR, Q2, 0, None, None, None, off, scratch)


def test_select_full_workload(torch_cuda, ctx):
    from synth import selection
    s = selection.make(1.0, 1000)
    R, Q, dR, dQ, dI = _setup(s)
    want_r, want_q = oracle.select_candidates(s.R.mbr, s.Q.mbr)
    r, q, v, off = run_select(torch_cuda, ctx, dI, dR, dQ, s.Q.n, len(want_r))
    _check_grouping(r, q, off, s.Q.n)
    order = np.lexsort((r, q))
    assert np.array_equal(r[order], want_r) and np.array_equal(q[order], want_q)
    hv, _ = A.april_host_filter(R, Q, r, q)
    assert np.array_equal(v, hv)
    idx = np.sort(np.random.default_rng(5).choice(len(r), 200, replace=False))
    assert np.array_equal(v[idx], _data.oracle_pairs(_Join(s), r[idx], q[idx]))
