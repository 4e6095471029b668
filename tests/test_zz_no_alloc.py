"""The allocation-free filter entry point (GPU only).

april_filter_pairs_noalloc is for callers that cannot allocate device memory
while they filter (allocation is forbidden or would stall the device on their
call path); its scratch is a static device array inside libapril.  These
tests call it through the C ABI and check it against april_filter_pairs on
the same pairs, twice in a row (the array keeps the previous call's contents,
so the second call checks that the state is reset), check that further calls
take no device memory, and read the entry point's own status word through
april_noalloc_sync_status (bad ids; a bounded wait made to run out at once by
the diagnostic wait limit, which needs no fault).  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from tests import _data
from paper_2307_01716_gb300 import april as A

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _setup(torch, cfg, scale):
    w = _data.workload(cfg, scale)
    g = A.global_grid(w.order)
    R = A.april_build_sets(w.R.xy, w.R.off, g)
    S = A.april_build_sets(w.S.xy, w.S.off, g)
    dR, dS = A.april_upload(R), A.april_upload(S)
    d_r = torch.from_numpy(w.pr.view(np.int32)).cuda()
    d_s = torch.from_numpy(w.ps.view(np.int32)).cuda()
    return w, R, S, dR, dS, d_r, d_s


@pytest.mark.parametrize("cfg,scale", [(1, 1.0), (3, 0.01)])
def test_noalloc_matches_allocating_entry_point(torch_cuda, cfg, scale):
    torch = torch_cuda
    w, R, S, dR, dS, d_r, d_s = _setup(torch, cfg, scale)
    n = len(w.pr)
    ctx = A.Context(0)
    ref = torch.zeros(n, dtype=torch.uint8, device="cuda")
    scratch = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device="cuda")
    ctx.april_filter_pairs(dR, dS, d_r, d_s, n, ref, A.MODE_BATCHED, scratch)
    ctx.april_sync_status()
    want = ref.cpu().numpy()
    for call in range(2):
        out = torch.full((n,), 0xEE, dtype=torch.uint8, device="cuda")
        A.april_filter_pairs_noalloc(dR, dS, d_r, d_s, n, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, want), f"call {call}: {np.nonzero(got != want)[0][:10]}"


def test_noalloc_rejects_oversize_and_bad_ids(torch_cuda):
    torch = torch_cuda
    w, R, S, dR, dS, d_r, d_s = _setup(torch, 1, 1.0)
    out = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AprilError) as e:
        A.april_filter_pairs_noalloc(dR, dS, d_r, d_s, A.NOALLOC_MAX_PAIRS + 1, out)
    assert e.value.status == -1 and "APRIL_NOALLOC_MAX_PAIRS" in str(e.value)
    bad_r = torch.from_numpy(np.array([0, 5000, 1], dtype=np.uint32).view(np.int32)).cuda()
    bad_s = torch.from_numpy(np.array([0, 0, 7000], dtype=np.uint32).view(np.int32)).cuda()
    A.april_filter_pairs_noalloc(dR, dS, bad_r, bad_s, 3, out)
    torch.cuda.synchronize()
    assert out[1:3].cpu().tolist() == [0xFF, 0xFF]
    # the status word keeps the bad ids until the query reads and clears it
    with pytest.raises(A.AprilError) as e:
        A.april_noalloc_sync_status()
    assert e.value.status == -2
    A.april_noalloc_sync_status()


def test_noalloc_takes_no_device_memory(torch_cuda):
    torch = torch_cuda
    w, R, S, dR, dS, d_r, d_s = _setup(torch, 1, 1.0)
    n = len(w.pr)
    out = torch.empty(n, dtype=torch.uint8, device="cuda")
    A.april_filter_pairs_noalloc(dR, dS, d_r, d_s, n, out)  # warm-up: loads the module if nothing had
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        A.april_filter_pairs_noalloc(dR, dS, d_r, d_s, n, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    A.april_noalloc_sync_status()


def test_noalloc_timeout_is_reported(torch_cuda):
    """With the wait limit at 0 every window wait gives up at once: the kernel
    waits for its copies, marks the pairs it held as errors and records the
    timeout, which the status query reports; the next call at the default
    limit is correct again."""
    torch = torch_cuda
    w, R, S, dR, dS, d_r, d_s = _setup(torch, 3, 0.01)
    n = len(w.pr)
    ctx = A.Context(0)
    ref = torch.zeros(n, dtype=torch.uint8, device="cuda")
    scratch = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device="cuda")
    ctx.april_filter_pairs(dR, dS, d_r, d_s, n, ref, A.MODE_BATCHED, scratch)
    ctx.april_sync_status()
    A.april_noalloc_sync_status()
    out = torch.full((n,), 0xEE, dtype=torch.uint8, device="cuda")
    try:
        A.april_debug_set_wait_limit(0)
        A.april_filter_pairs_noalloc(dR, dS, d_r, d_s, n, out)
        torch.cuda.synchronize()
    finally:
        A.april_debug_set_wait_limit(A.WAIT_LIMIT_DEFAULT)
    with pytest.raises(A.AprilError) as e:
        A.april_noalloc_sync_status()
    assert e.value.status == -5
    assert int((out.cpu().numpy() == 0xFF).sum()) > 0
    out.fill_(0xEE)
    A.april_filter_pairs_noalloc(dR, dS, d_r, d_s, n, out)
    A.april_noalloc_sync_status()
    assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
