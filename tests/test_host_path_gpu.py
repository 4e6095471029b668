"""The end-to-end entry point april_filter_pairs_host (GPU only): host pairs in,
host verdicts out.  In the batched modes it pipelines the pairs: with the
triage, in chunks doubling from 2^18 to 2^21 pairs, each triaged as it
arrives, then one lane-group launch over the rest list; without it, in
chunks of at least 2^22 over two kernel streams.  Its verdicts must equal
host Algorithm 2 (which the CPU tests pin to the oracle) pair for pair
whether the call takes one chunk or several with a ragged last one, on raw,
compressed and partitioned sets, with the triage on and off, and bad ids in
a later chunk must give error verdicts and the OUT_OF_RANGE_ID status."""
import numpy as np
import pytest

from tests import _data
from paper_2307_01716_gb300 import april as A

pytestmark = pytest.mark.gpu

CHUNK = 1 << 22  # the smallest chunk of the pipeline without the triage


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    return A.Context(0)


def _tiled(w, n, seed):
    """n pairs drawn (with repeats) from the workload's candidate pairs."""
    idx = np.random.default_rng(seed).integers(0, len(w.pr), n)
    return np.ascontiguousarray(w.pr[idx]), np.ascontiguousarray(w.ps[idx])


def _host_call(torch, ctx, dR, dS, pr, ps, mode):
    n = len(pr)
    h_r = torch.from_numpy(pr.view(np.int32)).pin_memory()
    h_s = torch.from_numpy(ps.view(np.int32)).pin_memory()
    h_v = torch.full((n,), 0xEE, dtype=torch.uint8).pin_memory()
    work = torch.empty(ctx.host_work_bytes(mode, n), dtype=torch.uint8, device="cuda")
    ctx.april_filter_pairs_host(dR, dS, h_r, h_s, n, h_v, mode, work)
    return h_v.numpy().copy()


@pytest.fixture(scope="module")
def global_sets():
    w = _data.workload(3, 0.02)
    g = A.global_grid(w.order)
    R = A.april_build_sets(w.R.xy, w.R.off, g)
    S = A.april_build_sets(w.S.xy, w.S.off, g)
    return w, R, S


@pytest.mark.parametrize("n", [1000, CHUNK, 2 * CHUNK + 12345])
@pytest.mark.parametrize("packed", [False, True])
def test_host_path_equals_host_alg2(torch_cuda, ctx, global_sets, n, packed):
    w, R, S = global_sets
    pr, ps = _tiled(w, n, n)
    want, _ = A.april_host_filter(R, S, pr, ps)
    if packed:
        R2 = A.april_build_sets(w.R.xy, w.R.off, A.global_grid(w.order))
        S2 = A.april_build_sets(w.S.xy, w.S.off, A.global_grid(w.order))
        R2.compress()
        S2.compress()
        dR, dS, mode = A.april_upload(R2), A.april_upload(S2), A.MODE_BATCHED_PACKED
    else:
        dR, dS, mode = A.april_upload(R), A.april_upload(S), A.MODE_BATCHED
    got = _host_call(torch_cuda, ctx, dR, dS, pr, ps, mode)
    bad = np.flatnonzero(got != want)
    assert len(bad) == 0, (len(bad), bad[:10])
    # again with the same buffers sizes (the context's pipeline is reused)
    got = _host_call(torch_cuda, ctx, dR, dS, pr, ps, mode)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("mode", [A.MODE_PLAIN, A.MODE_WARP])
def test_host_path_single_kernel_modes(torch_cuda, ctx, global_sets, mode):
    w, R, S = global_sets
    pr, ps = _tiled(w, 20_000, 5)
    want, _ = A.april_host_filter(R, S, pr, ps)
    got = _host_call(torch_cuda, ctx, A.april_upload(R), A.april_upload(S), pr, ps, mode)
    assert np.array_equal(got, want)


def test_host_path_without_triage(torch_cuda, ctx, global_sets):
    """triage_off: chunks of at least 2^22 pairs, each filtered whole."""
    w, R, S = global_sets
    n = 2 * CHUNK + 12345
    pr, ps = _tiled(w, n, 17)
    want, _ = A.april_host_filter(R, S, pr, ps)
    saved = ctx.get_tune()
    t = ctx.get_tune()
    t.triage_off = 1
    ctx.set_tune(t)
    try:
        got = _host_call(torch_cuda, ctx, A.april_upload(R), A.april_upload(S), pr, ps, A.MODE_BATCHED)
    finally:
        ctx.set_tune(saved)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("packed", [False, True])
def test_host_path_partitioned(torch_cuda, ctx, packed):
    w = _data.workload(4, 0.02)
    R, S = A.april_build_partitioned_sets(w.R.xy, w.R.off, w.S.xy, w.S.off, w.partitions, w.order)
    pr, ps = _tiled(w, CHUNK + 777, 9)
    want, _ = A.april_host_filter(R, S, pr, ps)
    if packed:
        R.compress()
        S.compress()
    mode = A.MODE_BATCHED_PACKED if packed else A.MODE_BATCHED
    got = _host_call(torch_cuda, ctx, A.april_upload(R), A.april_upload(S), pr, ps, mode)
    assert np.array_equal(got, want)


def test_host_path_bad_ids_in_a_later_chunk(torch_cuda, ctx, global_sets):
    w, R, S = global_sets
    n = 2 * CHUNK + 100
    pr, ps = _tiled(w, n, 3)
    bad = np.array([n - 1, n - 50, CHUNK + 3])
    pr[bad[:2]] = 0xFFFFFFF0
    ps[bad[2]] = 1 << 30
    want, _ = A.april_host_filter(R, S, pr, ps)
    assert (want[bad] == 0xFF).all()
    torch = torch_cuda
    h_r = torch.from_numpy(pr.view(np.int32)).pin_memory()
    h_s = torch.from_numpy(ps.view(np.int32)).pin_memory()
    h_v = torch.full((n,), 0xEE, dtype=torch.uint8).pin_memory()
    work = torch.empty(ctx.host_work_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AprilError) as e:
        ctx.april_filter_pairs_host(A.april_upload(R), A.april_upload(S), h_r, h_s, n, h_v, A.MODE_BATCHED, work)
    assert e.value.status == -2
    assert np.array_equal(h_v.numpy(), want)
    ctx.april_sync_status()  # the status was cleared
