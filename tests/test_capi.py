"""The C-ABI library loads on a machine without a GPU and exports every
function include/april.h declares; the binding uses the same names."""
import ctypes
import os
import re

from paper_2307_01716_gb300 import april as A

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "april.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(april_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("april_build_sets", "april_upload", "april_filter_pairs", "april_sync_status"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(A.load()._name)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert sorted(A.SIGNATURES) == declared_functions()


def test_no_device_error_paths():
    """Host-side argument errors come back as status codes, not crashes."""
    import pytest
    with pytest.raises(A.AprilError) as e:
        A.check(A.load().april_filter_scratch_bytes(99, 10, ctypes.byref(ctypes.c_size_t())))
    assert e.value.status == -1
    assert A.load().april_filter_pairs(None, None, None, None, None, 0, None, 0, None, 0, None) == -1


def test_host_work_bytes_cover_both_pipelines():
    """april_filter_host_work_bytes (no device needed) leaves room for the
    staged pairs and verdicts plus the batched scratch of all n pairs (the
    triage pipeline's one rest list) and of two chunks (the chunk-whole
    pipeline); the other modes need the pairs and verdicts only."""
    L = A.load()

    def q(fn, mode, n):
        b = ctypes.c_size_t()
        A.check(fn(mode, n, ctypes.byref(b)))
        return b.value

    for n in (1, 1000, (1 << 18) + 5, (1 << 22) - 1, 1 << 22, 3 * (1 << 22) + 77, 10_000_000):
        for mode in (A.MODE_BATCHED, A.MODE_BATCHED_PACKED):
            work = q(L.april_filter_host_work_bytes, mode, n)
            assert work >= 9 * n + q(L.april_filter_scratch_bytes, mode, n)
        for mode in (A.MODE_PLAIN, A.MODE_WARP):
            assert q(L.april_filter_scratch_bytes, mode, n) == 0
            assert q(L.april_filter_host_work_bytes, mode, n) >= 9 * n
