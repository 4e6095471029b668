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
