"""Thin ctypes binding of libapril (include/april.h).

Argument marshalling only: every step of the filter runs inside libapril's
CUDA kernels.  PyTorch supplies device memory and streams.  Importing this
module loads the in-tree libapril.so and raises if it is missing; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("APRIL_LIB", os.path.join(HERE, "libapril.so"))

APRIL_OK = 0
APRIL_PENDING = 1
ERRORS = {
    -1: "INVALID_ARG", -2: "OUT_OF_RANGE_ID", -3: "OVER_BUDGET", -4: "CUDA_ERROR",
    -5: "DEVICE_TIMEOUT", -6: "CANCELLED", -7: "NO_MEMORY", -8: "GEOMETRY",
}
TRUE_NEGATIVE, TRUE_HIT, INCONCLUSIVE, VERDICT_ERROR = 0, 1, 2, 0xFF
MODE_PLAIN, MODE_WARP, MODE_BATCHED, MODE_BATCHED_PACKED = 0, 1, 2, 3
PREDICATE_INTERSECTS, PREDICATE_WITHIN = 0, 1
MODES = {"plain": MODE_PLAIN, "warp": MODE_WARP, "batched": MODE_BATCHED}


class AprilError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"april status {status} ({ERRORS.get(status, '?')}): {msg}")
        self.status = status


class april_grid(ctypes.Structure):
    _fields_ = [("ox", ctypes.c_int64), ("oy", ctypes.c_int64),
                ("log2_cell", ctypes.c_uint32), ("order", ctypes.c_uint32)]


class april_sets_info(ctypes.Structure):
    _fields_ = [("n_objects", ctypes.c_uint32), ("order", ctypes.c_uint32),
                ("a_intervals", ctypes.c_uint64), ("f_intervals", ctypes.c_uint64),
                ("iv_slots", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("parts", ctypes.c_uint32), ("n_entries", ctypes.c_uint32), ("packed", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("raw_list_bytes", ctypes.c_uint64),
                ("packed_list_bytes", ctypes.c_uint64)]


class april_tune(ctypes.Structure):
    _fields_ = [("cta_threshold", ctypes.c_uint32), ("group_lanes", ctypes.c_uint32),
                ("group_window", ctypes.c_uint32), ("cta_window", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("ms", ctypes.c_float), ("join_order", ctypes.c_uint32),
                ("escalate_windows", ctypes.c_uint32), ("triage_off", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class april_req_stats(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_uint64), ("submit_ns", ctypes.c_int64), ("admit_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64), ("slot", ctypes.c_uint32), ("status", ctypes.c_int32)]


class april_server_info(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("pending", ctypes.c_uint64),
                ("in_flight", ctypes.c_uint64), ("max_concurrent", ctypes.c_uint64),
                ("arena_bytes", ctypes.c_uint64), ("arena_peak_bytes", ctypes.c_uint64)]


class april_device_build_info(ctypes.Structure):
    _fields_ = [("touched_cells", ctypes.c_uint64), ("work_bytes", ctypes.c_uint64), ("image_bytes", ctypes.c_uint64),
                ("iv_slots", ctypes.c_uint64)]


class april_index_info(ctypes.Structure):
    _fields_ = [("bucket_bits", ctypes.c_uint32), ("n_objects", ctypes.c_uint32), ("n_entries", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64)]


class april_dev_index(ctypes.Structure):
    _fields_ = [("off", ctypes.c_void_p), ("ent", ctypes.c_void_p), ("ebx", ctypes.c_void_p),
                ("bucket_bits", ctypes.c_uint32), ("n_objects", ctypes.c_uint32), ("n_entries", ctypes.c_uint64)]


class april_dev_sets(ctypes.Structure):
    _fields_ = [("desc", ctypes.c_void_p), ("iv", ctypes.c_void_p), ("n_objects", ctypes.c_uint32),
                ("order", ctypes.c_uint32), ("iv_slots", ctypes.c_uint64), ("n_entries", ctypes.c_uint32),
                ("parts", ctypes.c_uint32), ("obj_ll", ctypes.c_void_p), ("obj_entry", ctypes.c_void_p),
                ("entry_pid", ctypes.c_void_p), ("pdesc", ctypes.c_void_p), ("anchors", ctypes.c_void_p),
                ("gaps", ctypes.c_void_p), ("mbr", ctypes.c_void_p), ("posts", ctypes.c_void_p),
                ("grid_ox", ctypes.c_int64), ("grid_oy", ctypes.c_int64), ("grid_log2_cell", ctypes.c_uint32),
                ("grid_known", ctypes.c_uint32), ("part_grid", ctypes.c_void_p), ("grid_id", ctypes.c_uint64)]


_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_st = ctypes.c_int32

# name -> (restype, argtypes); the same names as include/april.h
SIGNATURES = {
    "april_last_error": (_st, [ctypes.c_char_p, ctypes.c_size_t]),
    "april_build_sets": (_st, [_vp, _vp, _u32, ctypes.POINTER(april_grid), _u32, ctypes.POINTER(_vp)]),
    "april_cell_ids": (_st, [ctypes.POINTER(april_grid), _vp, _vp, _u64, _vp]),
    "april_sets_destroy": (None, [_vp]),
    "april_sets_get_info": (_st, [_vp, ctypes.POINTER(april_sets_info)]),
    "april_sets_list": (_st, [_vp, _u32, ctypes.c_int, ctypes.POINTER(ctypes.POINTER(_u32)),
                              ctypes.POINTER(_u32)]),
    "april_upload": (_st, [_vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(april_dev_sets)]),
    "april_ctx_create": (_st, [ctypes.c_int, ctypes.POINTER(_vp)]),
    "april_ctx_destroy": (None, [_vp]),
    "april_ctx_graph_stats": (_st, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "april_filter_scratch_bytes": (_st, [ctypes.c_int, _u64, ctypes.POINTER(ctypes.c_size_t)]),
    "april_filter_pairs": (_st, [_vp, ctypes.POINTER(april_dev_sets), ctypes.POINTER(april_dev_sets), _vp, _vp,
                                 _u64, _vp, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "april_sync_status": (_st, [_vp, _vp]),
    "april_filter_host_work_bytes": (_st, [ctypes.c_int, _u64, ctypes.POINTER(ctypes.c_size_t)]),
    "april_filter_pairs_host": (_st, [_vp, ctypes.POINTER(april_dev_sets), ctypes.POINTER(april_dev_sets), _vp, _vp,
                                      _u64, _vp, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "april_host_filter": (_st, [_vp, _vp, _vp, _vp, _u64, _u32, _vp, _vp]),
    "april_host_filter_searched": (_st, [_vp, _vp, _vp, _vp, _u64, _u32, _vp, _vp]),
    "april_filter_pairs_ex": (_st, [_vp, ctypes.POINTER(april_dev_sets), ctypes.POINTER(april_dev_sets), _vp, _vp,
                                    _u64, _vp, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "april_host_filter_ex": (_st, [_vp, _vp, _vp, _vp, _u64, ctypes.c_int, _u32, _vp, _vp]),
    "april_sets_lengths": (_st, [_vp, _vp, _vp]),
    "april_route_pairs": (_st, [_vp, _vp, _vp, _vp, _u64, _vp, _vp]),
    "april_quantize_polygons": (_st, [_vp, _vp, _u32, _vp, _vp]),
    "april_build_sets_device": (_st, [_vp, _vp, _vp, _u32, ctypes.POINTER(april_grid), _vp, ctypes.c_size_t, _vp,
                                      ctypes.c_size_t, ctypes.POINTER(april_dev_sets),
                                      ctypes.POINTER(april_device_build_info), _vp]),
    "april_sets_from_lists": (_st, [_u32, _u32, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "april_index_build": (_st, [_vp, _u32, ctypes.POINTER(_vp)]),
    "april_index_destroy": (None, [_vp]),
    "april_index_get_info": (_st, [_vp, ctypes.POINTER(april_index_info)]),
    "april_index_upload": (_st, [_vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(april_dev_index)]),
    "april_select_scratch_bytes": (_st, [_u64, ctypes.POINTER(ctypes.c_size_t)]),
    "april_select": (_st, [_vp, ctypes.POINTER(april_dev_index), ctypes.POINTER(april_dev_sets),
                           ctypes.POINTER(april_dev_sets), _u64, _vp, _vp, _vp, _vp, ctypes.POINTER(_u64), _vp,
                           ctypes.c_size_t, _vp]),
    "april_sets_mbrs": (_st, [_vp, _vp]),
    "april_sets_object_entries": (_st, [_vp, _u32, ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    "april_sets_entry_grid": (_st, [_vp, _u32, ctypes.POINTER(_u32), ctypes.POINTER(april_grid)]),
    "april_build_partitioned_sets": (_st, [_vp, _vp, _u32, _vp, _vp, _u32, _u32, _u32, _u32, ctypes.POINTER(_vp),
                                           ctypes.POINTER(_vp)]),
    "april_sets_compress": (_st, [_vp]),
    "april_server_create": (_st, [_vp, ctypes.POINTER(april_dev_sets), ctypes.POINTER(april_dev_sets), _vp,
                                  ctypes.c_size_t, _u32, ctypes.POINTER(_vp)]),
    "april_submit": (_st, [_vp, _vp, _vp, _u64, _vp, ctypes.POINTER(_u64)]),
    "april_poll": (_st, [_vp, _u64, ctypes.POINTER(april_req_stats)]),
    "april_wait": (_st, [_vp, _u64, _u32, ctypes.POINTER(april_req_stats)]),
    "april_cancel": (_st, [_vp, _u64]),
    "april_server_get_info": (_st, [_vp, ctypes.POINTER(april_server_info)]),
    "april_server_destroy": (None, [_vp]),
    "april_sets_packed_list": (_st, [_vp, _u32, ctypes.c_int, ctypes.POINTER(ctypes.POINTER(_u32)),
                                     ctypes.POINTER(ctypes.POINTER(ctypes.c_uint8)), ctypes.POINTER(_u32)]),
    "april_filter_pairs_noalloc": (_st, [ctypes.POINTER(april_dev_sets), ctypes.POINTER(april_dev_sets), _vp, _vp,
                                         _u64, _vp, _vp]),
    "april_noalloc_sync_status": (_st, [_vp]),
    "april_debug_set_wait_limit": (_st, [_u32]),
    "april_set_tune": (_st, [_vp, ctypes.POINTER(april_tune)]),
    "april_get_tune": (_st, [_vp, ctypes.POINTER(april_tune)]),
    "april_autotune": (_st, [_vp, ctypes.POINTER(april_dev_sets), ctypes.POINTER(april_dev_sets), _vp, _vp, _u64,
                             _vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(april_tune)]),
}

_lib = None


def load():
    """Load libapril.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        from . import build as _build
        if LIB_PATH == _build.OUT and not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libapril.so missing at {LIB_PATH}")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    load().april_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def check(status: int) -> int:
    if status < 0:
        raise AprilError(status, last_error())
    return status


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (no copy)."""
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def global_grid(order: int) -> april_grid:
    return april_grid(0, 0, 24 - order, order)


def grid(order: int, ox: int = 0, oy: int = 0, log2_cell: int | None = None) -> april_grid:
    return april_grid(int(ox), int(oy), 24 - order if log2_cell is None else int(log2_cell), order)


class Sets:
    """Host A/F lists of one polygon set (april_build_sets)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.april_sets_destroy(self.handle)
            self.handle = None

    def info(self) -> april_sets_info:
        inf = april_sets_info()
        check(load().april_sets_get_info(self.handle, ctypes.byref(inf)))
        return inf

    def entries(self, obj: int):
        """(first, count) of the object's entries."""
        f, c = _u32(), _u32()
        check(load().april_sets_object_entries(self.handle, obj, ctypes.byref(f), ctypes.byref(c)))
        return f.value, c.value

    def entry_grid(self, entry: int):
        """(partition id, april_grid) of an entry of partitioned sets."""
        pid, g = _u32(), april_grid()
        check(load().april_sets_entry_grid(self.handle, entry, ctypes.byref(pid), ctypes.byref(g)))
        return pid.value, g

    def compress(self) -> None:
        check(load().april_sets_compress(self.handle))

    def packed_list(self, entry: int, which: int):
        """(n, [(anchor, wide, gap slots uint8[64 or 128]) per block]) of a compressed list."""
        b = ctypes.POINTER(_u32)()
        g = ctypes.POINTER(ctypes.c_uint8)()
        n = _u32()
        check(load().april_sets_packed_list(self.handle, entry, which, ctypes.byref(b), ctypes.byref(g),
                                            ctypes.byref(n)))
        nb = (2 * n.value + 31) // 32
        table = np.ctypeslib.as_array(b, shape=(2 * nb,)).reshape(nb, 2).copy() if nb else np.zeros((0, 2), np.uint32)
        base = ctypes.addressof(g.contents) if nb else 0
        out = []
        for anchor, meta in table:
            wide = int(meta) >> 31
            off = int(meta) & 0x7FFFFFFF
            size = 128 if wide else 64
            slots = np.ctypeslib.as_array((ctypes.c_uint8 * size).from_address(base + 64 * off)).copy()
            out.append((int(anchor), wide, slots))
        return n.value, out

    def mbrs(self) -> np.ndarray:
        """(n_objects, 4) int32 closed MBRs x0, y0, x1, y1 in lattice units."""
        out = np.zeros((self.info().n_objects, 4), dtype=np.int32)
        check(load().april_sets_mbrs(self.handle, _ptr(out)))
        return out

    def lengths(self):
        """(|A|, |F|) of every entry, two uint32 arrays."""
        n = self.info().n_entries
        a = np.zeros(n, dtype=np.uint32)
        f = np.zeros(n, dtype=np.uint32)
        check(load().april_sets_lengths(self.handle, _ptr(a), _ptr(f)))
        return a, f

    def list(self, obj: int, which: int) -> np.ndarray:
        """(n, 2) uint32 array [st, end) of the A (which=0) or F (1) list of an
        entry (the object itself for sets on one grid)."""
        p = ctypes.POINTER(_u32)()
        n = _u32()
        check(load().april_sets_list(self.handle, obj, which, ctypes.byref(p), ctypes.byref(n)))
        if n.value == 0:
            return np.zeros((0, 2), dtype=np.uint32)
        return np.ctypeslib.as_array(p, shape=(n.value * 2,)).reshape(-1, 2).copy()


def april_cell_ids(grd: april_grid, x, y) -> np.ndarray:
    """Hilbert ids of the grid cells holding lattice points (x, y) (UINT64_MAX outside the grid)."""
    x = np.ascontiguousarray(x, dtype=np.int64)
    y = np.ascontiguousarray(y, dtype=np.int64)
    ids = np.zeros(len(x), dtype=np.uint64)
    check(load().april_cell_ids(ctypes.byref(grd), _ptr(x), _ptr(y), len(x), _ptr(ids)))
    return ids


def april_quantize_polygons(xy, vert_off):
    """Data-space polygons (float64 (V, 2) in [0,1]^2, int offsets) to lattice
    polygons: (int32 (V', 2), uint64 offsets)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    off = np.ascontiguousarray(vert_off, dtype=np.uint64)
    out = np.zeros_like(xy, dtype=np.int32)
    out_off = np.zeros(len(off), dtype=np.uint64)
    check(load().april_quantize_polygons(_ptr(xy), _ptr(off), len(off) - 1, _ptr(out), _ptr(out_off)))
    return out[:int(out_off[-1])], out_off


def april_sets_from_lists(order: int, a_lists, f_lists, mbr=None) -> Sets:
    """Sets from per-object (k, 2) [st, end) arrays (sorted, disjoint)."""
    def flat(lists):
        off = np.zeros(len(lists) + 1, dtype=np.uint64)
        off[1:] = np.cumsum([len(L) for L in lists])
        iv = (np.concatenate([np.asarray(L, dtype=np.uint64).reshape(-1, 2) for L in lists]) if len(lists)
              else np.zeros((0, 2), np.uint64))
        return off, np.ascontiguousarray((iv & 0xFFFFFFFF).astype(np.uint32).reshape(-1))
    if len(a_lists) != len(f_lists):
        raise ValueError("a_lists and f_lists differ in length")
    ao, ai = flat(a_lists)
    fo, fi = flat(f_lists)
    m = None if mbr is None else np.ascontiguousarray(mbr, dtype=np.int32)
    h = _vp()
    check(load().april_sets_from_lists(len(a_lists), order, _ptr(ao), _ptr(ai), _ptr(fo), _ptr(fi), _ptr(m),
                                       ctypes.byref(h)))
    return Sets(h.value)


def april_build_sets(xy: np.ndarray, vert_off: np.ndarray, grd: april_grid, n_threads: int = 0) -> Sets:
    xy32 = np.ascontiguousarray(xy, dtype=np.int32).reshape(-1)
    off = np.ascontiguousarray(vert_off, dtype=np.uint64)
    h = _vp()
    check(load().april_build_sets(_ptr(xy32), _ptr(off), len(off) - 1, ctypes.byref(grd), n_threads,
                                  ctypes.byref(h)))
    return Sets(h.value)


def april_build_partitioned_sets(R_xy, R_off, S_xy, S_off, parts: int, order: int, n_threads: int = 0):
    rxy = np.ascontiguousarray(R_xy, dtype=np.int32).reshape(-1)
    sxy = np.ascontiguousarray(S_xy, dtype=np.int32).reshape(-1)
    roff = np.ascontiguousarray(R_off, dtype=np.uint64)
    soff = np.ascontiguousarray(S_off, dtype=np.uint64)
    hr, hs = _vp(), _vp()
    check(load().april_build_partitioned_sets(_ptr(rxy), _ptr(roff), len(roff) - 1, _ptr(sxy), _ptr(soff),
                                              len(soff) - 1, parts, order, n_threads, ctypes.byref(hr),
                                              ctypes.byref(hs)))
    return Sets(hr.value), Sets(hs.value)


@dataclass
class DevSets:
    """A device image of Sets; `buf` (a torch uint8 tensor) keeps the memory alive."""
    c: april_dev_sets
    buf: object

    @property
    def nbytes(self) -> int:
        return int(self.buf.numel())


def april_upload(sets: Sets, device=None, stream=None) -> DevSets:
    import torch
    inf = sets.info()
    buf = torch.empty(max(int(inf.device_bytes), 256), dtype=torch.uint8, device=device or "cuda")
    out = april_dev_sets()
    st = stream if stream is not None else torch.cuda.current_stream(buf.device)
    check(load().april_upload(sets.handle, buf.data_ptr(), buf.numel(), st.cuda_stream, ctypes.byref(out)))
    st.synchronize()  # the host image may be released after this
    return DevSets(out, buf)


class Index:
    """april_index: bucket index over a set's object MBRs (selection queries)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.april_index_destroy(self.handle)
            self.handle = None

    def info(self) -> april_index_info:
        inf = april_index_info()
        check(load().april_index_get_info(self.handle, ctypes.byref(inf)))
        return inf


def april_index_build(sets: Sets, bucket_bits: int = 0) -> Index:
    h = _vp()
    check(load().april_index_build(sets.handle, bucket_bits, ctypes.byref(h)))
    return Index(h.value)


@dataclass
class DevIndex:
    c: april_dev_index
    buf: object


def april_index_upload(index: Index, device=None, stream=None) -> DevIndex:
    import torch
    inf = index.info()
    buf = torch.empty(max(int(inf.device_bytes), 256), dtype=torch.uint8, device=device or "cuda")
    out = april_dev_index()
    st = stream if stream is not None else torch.cuda.current_stream(buf.device)
    check(load().april_index_upload(index.handle, buf.data_ptr(), buf.numel(), st.cuda_stream, ctypes.byref(out)))
    st.synchronize()
    return DevIndex(out, buf)


STATUS_OVER_BUDGET = -3


class Context:
    """april_ctx: device status block and kernel dispatch.  One host thread
    at a time (its captured graph and tuning are unguarded)."""

    def __init__(self, device: int = 0):
        h = _vp()
        check(load().april_ctx_create(device, ctypes.byref(h)))
        self.handle = h.value
        self.device = device

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.april_ctx_destroy(self.handle)
            self.handle = None

    def scratch_bytes(self, mode: int, n: int) -> int:
        b = ctypes.c_size_t()
        check(load().april_filter_scratch_bytes(mode, n, ctypes.byref(b)))
        return b.value

    def april_filter_pairs(self, R: DevSets, S: DevSets, d_r, d_s, n: int, d_verdict, mode: int,
                           scratch=None, stream=None) -> None:
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        sb = 0 if scratch is None else int(scratch.numel() * scratch.element_size())
        check(load().april_filter_pairs(self.handle, ctypes.byref(R.c), ctypes.byref(S.c), _ptr(d_r), _ptr(d_s),
                                        n, _ptr(d_verdict), mode, _ptr(scratch), sb, st.cuda_stream))

    def april_filter_pairs_ex(self, R: DevSets, S: DevSets, d_r, d_s, n: int, d_verdict, predicate: int, scratch,
                              stream=None) -> None:
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        check(load().april_filter_pairs_ex(self.handle, ctypes.byref(R.c), ctypes.byref(S.c), _ptr(d_r), _ptr(d_s), n,
                                           _ptr(d_verdict), predicate, _ptr(scratch), int(scratch.numel()),
                                           st.cuda_stream))

    @staticmethod
    def select_scratch_bytes(capacity: int) -> int:
        b = ctypes.c_size_t()
        check(load().april_select_scratch_bytes(capacity, ctypes.byref(b)))
        return b.value

    def april_select(self, index: DevIndex, R: DevSets, Q: DevSets, capacity: int, d_r, d_q, d_verdict, d_query_off,
                     scratch, stream=None) -> int:
        """Candidate pairs of the queries Q over R and their verdicts; returns
        the number of pairs (d_r, d_q, d_verdict None: count only)."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        n = _u64()
        check(load().april_select(self.handle, ctypes.byref(index.c), ctypes.byref(R.c), ctypes.byref(Q.c), capacity,
                                  _ptr(d_r), _ptr(d_q), _ptr(d_verdict), _ptr(d_query_off), ctypes.byref(n),
                                  _ptr(scratch), int(scratch.numel()), st.cuda_stream))
        return n.value

    def april_build_sets_device(self, d_xy, d_off, grd: april_grid, work=None, image=None, stream=None):
        """GPU construction of the sets of the polygons in device memory
        (d_xy: int32 (V, 2), d_off: int64 (n + 1,) on the device).  Returns
        (DevSets over the image tensor, april_device_build_info).  Buffers that
        are missing or too small are (re)allocated as torch tensors."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(d_xy.device)
        n = int(d_off.numel()) - 1
        info = april_device_build_info()
        out = april_dev_sets()
        fn = load().april_build_sets_device
        for _ in range(3):
            status = fn(self.handle, _ptr(d_xy), _ptr(d_off), n, ctypes.byref(grd), _ptr(work),
                        0 if work is None else int(work.numel()), _ptr(image), 0 if image is None else int(image.numel()),
                        ctypes.byref(out), ctypes.byref(info), st.cuda_stream)
            if status != STATUS_OVER_BUDGET:
                check(status)
                return DevSets(out, image), info
            if work is None or work.numel() < info.work_bytes:
                work = torch.empty(int(info.work_bytes), dtype=torch.uint8, device=d_xy.device)
            if info.image_bytes and (image is None or image.numel() < info.image_bytes):
                image = torch.empty(int(info.image_bytes), dtype=torch.uint8, device=d_xy.device)
        check(status)

    def get_tune(self) -> april_tune:
        t = april_tune()
        check(load().april_get_tune(self.handle, ctypes.byref(t)))
        return t

    def set_tune(self, t: april_tune) -> None:
        check(load().april_set_tune(self.handle, ctypes.byref(t)))

    def april_autotune(self, R: DevSets, S: DevSets, d_r, d_s, n: int, d_verdict, scratch, stream=None) -> april_tune:
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        t = april_tune()
        check(load().april_autotune(self.handle, ctypes.byref(R.c), ctypes.byref(S.c), _ptr(d_r), _ptr(d_s), n,
                                    _ptr(d_verdict), _ptr(scratch), int(scratch.numel()), st.cuda_stream,
                                    ctypes.byref(t)))
        return t

    def host_work_bytes(self, mode: int, n: int) -> int:
        b = ctypes.c_size_t()
        check(load().april_filter_host_work_bytes(mode, n, ctypes.byref(b)))
        return b.value

    def april_filter_pairs_host(self, R: DevSets, S: DevSets, h_r, h_s, n: int, h_verdict, mode: int, work,
                                stream=None) -> int:
        """Host pairs in, host verdicts out (synchronous); `work` is a device uint8 tensor."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        return check(load().april_filter_pairs_host(self.handle, ctypes.byref(R.c), ctypes.byref(S.c), _ptr(h_r),
                                                    _ptr(h_s), n, _ptr(h_verdict), mode, _ptr(work),
                                                    int(work.numel()), st.cuda_stream))

    def april_ctx_graph_stats(self):
        """(captures, launches) of the batched pipeline's CUDA graph."""
        c, l = ctypes.c_uint64(), ctypes.c_uint64()
        check(load().april_ctx_graph_stats(self.handle, ctypes.byref(c), ctypes.byref(l)))
        return c.value, l.value

    def april_sync_status(self, stream=None) -> int:
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        return check(load().april_sync_status(self.handle, st.cuda_stream))


class Server:
    """Serving loop over resident sets (april_server_*).  Keeps the arena,
    the sets and every submitted request's host buffers alive."""

    def __init__(self, ctx: "Context", R: DevSets, S: DevSets, arena, max_inflight: int = 4):
        self._ctx, self._R, self._S, self._arena = ctx, R, S, arena
        h = _vp()
        check(load().april_server_create(ctx.handle, ctypes.byref(R.c), ctypes.byref(S.c), _ptr(arena),
                                         int(arena.numel()), max_inflight, ctypes.byref(h)))
        self.handle = h.value
        self._live = {}

    def april_submit(self, h_r, h_s, h_verdict) -> int:
        t = _u64()
        n = len(h_r)
        check(load().april_submit(self.handle, _ptr(h_r), _ptr(h_s), n, _ptr(h_verdict), ctypes.byref(t)))
        self._live[t.value] = (h_r, h_s, h_verdict)
        return t.value

    def april_poll(self, ticket: int):
        """None while pending, else april_req_stats (raises on a failed request)."""
        st = april_req_stats()
        rc = load().april_poll(self.handle, ticket, ctypes.byref(st))
        if rc == APRIL_PENDING:
            return None
        self._live.pop(ticket, None)
        check(rc)
        return st

    def april_wait(self, ticket: int, timeout_ms: int = 60000):
        st = april_req_stats()
        rc = load().april_wait(self.handle, ticket, timeout_ms, ctypes.byref(st))
        if rc == APRIL_PENDING:
            return None
        self._live.pop(ticket, None)
        check(rc)
        return st

    def april_cancel(self, ticket: int) -> int:
        return check(load().april_cancel(self.handle, ticket))

    def info(self) -> april_server_info:
        i = april_server_info()
        check(load().april_server_get_info(self.handle, ctypes.byref(i)))
        return i

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.april_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        self.close()


NOALLOC_MAX_PAIRS = 4194304


def april_filter_pairs_noalloc(R: DevSets, S: DevSets, d_r, d_s, n: int, d_verdict, stream=None) -> None:
    """Batched filter with library-owned static scratch, for callers that
    cannot allocate device memory while filtering (see include/april.h)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    check(load().april_filter_pairs_noalloc(ctypes.byref(R.c), ctypes.byref(S.c), _ptr(d_r), _ptr(d_s), n,
                                            _ptr(d_verdict), st.cuda_stream))


def april_noalloc_sync_status(stream=None) -> None:
    """Reads and clears the allocation-free entry point's status word on the
    current device; raises AprilError for a timeout or an out-of-range id."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    check(load().april_noalloc_sync_status(st.cuda_stream))


WAIT_LIMIT_DEFAULT = 16777216


def april_debug_set_wait_limit(spins: int) -> None:
    """Diagnostic: the poll limit of the filter kernels' bounded waits on the
    current device (0: every wait gives up at once)."""
    check(load().april_debug_set_wait_limit(spins))


def april_route_pairs(R: Sets, S: Sets, pr: np.ndarray, ps: np.ndarray):
    """The entries each pair is evaluated on (partitioned sets: the partition
    of the lower-left corner of MBR(r) n MBR(s)); two uint32 arrays."""
    pr = np.ascontiguousarray(pr, dtype=np.uint32)
    ps = np.ascontiguousarray(ps, dtype=np.uint32)
    er = np.zeros(len(pr), dtype=np.uint32)
    es = np.zeros(len(pr), dtype=np.uint32)
    check(load().april_route_pairs(R.handle, S.handle, _ptr(pr), _ptr(ps), len(pr), _ptr(er), _ptr(es)))
    return er, es


def april_host_filter_ex(R: Sets, S: Sets, pr: np.ndarray, ps: np.ndarray, predicate: int, n_threads: int = 0):
    """Host execution of the filter variants: (verdicts, consumed intervals)."""
    pr = np.ascontiguousarray(pr, dtype=np.uint32)
    ps = np.ascontiguousarray(ps, dtype=np.uint32)
    v = np.zeros(len(pr), dtype=np.uint8)
    c = np.zeros(len(pr), dtype=np.uint64)
    check(load().april_host_filter_ex(R.handle, S.handle, _ptr(pr), _ptr(ps), len(pr), predicate, n_threads,
                                      _ptr(v), _ptr(c)))
    return v, c


def april_host_filter(R: Sets, S: Sets, pr: np.ndarray, ps: np.ndarray, n_threads: int = 0, searched: bool = False):
    """Host Algorithm 2 over built sets: (verdicts, consumed intervals).
    searched=True starts every join at the searched start the GPU kernels look for
    (april_host_filter_searched: same verdicts, the kernels' reading model)."""
    pr = np.ascontiguousarray(pr, dtype=np.uint32)
    ps = np.ascontiguousarray(ps, dtype=np.uint32)
    v = np.zeros(len(pr), dtype=np.uint8)
    c = np.zeros(len(pr), dtype=np.uint64)
    fn = load().april_host_filter_searched if searched else load().april_host_filter
    check(fn(R.handle, S.handle, _ptr(pr), _ptr(ps), len(pr), n_threads, _ptr(v), _ptr(c)))
    return v, c
