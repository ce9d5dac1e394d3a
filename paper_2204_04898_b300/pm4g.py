"""Python binding of the C ABI in include/pm4g.h (argument marshalling only).

Every function here has the name of the C call it wraps and does nothing but
turn tensors/arrays into pointers and sizes, call the library, and turn the
library's host result arrays into numpy arrays. All computation runs in the
CUDA kernels of libpm4g.so. There is no fallback: if the library is missing,
importing this module fails.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

OK, EINVAL, ERANGE, ENOMEM, ECUDA, ETIMEOUT = 0, -1, -2, -3, -4, -5
HOST_PTRS, DEVICE_PTRS = 0x1, 0x2
VARIANTS_CASES = 0x1
TW_NONE, TW_EVENTS, TW_CASES_CONTAINED, TW_CASES_INTERSECTING = 0, 1, 2, 3
OPT_TIMING, OPT_TEST_HASH_BITS, OPT_TEST_BUCKET_CAP = 1, 2, 3
OPT_BATCH_CHUNK, OPT_BATCH_STAGES, OPT_BATCH_ITEMS_PER_SM = 4, 5, 6
OPT_EDGE_TABLE, OPT_LOAD_CLB, OPT_LOAD_SPLITS, OPT_STREAM_WARPS, OPT_STREAM_OFF = 7, 8, 9, 10, 11
OPT_PART1_ITEMS, OPT_PART2_ITEMS, OPT_PART_FBITS = 12, 13, 14
MAX_ACTIVITIES = 65536

_P = ctypes.c_void_p
_i32, _i64, _u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32


class _Alloc(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(_P, ctypes.c_size_t, _P, _P)),
                ("free", ctypes.CFUNCTYPE(None, _P, ctypes.c_size_t, _P, _P)),
                ("user", _P)]


class _Dfg(ctypes.Structure):
    _fields_ = [("n_edges", _i64), ("src", _P), ("dst", _P), ("count", _P)]


class _PerfDfg(ctypes.Structure):
    _fields_ = [("n_edges", _i64), ("src", _P), ("dst", _P), ("count", _P), ("sum_lo", _P),
                ("sum_hi", _P), ("min", _P), ("max", _P), ("mean", _P)]


class _Variants(ctypes.Structure):
    _fields_ = [("n_variants", _i64), ("n_out", _i64), ("count", _P), ("min_case", _P), ("off", _P),
                ("acts", _P), ("n_cases", _i64), ("case_ids", _P), ("case_variant", _P)]


class _FilterSpec(ctypes.Structure):
    _fields_ = [("attr_set", _P), ("n_attr", _i32), ("t_lo", _i64), ("t_hi", _i64), ("mode", _i32)]


class _CaseFilter(ctypes.Structure):
    _fields_ = [("min_events", _i64), ("max_events", _i64), ("min_duration", _i64), ("max_duration", _i64),
                ("start_set", _P), ("n_start", _i32), ("end_set", _P), ("n_end", _i32), ("act_set", _P),
                ("n_act", _i32), ("variant_set", _P), ("n_variant", _i32), ("exclude", _i32)]


class _Efg(ctypes.Structure):
    _fields_ = [("n_pairs", _i64)] + [(k, _P) for k in ("src", "dst", "count", "sum_lo", "sum_hi", "sq0", "sq1",
                                                          "sq2", "mean", "stdev")]


class _BatchSpec(ctypes.Structure):
    _fields_ = [("n_sub", _i32), ("attr_off", _P), ("attr_vals", _P), ("t_lo", _P), ("t_hi", _P),
                ("mode", _P), ("var_top_k", _i64)]


class _BatchDfg(ctypes.Structure):
    _fields_ = [("n_sub", _i32), ("n_activities", _i32), ("n_events", _P), ("n_cases", _P),
                ("edge_off", _P), ("src", _P), ("dst", _P), ("count", _P), ("sum_lo", _P), ("sum_hi", _P),
                ("min", _P), ("max", _P), ("mean", _P), ("start", _P), ("end", _P), ("freq", _P),
                ("n_variants", _P), ("var_off", _P), ("var_count", _P), ("var_min_case", _P),
                ("var_seq_off", _P), ("var_acts", _P), ("var_capacity", _i64), ("acts_capacity", _i64)]


LIBRARY = _build.LIB
if not os.path.exists(LIBRARY):
    raise ImportError(f"{LIBRARY} is missing: build it with `python -m paper_2204_04898_b300.build`")
lib = ctypes.CDLL(LIBRARY)

lib.pm4g_ctx_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.POINTER(_Alloc)]
lib.pm4g_ctx_destroy.argtypes = [_P]
lib.pm4g_ctx_set_option.argtypes = [_P, ctypes.c_int, _i64]
lib.pm4g_ctx_timing.argtypes = [_P, ctypes.c_char_p, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double)]
lib.pm4g_ctx_timing_reset.argtypes = [_P]
lib.pm4g_kernel_names.restype = ctypes.c_char_p
lib.pm4g_kernel_names.argtypes = []
lib.pm4g_load_log.argtypes = [_P, _P, _P, _P, _P, _i64, _i32, _u32, ctypes.POINTER(_P)]
lib.pm4g_log_info.argtypes = [_P, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
lib.pm4g_log_activities.argtypes = [_P, ctypes.POINTER(_i32)]
lib.pm4g_log_free.argtypes = [_P]
lib.pm4g_log_export.argtypes = [_P, _P, _P, _P, _P]
lib.pm4g_dfg.argtypes = [_P, ctypes.POINTER(_Dfg)]
lib.pm4g_dfg_free.argtypes = [ctypes.POINTER(_Dfg)]
lib.pm4g_perf_dfg.argtypes = [_P, ctypes.POINTER(_PerfDfg)]
lib.pm4g_perf_dfg_free.argtypes = [ctypes.POINTER(_PerfDfg)]
lib.pm4g_start_end.argtypes = [_P, _P, _P, _P]
lib.pm4g_variants.argtypes = [_P, _i64, _u32, ctypes.POINTER(_Variants)]
lib.pm4g_variants_free.argtypes = [ctypes.POINTER(_Variants)]
lib.pm4g_filter.argtypes = [_P, ctypes.POINTER(_FilterSpec), ctypes.POINTER(_P)]
lib.pm4g_filter_cases.argtypes = [_P, ctypes.POINTER(_CaseFilter), ctypes.POINTER(_P)]
lib.pm4g_efg.argtypes = [_P, ctypes.POINTER(_Efg)]
lib.pm4g_efg_free.argtypes = [ctypes.POINTER(_Efg)]
lib.pm4g_filter_paths.argtypes = [_P, _P, _P, _i32, _i32, ctypes.POINTER(_P)]
lib.pm4g_batch_dfg.argtypes = [_P, ctypes.POINTER(_BatchSpec), ctypes.POINTER(_BatchDfg)]
lib.pm4g_batch_dfg_free.argtypes = [ctypes.POINTER(_BatchDfg)]
lib.pm4g_batch_dfg_into.argtypes = [_P, ctypes.POINTER(_BatchSpec), ctypes.POINTER(_BatchDfg), _i64]
lib.pm4g_last_error.restype = ctypes.c_char_p
lib.pm4g_last_error.argtypes = []
lib.pm4g_dfg_noalloc.argtypes = [_P, _P, _P, _i64, _i32, _P] + [_P] * 7
lib.pm4g_dfg_noalloc_async.argtypes = [_P, _P, _P, _P, _i32, _P] + [_P] * 8


class Pm4gError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = lib.pm4g_last_error().decode(errors="replace")
        super().__init__(f"{what}: status {status}: {msg}")
        self.status = status


def _check(st: int, what: str) -> None:
    if st != OK:
        raise Pm4gError(st, what)


def _np(ptr, n, dtype):
    if n == 0:
        return np.empty(0, dtype=dtype)
    buf = (ctypes.c_char * (n * np.dtype(dtype).itemsize)).from_address(ptr)
    return np.frombuffer(buf, dtype=dtype).copy()


def pm4g_last_error() -> str:
    return lib.pm4g_last_error().decode(errors="replace")


def pm4g_kernel_names() -> list[str]:
    return lib.pm4g_kernel_names().decode().split(",")


def pm4g_ctx_create(device: int = 0, stream: int | None = None, allocator=None) -> int:
    """Create a context on `device`. `stream` is a raw cudaStream_t (e.g.
    torch.cuda.current_stream().cuda_stream) or None for a private stream.
    `allocator` is an optional (alloc(bytes, stream) -> ptr, free(ptr, bytes,
    stream)) pair of Python callables."""
    h = _P()
    a = None
    if allocator is not None:
        fa, ff = allocator
        a = _Alloc(_Alloc._fields_[0][1](lambda n, s, u: fa(int(n), s) or None),
                   _Alloc._fields_[1][1](lambda p, n, s, u: ff(p, int(n), s)), None)
    _check(lib.pm4g_ctx_create(ctypes.byref(h), device, stream, ctypes.byref(a) if a else None),
           "pm4g_ctx_create")
    if a is not None:
        _keepalive[h.value] = a
    return h.value


_keepalive: dict = {}


def pm4g_ctx_destroy(ctx: int) -> None:
    _check(lib.pm4g_ctx_destroy(ctx), "pm4g_ctx_destroy")
    _keepalive.pop(ctx, None)


def pm4g_ctx_set_option(ctx: int, option: int, value: int) -> None:
    _check(lib.pm4g_ctx_set_option(ctx, option, value), "pm4g_ctx_set_option")


def pm4g_ctx_timing(ctx: int, name: str) -> tuple[int, float]:
    n, ms = _i64(), ctypes.c_double()
    _check(lib.pm4g_ctx_timing(ctx, name.encode(), ctypes.byref(n), ctypes.byref(ms)), "pm4g_ctx_timing")
    return n.value, ms.value


def pm4g_ctx_timing_reset(ctx: int) -> None:
    _check(lib.pm4g_ctx_timing_reset(ctx), "pm4g_ctx_timing_reset")


def _column(x, dtype, name):
    """(pointer, n, is_device) of a 1-D contiguous column (torch tensor or numpy)."""
    if x is None:
        return None, None, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = {np.int32: torch.int32, np.int64: torch.int64}[dtype]
            if x.dtype != want or x.dim() != 1 or not x.is_contiguous():
                raise TypeError(f"{name}: need a contiguous 1-D {want} tensor")
            return x.data_ptr(), x.numel(), x.is_cuda
    except ImportError:
        pass
    a = np.asarray(x)
    if a.dtype != np.dtype(dtype) or a.ndim != 1 or not a.flags.c_contiguous:
        raise TypeError(f"{name}: need a contiguous 1-D {np.dtype(dtype)} array")
    return a.ctypes.data, a.shape[0], False


def pm4g_load_log(ctx: int, case_id, activity, ts_ns, case_attr=None, n_activities: int = 0) -> int:
    """Ingest and format a log. Columns are all torch CUDA tensors (device
    pointers) or all host arrays/tensors (copied by the library)."""
    pc, n, dc = _column(case_id, np.int32, "case_id")
    pa, na, da = _column(activity, np.int32, "activity")
    pt, nt, dt = _column(ts_ns, np.int64, "ts_ns")
    px, nx, dx = _column(case_attr, np.int32, "case_attr")
    if not (n == na == nt) or (px is not None and nx != n):
        raise ValueError("columns differ in length")
    devs = {dc, da, dt} | ({dx} if px is not None else set())
    if len(devs) != 1:
        raise ValueError("columns must all live on the device or all on the host")
    flags = DEVICE_PTRS if dc else HOST_PTRS
    h = _P()
    _check(lib.pm4g_load_log(ctx, pc, pa, pt, px, n, n_activities, flags, ctypes.byref(h)), "pm4g_load_log")
    return h.value


def pm4g_log_info(log: int) -> tuple[int, int]:
    ne, nc = _i64(), _i64()
    _check(lib.pm4g_log_info(log, ctypes.byref(ne), ctypes.byref(nc)), "pm4g_log_info")
    return ne.value, nc.value


def pm4g_log_activities(log: int) -> int:
    a = _i32()
    _check(lib.pm4g_log_activities(log, ctypes.byref(a)), "pm4g_log_activities")
    return a.value


def pm4g_log_free(log: int) -> None:
    _check(lib.pm4g_log_free(log), "pm4g_log_free")


def pm4g_log_export(log: int) -> dict:
    """The formatted log: every event in (case, timestamp, row) order."""
    n, _ = pm4g_log_info(log)
    out = {"case_id": np.empty(n, np.int32), "activity": np.empty(n, np.int32),
           "ts_ns": np.empty(n, np.int64), "row": np.empty(n, np.int64)}
    _check(lib.pm4g_log_export(log, *(out[k].ctypes.data for k in ("case_id", "activity", "ts_ns", "row"))),
           "pm4g_log_export")
    return out


@dataclass
class PerfDfg:
    src: np.ndarray
    dst: np.ndarray
    count: np.ndarray
    sum_lo: np.ndarray
    sum_hi: np.ndarray
    min: np.ndarray
    max: np.ndarray
    mean: np.ndarray

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])


def pm4g_dfg(log: int) -> dict:
    r = _Dfg()
    _check(lib.pm4g_dfg(log, ctypes.byref(r)), "pm4g_dfg")
    try:
        E = r.n_edges
        return {"src": _np(r.src, E, np.int32), "dst": _np(r.dst, E, np.int32),
                "count": _np(r.count, E, np.uint64)}
    finally:
        lib.pm4g_dfg_free(ctypes.byref(r))


def pm4g_perf_dfg(log: int) -> PerfDfg:
    r = _PerfDfg()
    _check(lib.pm4g_perf_dfg(log, ctypes.byref(r)), "pm4g_perf_dfg")
    try:
        E = r.n_edges
        u = np.uint64
        return PerfDfg(_np(r.src, E, np.int32), _np(r.dst, E, np.int32), _np(r.count, E, u),
                       _np(r.sum_lo, E, u), _np(r.sum_hi, E, u), _np(r.min, E, u), _np(r.max, E, u),
                       _np(r.mean, E, np.float64))
    finally:
        lib.pm4g_perf_dfg_free(ctypes.byref(r))


def pm4g_start_end(log: int, n_activities: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    s, e, f = (np.empty(n_activities, np.uint64) for _ in range(3))
    _check(lib.pm4g_start_end(log, s.ctypes.data, e.ctypes.data, f.ctypes.data), "pm4g_start_end")
    return s, e, f


@dataclass
class Variants:
    n_variants: int
    count: np.ndarray      # uint64[n_out]
    min_case: np.ndarray   # int32[n_out]
    off: np.ndarray        # int64[n_out+1]
    acts: np.ndarray       # int32
    case_ids: np.ndarray | None
    case_variant: np.ndarray | None


def pm4g_variants(log: int, top_k: int = -1, cases: bool = False) -> Variants:
    r = _Variants()
    _check(lib.pm4g_variants(log, top_k, VARIANTS_CASES if cases else 0, ctypes.byref(r)), "pm4g_variants")
    try:
        k = r.n_out
        off = _np(r.off, k + 1, np.int64)
        acts = _np(r.acts, int(off[-1]) if k else 0, np.int32)
        cids = _np(r.case_ids, r.n_cases, np.int32) if cases else None
        cvar = _np(r.case_variant, r.n_cases, np.int32) if cases else None
        return Variants(r.n_variants, _np(r.count, k, np.uint64), _np(r.min_case, k, np.int32), off, acts,
                        cids, cvar)
    finally:
        lib.pm4g_variants_free(ctypes.byref(r))


def pm4g_filter(log: int, attr_set=None, t_lo: int = -(2**63), t_hi: int = 2**63 - 1,
                mode: int = TW_NONE) -> int:
    aset = np.ascontiguousarray(np.asarray(attr_set if attr_set is not None else [], dtype=np.int32))
    spec = _FilterSpec(aset.ctypes.data if aset.size else None, int(aset.size), int(t_lo), int(t_hi), int(mode))
    h = _P()
    _check(lib.pm4g_filter(log, ctypes.byref(spec), ctypes.byref(h)), "pm4g_filter")
    return h.value


def pm4g_filter_paths(log: int, pairs, exclude: bool = False) -> int:
    """A new log of the events whose (previous activity in the case, activity)
    is one of `pairs` ((src, dst) activity codes), or with exclude the other
    events."""
    pr = np.asarray(pairs if len(pairs) else np.empty((0, 2)), dtype=np.int32).reshape(-1, 2)
    src, dst = np.ascontiguousarray(pr[:, 0]), np.ascontiguousarray(pr[:, 1])
    h = _P()
    _check(lib.pm4g_filter_paths(log, src.ctypes.data if src.size else None, dst.ctypes.data if dst.size else None,
                                 int(src.size), int(bool(exclude)), ctypes.byref(h)), "pm4g_filter_paths")
    return h.value


def pm4g_filter_cases(log: int, min_events: int = -1, max_events: int = -1, min_duration: int = -1,
                      max_duration: int = -1, start_set=(), end_set=(), act_set=(), variant_set=(),
                      exclude: bool = False) -> int:
    """A new log of the cases that meet every given criterion (bounds
    inclusive, negative = absent; empty set = absent; variant ids are the ranks
    of pm4g_variants), or with exclude the other cases."""
    sets = [np.ascontiguousarray(np.asarray(x, dtype=np.int32).ravel()) for x in (start_set, end_set, act_set,
                                                                                  variant_set)]
    ptr = [x.ctypes.data if x.size else None for x in sets]
    spec = _CaseFilter(int(min_events), int(max_events), int(min_duration), int(max_duration), ptr[0],
                       int(sets[0].size), ptr[1], int(sets[1].size), ptr[2], int(sets[2].size), ptr[3],
                       int(sets[3].size), int(bool(exclude)))
    h = _P()
    _check(lib.pm4g_filter_cases(log, ctypes.byref(spec), ctypes.byref(h)), "pm4g_filter_cases")
    return h.value


@dataclass
class Efg:
    """Eventually-follows graph and temporal profile, pairs ascending by
    (src, dst): counts, exact sums (sum_lo/sum_hi), exact sums of squares
    (sq0 low word .. sq2), means and population standard deviations."""
    src: np.ndarray
    dst: np.ndarray
    count: np.ndarray
    sum_lo: np.ndarray
    sum_hi: np.ndarray
    sq0: np.ndarray
    sq1: np.ndarray
    sq2: np.ndarray
    mean: np.ndarray
    stdev: np.ndarray


def pm4g_efg(log: int) -> Efg:
    r = _Efg()
    _check(lib.pm4g_efg(log, ctypes.byref(r)), "pm4g_efg")
    try:
        P = int(r.n_pairs)
        u = np.uint64
        return Efg(_np(r.src, P, np.int32), _np(r.dst, P, np.int32), _np(r.count, P, u), _np(r.sum_lo, P, u),
                   _np(r.sum_hi, P, u), _np(r.sq0, P, u), _np(r.sq1, P, u), _np(r.sq2, P, u),
                   _np(r.mean, P, np.float64), _np(r.stdev, P, np.float64))
    finally:
        lib.pm4g_efg_free(ctypes.byref(r))


@dataclass
class BatchDfg:
    """Per-sub-log results of pm4g_batch_dfg; sub-log i's edges are rows
    edge_off[i]:edge_off[i+1] of the edge arrays."""
    n_events: np.ndarray   # int64[Q]
    n_cases: np.ndarray    # int64[Q]
    edge_off: np.ndarray   # int64[Q+1]
    src: np.ndarray
    dst: np.ndarray
    count: np.ndarray
    sum_lo: np.ndarray
    sum_hi: np.ndarray
    min: np.ndarray
    max: np.ndarray
    mean: np.ndarray
    start: np.ndarray      # uint64[Q, A]
    end: np.ndarray
    freq: np.ndarray
    n_variants: np.ndarray | None = None   # int64[Q] (with variants)
    var_off: np.ndarray | None = None      # int64[Q+1]
    var_count: np.ndarray | None = None
    var_min_case: np.ndarray | None = None
    var_seq_off: np.ndarray | None = None  # int64[rows+1]
    var_acts: np.ndarray | None = None

    def sub(self, i: int) -> dict:
        a, b = int(self.edge_off[i]), int(self.edge_off[i + 1])
        return {k: getattr(self, k)[a:b] for k in ("src", "dst", "count", "sum_lo", "sum_hi", "min", "max", "mean")}

    def sub_variants(self, i: int) -> tuple[np.ndarray, np.ndarray, list]:
        """(counts, smallest case ids, sequences) of sub-log i's returned variants."""
        a, b = int(self.var_off[i]), int(self.var_off[i + 1])
        so = self.var_seq_off
        seqs = [tuple(int(x) for x in self.var_acts[so[r]:so[r + 1]]) for r in range(a, b)]
        return self.var_count[a:b], self.var_min_case[a:b], seqs


class BatchBuffers:
    """Reusable host arrays for pm4g_batch_dfg_into, page-locked through torch
    when it is available (then the device writes them directly). Results
    returned with these buffers are views, valid until their next use."""

    def __init__(self, n_sub: int = 0, n_act: int = 0, edges: int = 0, var_rows: int = 0, var_acts: int = 0):
        self.n_sub = self.n_act = self.edges = self.var_rows = self.var_acts_cap = -1
        self.ensure(n_sub, n_act, edges, var_rows, var_acts)

    @staticmethod
    def _alloc(n, dtype):
        try:
            import torch
            tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint64: torch.uint64,
                   np.float64: torch.float64}[dtype]
            return torch.empty(max(n, 1), dtype=tdt, pin_memory=torch.cuda.is_available()).numpy()
        except (ImportError, KeyError):
            return np.empty(max(n, 1), dtype)

    def ensure(self, n_sub: int, n_act: int, edges: int, var_rows: int = 0, var_acts: int = 0) -> None:
        # every array grows to at least twice its size (page-locking new host
        # memory takes milliseconds per megabyte, so a server that sees ever
        # larger batches reallocates a few times only)
        if n_sub > self.n_sub or n_act > self.n_act or n_sub * n_act > max(self.n_sub, 0) * max(self.n_act, 0):
            self.n_sub = max(n_sub, 2 * self.n_sub) if n_sub > self.n_sub else self.n_sub
            self.n_act = max(n_act, self.n_act)
            q, qa = self.n_sub, self.n_sub * self.n_act
            self.n_events, self.n_cases = self._alloc(q, np.int64), self._alloc(q, np.int64)
            self.edge_off = self._alloc(q + 1, np.int64)
            self.start, self.end, self.freq = (self._alloc(qa, np.uint64) for _ in range(3))
            self.n_variants, self.var_off = self._alloc(q, np.int64), self._alloc(q + 1, np.int64)
        if var_rows > self.var_rows:
            self.var_rows = max(int(var_rows * 1.25), 2 * self.var_rows) + 1024
            self.var_count = self._alloc(self.var_rows, np.uint64)
            self.var_min_case = self._alloc(self.var_rows, np.int32)
            self.var_seq_off = self._alloc(self.var_rows + 1, np.int64)
        if var_acts > self.var_acts_cap:
            self.var_acts_cap = max(int(var_acts * 1.25), 2 * self.var_acts_cap) + 4096
            self.var_acts = self._alloc(self.var_acts_cap, np.int32)
        if edges > self.edges:
            self.edges = max(int(edges * 1.25), 2 * self.edges) + 1024
            e = self.edges
            self.src, self.dst = self._alloc(e, np.int32), self._alloc(e, np.int32)
            (self.count, self.sum_lo, self.sum_hi, self.min,
             self.max) = (self._alloc(e, np.uint64) for _ in range(5))
            self.mean = self._alloc(e, np.float64)


class BatchSpec:
    """The views of a batch as the flat arrays of pm4g_batch_spec (attribute
    lists in CSR form, windows, modes); build once and pass to pm4g_batch_dfg
    as many times as needed."""

    def __init__(self, attr_sets, t_lo, t_hi, modes):
        self.Q = Q = len(t_lo)
        sets = [np.asarray(x if x is not None else [], np.int32).ravel() for x in attr_sets]
        if len(sets) != Q or len(t_hi) != Q or len(modes) != Q:
            raise ValueError("spec lists differ in length")
        self.off = np.zeros(Q + 1, np.int64)
        self.off[1:] = np.cumsum([x.size for x in sets])
        self.vals = np.ascontiguousarray(np.concatenate(sets) if Q else np.empty(0, np.int32), np.int32)
        self.tl = np.ascontiguousarray(t_lo, np.int64)
        self.th = np.ascontiguousarray(t_hi, np.int64)
        self.md = np.ascontiguousarray(modes, np.int32)

    def struct(self, var_top_k: int) -> _BatchSpec:
        return _BatchSpec(self.Q, self.off.ctypes.data, self.vals.ctypes.data if self.vals.size else None,
                          self.tl.ctypes.data, self.th.ctypes.data, self.md.ctypes.data, int(var_top_k))


def pm4g_batch_dfg(log: int, attr_sets=None, t_lo=None, t_hi=None, modes=None, out: BatchBuffers | None = None,
                   var_top_k: int = 0, spec: BatchSpec | None = None) -> BatchDfg:
    """Batched drill-down: sub-log i keeps the cases whose attribute is in
    attr_sets[i] (empty or None: all) and applies window [t_lo[i], t_hi[i]]
    with mode modes[i] (or the views of a prepared `spec`); var_top_k != 0 adds
    each sub-log's variants (< 0: all). With `out`, results are written into
    those reusable buffers (pm4g_batch_dfg_into) and returned as views of them."""
    bs = spec if spec is not None else BatchSpec(attr_sets, t_lo, t_hi, modes)
    Q = bs.Q
    spec = bs.struct(var_top_k)
    if out is not None:
        return _batch_into(log, spec, Q, out, var_top_k)
    r = _BatchDfg()
    _check(lib.pm4g_batch_dfg(log, ctypes.byref(spec), ctypes.byref(r)), "pm4g_batch_dfg")
    try:
        A = r.n_activities
        eo = _np(r.edge_off, Q + 1, np.int64)
        E = int(eo[-1]) if Q else 0
        u = np.uint64
        B = BatchDfg(_np(r.n_events, Q, np.int64), _np(r.n_cases, Q, np.int64), eo,
                     _np(r.src, E, np.int32), _np(r.dst, E, np.int32), _np(r.count, E, u),
                     _np(r.sum_lo, E, u), _np(r.sum_hi, E, u), _np(r.min, E, u), _np(r.max, E, u),
                     _np(r.mean, E, np.float64), _np(r.start, Q * A, u).reshape(Q, A),
                     _np(r.end, Q * A, u).reshape(Q, A), _np(r.freq, Q * A, u).reshape(Q, A))
        if var_top_k:
            vo = _np(r.var_off, Q + 1, np.int64)
            rows = int(vo[-1]) if Q else 0
            so = _np(r.var_seq_off, rows + 1, np.int64)
            B.n_variants, B.var_off, B.var_seq_off = _np(r.n_variants, Q, np.int64), vo, so
            B.var_count, B.var_min_case = _np(r.var_count, rows, u), _np(r.var_min_case, rows, np.int32)
            B.var_acts = _np(r.var_acts, int(so[-1]), np.int32)
        return B
    finally:
        lib.pm4g_batch_dfg_free(ctypes.byref(r))


def pm4g_batch_dfg_into(log: int, attr_sets=None, t_lo=None, t_hi=None, modes=None, out: BatchBuffers = None,
                        var_top_k: int = 0, spec: BatchSpec | None = None) -> BatchDfg:
    """pm4g_batch_dfg into caller-owned reusable buffers."""
    return pm4g_batch_dfg(log, attr_sets, t_lo, t_hi, modes, out=out, var_top_k=var_top_k, spec=spec)


def _batch_into(log, spec, Q, out: BatchBuffers, var_top_k: int) -> BatchDfg:
    A = pm4g_log_activities(log)
    out.ensure(Q, A, 0, 1, 1)
    for _ in range(2):
        r = _BatchDfg(Q, A, *(x.ctypes.data for x in (out.n_events, out.n_cases, out.edge_off, out.src, out.dst,
                                                    out.count, out.sum_lo, out.sum_hi, out.min, out.max,
                                                    out.mean, out.start, out.end, out.freq, out.n_variants,
                                                    out.var_off, out.var_count, out.var_min_case,
                                                    out.var_seq_off, out.var_acts)),
                      out.var_rows, out.var_acts_cap)
        st = lib.pm4g_batch_dfg_into(log, ctypes.byref(spec), ctypes.byref(r), out.edges)
        if st == ERANGE:  # more than the buffers hold: grow to the reported sizes and run again
            out.ensure(Q, A, int(out.edge_off[Q]), int(out.var_off[Q]) if var_top_k else 0,
                       int(r.acts_capacity) if var_top_k else 0)
            continue
        _check(st, "pm4g_batch_dfg_into")
        E = int(out.edge_off[Q])
        B = BatchDfg(out.n_events[:Q], out.n_cases[:Q], out.edge_off[:Q + 1], out.src[:E], out.dst[:E],
                     out.count[:E], out.sum_lo[:E], out.sum_hi[:E], out.min[:E], out.max[:E], out.mean[:E],
                     out.start[:Q * A].reshape(Q, A), out.end[:Q * A].reshape(Q, A),
                     out.freq[:Q * A].reshape(Q, A))
        if var_top_k:
            rows = int(out.var_off[Q])
            B.n_variants, B.var_off = out.n_variants[:Q], out.var_off[:Q + 1]
            B.var_count, B.var_min_case = out.var_count[:rows], out.var_min_case[:rows]
            B.var_seq_off = out.var_seq_off[:rows + 1]
            B.var_acts = out.var_acts[:int(out.var_seq_off[rows])]
        return B
    raise Pm4gError(ERANGE, "pm4g_batch_dfg_into")


def pm4g_dfg_noalloc(case_id, activity, ts_ns, n_activities: int, stream: int | None = None) -> dict:
    """Allocation-free DFG of a small log, for callers that cannot allocate
    device memory at call time (graph capture, fixed-budget serving, foreign
    memory pools): the library call uses only its fixed internal scratch. The
    inputs are CUDA tensors; the dense outputs (count, sum_lo, sum_hi, min, max
    over n_activities^2 cells; start, end) are CUDA int64 tensors allocated
    here, on the caller's side, and filled by the call."""
    import torch
    for x in (case_id, activity, ts_ns):
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.is_contiguous() and x.dim() == 1):
            raise TypeError("pm4g_dfg_noalloc takes contiguous 1-D CUDA tensors")
    n = case_id.numel()
    if activity.numel() != n or ts_ns.numel() != n:
        raise ValueError("columns differ in length")
    A = int(n_activities)
    dev = case_id.device
    out = {k: torch.empty(A * A, dtype=torch.int64, device=dev) for k in ("count", "sum_lo", "sum_hi", "min", "max")}
    out["start"] = torch.empty(A, dtype=torch.int64, device=dev)
    out["end"] = torch.empty(A, dtype=torch.int64, device=dev)
    _check(lib.pm4g_dfg_noalloc(case_id.data_ptr(), activity.data_ptr(), ts_ns.data_ptr(), n, A, stream,
                                *(out[k].data_ptr() for k in ("count", "sum_lo", "sum_hi", "min", "max", "start",
                                                              "end"))),
           "pm4g_dfg_noalloc")
    return out


NOALLOC_MAX_EVENTS = 1 << 18


def pm4g_dfg_noalloc_async(case_id, activity, ts_ns, n_events_dev, n_activities: int, out: dict, status,
                           stream: int | None = None) -> None:
    """The capturable allocation-free DFG: enqueues the summary of the first
    *n_events_dev events of the CUDA tensors case_id/activity/ts_ns on
    `stream` into the caller's CUDA int64 tensors out[count, sum_lo, sum_hi,
    min, max, start, end] and the int32 CUDA tensor `status`; returns at once
    (no synchronisation, so it can be captured in a CUDA graph)."""
    _check(lib.pm4g_dfg_noalloc_async(case_id.data_ptr(), activity.data_ptr(), ts_ns.data_ptr(),
                                      n_events_dev.data_ptr(), int(n_activities), stream,
                                      *(out[k].data_ptr() for k in ("count", "sum_lo", "sum_hi", "min", "max",
                                                                    "start", "end")),
                                      status.data_ptr()), "pm4g_dfg_noalloc_async")


class NoallocGraph:
    """pm4g_dfg_noalloc_async captured once in a CUDA graph over static device
    buffers of NOALLOC_MAX_EVENTS events: run(case_id, activity, ts_ns) copies a
    log (host arrays or CUDA tensors, at most that many events) into the
    buffers, replays the graph and returns the dense outputs (count, sum_lo,
    sum_hi, min, max over n_activities^2 cells; start, end) as CUDA int64
    tensors owned by this object (valid until the next run) and the status
    word (see pm4g_dfg_noalloc_async). One replay is the whole summary: its
    launches go to the GPU as one graph."""

    def __init__(self, n_activities: int, device: int = 0):
        import torch
        self.A = A = int(n_activities)
        dev = torch.device("cuda", device)
        m = NOALLOC_MAX_EVENTS
        self.case_id = torch.zeros(m, dtype=torch.int32, device=dev)
        self.activity = torch.zeros(m, dtype=torch.int32, device=dev)
        self.ts_ns = torch.zeros(m, dtype=torch.int64, device=dev)
        self.n = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.out = {k: torch.empty(A * A, dtype=torch.int64, device=dev) for k in ("count", "sum_lo", "sum_hi", "min",
                                                                                   "max")}
        self.out["start"] = torch.empty(A, dtype=torch.int64, device=dev)
        self.out["end"] = torch.empty(A, dtype=torch.int64, device=dev)
        self.stream = torch.cuda.Stream(device=dev)
        def call(stream):
            pm4g_dfg_noalloc_async(self.case_id, self.activity, self.ts_ns, self.n, A, self.out, self.status, stream)

        with torch.cuda.stream(self.stream):
            call(self.stream.cuda_stream)  # the first call (outside capture) looks up the scratch array
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            call(self.stream.cuda_stream)

    def run(self, case_id, activity, ts_ns) -> tuple[dict, int]:
        import torch
        n = len(case_id)
        if n > NOALLOC_MAX_EVENTS or len(activity) != n or len(ts_ns) != n:
            raise ValueError("a log of at most NOALLOC_MAX_EVENTS events, columns of equal length")
        if any(isinstance(x, torch.Tensor) and x.is_cuda for x in (case_id, activity, ts_ns)):
            # device inputs may still be being written on the caller's stream
            self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            for dst, src in ((self.case_id, case_id), (self.activity, activity), (self.ts_ns, ts_ns)):
                dst[:n].copy_(torch.as_tensor(src), non_blocking=True)
            self.n.fill_(n)
            self.graph.replay()
        self.stream.synchronize()
        return self.out, int(self.status.item())
