"""CPU oracle for the process-mining summaries (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline``
leg may import this package. The engine in ``paper_2204_04898_b300`` never does,
and the two share no code.

``pm4g_oracle.cpp`` is a plain single-threaded C++17 statement of the
definitions in Section 3 of the paper (ordering by case, timestamp and row;
directly-follows pairs; performance aggregates; start/end activities; variants;
timestamp and attribute filters; paths and case filters; the eventually-follows
graph and temporal profile). This module compiles it with g++ and exposes
it through ctypes with numpy arrays.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "pm4g_oracle.cpp")
_LIB = os.path.join(_HERE, "libpm4g_oracle.so")

OK, EINVAL, ERANGE = 0, -1, -2
TW_NONE, TW_EVENTS, TW_CASES_CONTAINED, TW_CASES_INTERSECTING = 0, 1, 2, 3

_P = ctypes.c_void_p


def compile_library(source: str, out: str) -> str:
    """Compile an oracle source file into a shared library."""
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", source, "-o", out])
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(SOURCE):
        tmp = _LIB + f".{os.getpid()}.tmp"
        compile_library(SOURCE, tmp)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.oracle_summarize.restype = ctypes.c_int
    lib.oracle_summarize.argtypes = [_P, _P, _P, i64, i32, ctypes.POINTER(_P)]
    lib.oracle_free.argtypes = [_P]
    lib.oracle_free.restype = None
    for f in ("oracle_n_events", "oracle_n_cases", "oracle_n_edges", "oracle_n_variants",
              "oracle_n_variant_acts"):
        getattr(lib, f).restype = i64
        getattr(lib, f).argtypes = [_P]
    lib.oracle_sorted_rows.argtypes = [_P, _P]
    lib.oracle_edges.argtypes = [_P] * 9
    lib.oracle_endpoints.argtypes = [_P] * 4
    lib.oracle_variants.argtypes = [_P] * 5
    lib.oracle_cases.argtypes = [_P] * 4
    for f in ("oracle_sorted_rows", "oracle_edges", "oracle_endpoints", "oracle_variants",
              "oracle_cases"):
        getattr(lib, f).restype = None
    lib.oracle_filter.restype = i64
    lib.oracle_filter.argtypes = [_P, _P, _P, _P, i64, i32, _P, i32, i64, i64, i32, _P]
    lib.oracle_filter_paths.restype = i64
    lib.oracle_filter_paths.argtypes = [_P, _P, _P, i64, i32, _P, _P, i32, i32, _P]
    lib.oracle_efg.restype = _P
    lib.oracle_efg.argtypes = [_P, _P, _P, i64, i32, _P]
    lib.oracle_efg_pairs.restype = None
    lib.oracle_efg_pairs.argtypes = [_P] * 11
    lib.oracle_free_efg.restype = None
    lib.oracle_free_efg.argtypes = [_P]
    lib.oracle_filter_cases.restype = i64
    lib.oracle_filter_cases.argtypes = [_P, _P, _P, i64, i32, i64, i64, i64, i64, _P, i32, _P, i32, _P, i32, _P, i32,
                                        i32, _P]
    return lib


_lib = None


def load(path: str | None = None):
    """Load the oracle library (``path`` loads an alternative build, e.g. a
    deliberately mutated copy used to show that the pins catch mistakes)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status: int):
        super().__init__(f"oracle status {status}")
        self.status = status


@dataclass
class Summary:
    """Every output of the method for one log (Section 3)."""

    n_events: int
    n_activities: int
    sorted_rows: np.ndarray      # int64[N]: rows in (case, ts, row) order
    case_ids: np.ndarray         # int32[C], ascending
    case_len: np.ndarray         # int64[C]
    case_variant: np.ndarray     # int32[C]
    src: np.ndarray              # int32[E]
    dst: np.ndarray              # int32[E]
    count: np.ndarray            # uint64[E]
    sum_lo: np.ndarray           # uint64[E]
    sum_hi: np.ndarray           # uint64[E]
    min: np.ndarray              # uint64[E]
    max: np.ndarray              # uint64[E]
    mean: np.ndarray             # float64[E]
    start: np.ndarray            # uint64[A]
    end: np.ndarray              # uint64[A]
    freq: np.ndarray             # uint64[A]
    var_count: np.ndarray        # uint64[V]
    var_min_case: np.ndarray     # int32[V]
    var_off: np.ndarray          # int64[V+1]
    var_acts: np.ndarray         # int32[sum of lengths]

    @property
    def n_cases(self) -> int:
        return int(self.case_ids.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])

    @property
    def n_variants(self) -> int:
        return int(self.var_count.shape[0])

    def edge_sums(self) -> list[int]:
        """Exact per-edge duration sums as Python ints."""
        return [int(lo) + (int(hi) << 64) for lo, hi in zip(self.sum_lo, self.sum_hi)]

    def variant_seqs(self) -> list[tuple[int, ...]]:
        return [tuple(int(a) for a in self.var_acts[self.var_off[k]:self.var_off[k + 1]])
                for k in range(self.n_variants)]


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def summarize(case_id, activity, ts_ns, n_activities: int, lib=None) -> Summary:
    """Run the oracle on one log; raises OracleError on a bad status."""
    lib = lib or load()
    case_id, activity, ts_ns = _c(case_id, np.int32), _c(activity, np.int32), _c(ts_ns, np.int64)
    n = int(case_id.shape[0])
    if activity.shape[0] != n or ts_ns.shape[0] != n:
        raise ValueError("columns differ in length")
    h = _P()
    st = lib.oracle_summarize(_ptr(case_id), _ptr(activity), _ptr(ts_ns), n, int(n_activities),
                              ctypes.byref(h))
    if st != 0:
        raise OracleError(st)
    try:
        C, E, V = lib.oracle_n_cases(h), lib.oracle_n_edges(h), lib.oracle_n_variants(h)
        NA = lib.oracle_n_variant_acts(h)
        A = int(n_activities)
        rows = np.empty(n, np.int64)
        lib.oracle_sorted_rows(h, _ptr(rows))
        src, dst = np.empty(E, np.int32), np.empty(E, np.int32)
        cnt, slo, shi = np.empty(E, np.uint64), np.empty(E, np.uint64), np.empty(E, np.uint64)
        mn, mx, mean = np.empty(E, np.uint64), np.empty(E, np.uint64), np.empty(E, np.float64)
        lib.oracle_edges(h, *(_ptr(x) for x in (src, dst, cnt, slo, shi, mn, mx, mean)))
        st_, en_, fr_ = np.empty(A, np.uint64), np.empty(A, np.uint64), np.empty(A, np.uint64)
        lib.oracle_endpoints(h, _ptr(st_), _ptr(en_), _ptr(fr_))
        vc, vm = np.empty(V, np.uint64), np.empty(V, np.int32)
        vo, va = np.empty(V + 1, np.int64), np.empty(NA, np.int32)
        lib.oracle_variants(h, _ptr(vc), _ptr(vm), _ptr(vo), _ptr(va))
        cid, clen, cvar = np.empty(C, np.int32), np.empty(C, np.int64), np.empty(C, np.int32)
        lib.oracle_cases(h, _ptr(cid), _ptr(clen), _ptr(cvar))
    finally:
        lib.oracle_free(h)
    return Summary(n, A, rows, cid, clen, cvar, src, dst, cnt, slo, shi, mn, mx, mean,
                   st_, en_, fr_, vc, vm, vo, va)


def filter_rows(case_id, activity, ts_ns, case_attr, n_activities: int, attr_set, t_lo: int,
                t_hi: int, mode: int, lib=None) -> np.ndarray:
    """Rows (ascending) kept by the drill-down filter."""
    lib = lib or load()
    case_id, activity, ts_ns = _c(case_id, np.int32), _c(activity, np.int32), _c(ts_ns, np.int64)
    n = int(case_id.shape[0])
    attr_set = _c(attr_set if attr_set is not None else [], np.int32)
    attr = None if case_attr is None else _c(case_attr, np.int32)
    out = np.empty(max(n, 1), np.int64)
    m = lib.oracle_filter(_ptr(case_id), _ptr(activity), _ptr(ts_ns), _ptr(attr), n,
                          int(n_activities), _ptr(attr_set), int(attr_set.shape[0]), int(t_lo),
                          int(t_hi), int(mode), _ptr(out))
    if m < 0:
        raise OracleError(int(m))
    return out[:m].copy()


def filter_paths(case_id, activity, ts_ns, n_activities: int, pairs, exclude: bool = False,
                 lib=None) -> np.ndarray:
    """Rows (ascending) kept by the paths filter: events whose (previous
    activity in the case, activity) is one of `pairs` (or, with exclude, the
    other events)."""
    lib = lib or load()
    case_id, activity, ts_ns = _c(case_id, np.int32), _c(activity, np.int32), _c(ts_ns, np.int64)
    n = int(case_id.shape[0])
    pr = np.asarray(pairs, np.int32).reshape(-1, 2)
    src, dst = _c(pr[:, 0], np.int32), _c(pr[:, 1], np.int32)
    out = np.empty(max(n, 1), np.int64)
    m = lib.oracle_filter_paths(_ptr(case_id), _ptr(activity), _ptr(ts_ns), n, int(n_activities), _ptr(src),
                                _ptr(dst), int(pr.shape[0]), int(bool(exclude)), _ptr(out))
    if m < 0:
        raise OracleError(int(m))
    return out[:m].copy()


def filter_cases(case_id, activity, ts_ns, n_activities: int, min_events: int = -1, max_events: int = -1,
                 min_duration: int = -1, max_duration: int = -1, start_set=(), end_set=(), act_set=(),
                 variant_set=(), exclude: bool = False, lib=None) -> np.ndarray:
    """Rows (ascending) kept by the case filters (bounds inclusive, negative =
    absent; empty set = absent; variant ids are ranks)."""
    lib = lib or load()
    case_id, activity, ts_ns = _c(case_id, np.int32), _c(activity, np.int32), _c(ts_ns, np.int64)
    n = int(case_id.shape[0])
    sets = [_c(np.asarray(x, np.int32).ravel(), np.int32) for x in (start_set, end_set, act_set, variant_set)]
    out = np.empty(max(n, 1), np.int64)
    args = []
    for x in sets:
        args += [_ptr(x), int(x.shape[0])]
    m = lib.oracle_filter_cases(_ptr(case_id), _ptr(activity), _ptr(ts_ns), n, int(n_activities), int(min_events),
                                int(max_events), int(min_duration), int(max_duration), *args, int(bool(exclude)),
                                _ptr(out))
    if m < 0:
        raise OracleError(int(m))
    return out[:m].copy()


@dataclass
class Efg:
    """Eventually-follows graph and temporal profile, pairs ascending by (a, b)."""

    src: np.ndarray      # int32[P]
    dst: np.ndarray      # int32[P]
    count: np.ndarray    # uint64[P]
    sum_lo: np.ndarray   # uint64[P]
    sum_hi: np.ndarray   # uint64[P]
    sq0: np.ndarray      # uint64[P]: sum of squares, low word
    sq1: np.ndarray      # uint64[P]
    sq2: np.ndarray      # uint64[P]: high word
    mean: np.ndarray     # float64[P]
    stdev: np.ndarray    # float64[P]

    def sums(self) -> list[int]:
        return [int(lo) | (int(hi) << 64) for lo, hi in zip(self.sum_lo, self.sum_hi)]

    def squares(self) -> list[int]:
        return [int(a) | (int(b) << 64) | (int(c) << 128) for a, b, c in zip(self.sq0, self.sq1, self.sq2)]


def efg(case_id, activity, ts_ns, n_activities: int, lib=None) -> Efg:
    """Eventually-follows graph and temporal profile of a log."""
    lib = lib or load()
    case_id, activity, ts_ns = _c(case_id, np.int32), _c(activity, np.int32), _c(ts_ns, np.int64)
    n = int(case_id.shape[0])
    P = ctypes.c_int64()
    h = lib.oracle_efg(_ptr(case_id), _ptr(activity), _ptr(ts_ns), n, int(n_activities), ctypes.byref(P))
    if not h:
        raise OracleError(EINVAL)
    try:
        m = int(P.value)
        i32 = [np.empty(max(m, 1), np.int32) for _ in range(2)]
        u64 = [np.empty(max(m, 1), np.uint64) for _ in range(6)]
        f64 = [np.empty(max(m, 1), np.float64) for _ in range(2)]
        lib.oracle_efg_pairs(h, *[_ptr(x) for x in i32 + u64 + f64])
        return Efg(*[x[:m].copy() for x in i32 + u64 + f64])
    finally:
        lib.oracle_free_efg(h)


def mutant_library(replace_from: str, replace_to: str, count: int = 1) -> str:
    """Compile a copy of the oracle with one textual change (a planted mistake)
    and return the library path. Used only by the tests that show the pins
    catch plausible mistakes."""
    with open(SOURCE) as f:
        src = f.read()
    if src.count(replace_from) < count:
        raise ValueError(f"pattern not found: {replace_from!r}")
    src = src.replace(replace_from, replace_to, count)
    d = tempfile.mkdtemp(prefix="pm4g_mutant_")
    path = os.path.join(d, "mutant.cpp")
    with open(path, "w") as f:
        f.write(src)
    return compile_library(path, os.path.join(d, "libmutant.so"))
