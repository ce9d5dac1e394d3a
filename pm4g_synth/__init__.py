"""Seeded synthetic event logs shaped like the paper's workloads.

The paper measures on the Road Traffic Fine, BPI Challenge 2019 and BPI
Challenge 2018 logs with replicated cases (Section 4, Table 1). Those logs are
not available here; these generators stand in for their shapes (tens of
activities, 4 to 57 events per case, case-level repetition of variants) and push
them to larger sizes.

This module draws inputs only. It holds none of the summaries' arithmetic, and
both the CPU oracle and the CUDA engine consume its output unchanged.

Workloads (seed of workload k is 20220411 + k):

1. ``single_log``: 10,000 cases, geometric lengths (mean 10), 10 activities
   from a Markov chain with Dirichlet(0.5) rows, exponential gaps (mean 1 h),
   rows shuffled.
2. ``large_log``: 1M cases, lognormal lengths (median 15, sigma 0.8, cap 500),
   50 activities with Zipf(1.1) frequencies and 20 % restart noise, Pareto(1.5)
   gaps with 5 % zero gaps, rows shuffled.
3. ``very_large_log``: 10M cases, lognormal lengths as above (~206M events),
   500 activities (Zipf 1.0) from a sparse chain with at most 12 successors,
   Pareto gaps, rows sorted by timestamp only.
4. ``drilldown_log``: workload-3 law with 2,000 activities, about 100M events,
   a uniform int32 case attribute in [0, 4096), plus 4,096 drill-down specs.
5. ``serving_log``: the workload-3 law (device-resident log for serving).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.cpp")
_LIB = os.path.join(_HERE, "libpm4g_synth.so")

LEN_GEOMETRIC, LEN_LOGNORMAL, LEN_FIXED = 0, 1, 2
ACT_DIRICHLET_MARKOV, ACT_ZIPF_RESTART, ACT_SPARSE_CHAIN = 0, 1, 2
GAP_EXPONENTIAL, GAP_PARETO = 0, 1
ROWS_SHUFFLED, ROWS_TS_SORTED, ROWS_CASE_ORDER = 0, 1, 2

NS_PER_MIN = 60 * 10**9
NS_PER_HOUR = 3600 * 10**9
NS_PER_DAY = 86400 * 10**9
BASE_SEED = 20220411


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_cases", ctypes.c_int64),
        ("n_activities", ctypes.c_int32),
        ("len_law", ctypes.c_int32),
        ("len_p", ctypes.c_double),
        ("len_median", ctypes.c_double),
        ("len_sigma", ctypes.c_double),
        ("len_cap", ctypes.c_int32),
        ("act_model", ctypes.c_int32),
        ("dirichlet_alpha", ctypes.c_double),
        ("zipf_s", ctypes.c_double),
        ("restart_p", ctypes.c_double),
        ("max_succ", ctypes.c_int32),
        ("gap_law", ctypes.c_int32),
        ("gap_mean_ns", ctypes.c_double),
        ("pareto_alpha", ctypes.c_double),
        ("pareto_xm_ns", ctypes.c_double),
        ("p_zero_gap", ctypes.c_double),
        ("gap_cap_ns", ctypes.c_double),
        ("start_span_ns", ctypes.c_double),
        ("row_order", ctypes.c_int32),
        ("n_attr_values", ctypes.c_int32),
        ("n_threads", ctypes.c_int32),
    ]


@dataclass(frozen=True)
class LogSpec:
    """Parameters of one synthetic log (all lengths in events, times in ns)."""

    name: str
    seed: int
    n_cases: int
    n_activities: int
    len_law: int = LEN_LOGNORMAL
    len_p: float = 0.1
    len_median: float = 15.0
    len_sigma: float = 0.8
    len_cap: int = 500
    act_model: int = ACT_SPARSE_CHAIN
    dirichlet_alpha: float = 0.5
    zipf_s: float = 1.0
    restart_p: float = 0.0
    max_succ: int = 12
    gap_law: int = GAP_PARETO
    gap_mean_ns: float = float(NS_PER_HOUR)
    pareto_alpha: float = 1.5
    pareto_xm_ns: float = float(20 * NS_PER_MIN)
    p_zero_gap: float = 0.05
    # One gap is clamped to 2^52 ns (~52 days): it touches about 4 in a million
    # Pareto draws and keeps every timestamp far below 2^63.
    gap_cap_ns: float = float(2**52)
    start_span_ns: float = float(365 * NS_PER_DAY)
    row_order: int = ROWS_SHUFFLED
    n_attr_values: int = 0
    extra: dict = field(default_factory=dict, compare=False)

    def scaled(self, n_cases: int, name: str | None = None) -> "LogSpec":
        return replace(self, n_cases=int(n_cases), name=name or f"{self.name}@{n_cases}")


def single_log(n_cases: int = 10_000) -> LogSpec:
    return LogSpec(
        name="single_log", seed=BASE_SEED + 1, n_cases=n_cases, n_activities=10,
        len_law=LEN_GEOMETRIC, len_p=0.1, len_cap=1 << 30,
        act_model=ACT_DIRICHLET_MARKOV, dirichlet_alpha=0.5,
        gap_law=GAP_EXPONENTIAL, gap_mean_ns=float(NS_PER_HOUR), p_zero_gap=0.0,
        row_order=ROWS_SHUFFLED)


def large_log(n_cases: int = 1_000_000) -> LogSpec:
    return LogSpec(
        name="large_log", seed=BASE_SEED + 2, n_cases=n_cases, n_activities=50,
        act_model=ACT_ZIPF_RESTART, zipf_s=1.1, restart_p=0.2, dirichlet_alpha=0.5,
        row_order=ROWS_SHUFFLED)


def very_large_log(n_cases: int = 10_000_000) -> LogSpec:
    return LogSpec(
        name="very_large_log", seed=BASE_SEED + 3, n_cases=n_cases, n_activities=500,
        act_model=ACT_SPARSE_CHAIN, zipf_s=1.0, max_succ=12,
        row_order=ROWS_TS_SORTED)


def drilldown_log(n_cases: int = 4_850_000) -> LogSpec:
    return LogSpec(
        name="drilldown_log", seed=BASE_SEED + 4, n_cases=n_cases, n_activities=2000,
        act_model=ACT_SPARSE_CHAIN, zipf_s=1.0, max_succ=12,
        row_order=ROWS_TS_SORTED, n_attr_values=4096)


def serving_log(n_cases: int = 10_000_000) -> LogSpec:
    """Workload-3 law with its own seed and a uniform case attribute in
    [0, 4096), for filter(attribute set, window) requests."""
    return replace(very_large_log(n_cases), name="serving_log", seed=BASE_SEED + 5, n_attr_values=4096)


WORKLOADS = {
    "single_log": single_log,
    "large_log": large_log,
    "very_large_log": very_large_log,
    "drilldown_log": drilldown_log,
    "serving_log": serving_log,
}


def build(force: bool = False) -> str:
    """Compile the generator library in place (seconds)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", _LIB + ".tmp"])
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.synth_count.restype = ctypes.c_int64
        _lib.synth_count.argtypes = [ctypes.POINTER(_Params)]
        _lib.synth_fill.restype = ctypes.c_int64
        _lib.synth_fill.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
    return _lib


def _params(spec: LogSpec, n_threads: int) -> _Params:
    p = _Params()
    for name, _ in _Params._fields_:
        if name == "n_threads":
            p.n_threads = n_threads
        else:
            setattr(p, name, getattr(spec, name))
    return p


@dataclass
class EventLog:
    """Columnar event log: one row per event, in input-row order."""

    case_id: np.ndarray   # int32[N]
    activity: np.ndarray  # int32[N]
    ts_ns: np.ndarray     # int64[N]
    case_attr: np.ndarray | None  # int32[N] or None
    n_activities: int
    spec: LogSpec | None = None

    @property
    def n_events(self) -> int:
        return int(self.case_id.shape[0])

    def take(self, rows: np.ndarray) -> "EventLog":
        rows = np.asarray(rows, dtype=np.int64)
        return EventLog(self.case_id[rows], self.activity[rows], self.ts_ns[rows],
                        None if self.case_attr is None else self.case_attr[rows],
                        self.n_activities, self.spec)


def generate(spec: LogSpec, n_threads: int = 0, pinned: bool = False) -> EventLog:
    """Draw the log described by ``spec``.

    With ``pinned=True`` the columns live in page-locked host memory (torch
    pinned tensors viewed as numpy), ready for asynchronous host-to-device copies.
    """
    lib = _load()
    p = _params(spec, n_threads)
    n = lib.synth_count(ctypes.byref(p))
    if n < 0:
        raise ValueError(f"bad log spec {spec}")

    def alloc(dtype):
        if pinned:
            import torch
            tdt = {np.int32: torch.int32, np.int64: torch.int64}[dtype]
            return torch.empty(n, dtype=tdt, pin_memory=True).numpy()
        return np.empty(n, dtype=dtype)

    case_id, act, ts = alloc(np.int32), alloc(np.int32), alloc(np.int64)
    attr = alloc(np.int32) if spec.n_attr_values > 0 else None
    got = lib.synth_fill(ctypes.byref(p), case_id.ctypes.data, act.ctypes.data, ts.ctypes.data,
                         None if attr is None else attr.ctypes.data)
    if got != n:
        raise RuntimeError("generator failed")
    return EventLog(case_id, act, ts, attr, spec.n_activities, spec)


@dataclass(frozen=True)
class DrilldownSpec:
    """One drill-down view: a case-attribute set and a closed time window."""

    attr_set: np.ndarray  # int32[k]
    t_lo: int
    t_hi: int
    target_events: int


def drilldown_specs(log: EventLog, n_views: int = 4096, seed: int = BASE_SEED + 4,
                    lo_events: float = 1e3, hi_events: float = 1e6,
                    n_attr_values: int = 4096) -> list[DrilldownSpec]:
    """Drill-down views over ``log``: view i targets s_i ~ LogUniform(lo, hi)
    events, takes a window covering a fraction f_i ~ U(0.25, 1) of the log's time
    span at a uniform offset, and a set of k_i = clamp(round(s_i*V/(N*f_i)), 1, V)
    attribute values drawn without replacement (V attribute values)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t0, t1 = int(log.ts_ns.min()), int(log.ts_ns.max())
    span = t1 - t0
    out = []
    for _ in range(n_views):
        s = float(np.exp(rng.uniform(np.log(lo_events), np.log(hi_events))))
        f = float(rng.uniform(0.25, 1.0))
        off = float(rng.uniform(0.0, 1.0 - f))
        lo = t0 + int(off * span)
        hi = lo + int(f * span)
        k = int(min(max(round(s * n_attr_values / (max(1, log.n_events) * f)), 1), n_attr_values))
        attrs = np.sort(rng.choice(n_attr_values, size=k, replace=False)).astype(np.int32)
        out.append(DrilldownSpec(attrs, lo, hi, int(s)))
    return out
