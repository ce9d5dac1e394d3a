"""Whole-log results checked against the oracle run on groups of cases.

Every output of the method is a sum over cases (edge counts, exact duration
sums and sums of squares, start, end and activity counts), an extreme over
cases (edge minimum and maximum), or a per-case value (the formatted order of
a case's events, the variant of a case). Split the cases of a log into
disjoint groups and the oracle's results on the groups fix the whole log's
result: sums add, extremes combine, per-case values carry over, and the means
and deviations follow from the summed exact moments by their definitions
(formed once in FP64 from the exact integers, each conversion and operation
correctly rounded: the performance DFG of Section 3 and the temporal profile
of the eventually-follows graph). This lets the oracle check logs it could not
summarise whole within a test: the groups run in parallel threads (the oracle
is a C library, called through ctypes without the interpreter lock).

The variant table is checked per case (each case's sequence under the
engine's rank equals its sequence under the oracle) and as a table (counts
and smallest cases follow from the per-case ranks, the ranking order holds,
and no two ranks share a sequence), which together fix it.
"""

from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass
from types import SimpleNamespace

import numpy as np

import oracle

U64_MAX = np.iinfo(np.uint64).max


def workers() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def pool_map(fn, items):
    with ThreadPoolExecutor(max_workers=workers()) as ex:
        return list(ex.map(fn, items))


def case_groups(case_id: np.ndarray, G: int):
    """Rows of each group of cases (case id mod G), ascending within a group:
    group g's rows are order[bounds[g]:bounds[g + 1]]."""
    assert 1 <= G <= 256
    key = np.remainder(case_id, G).astype(np.uint8)
    order = np.argsort(key, kind="stable")
    bounds = np.zeros(G + 1, np.int64)
    bounds[1:] = np.cumsum(np.bincount(key, minlength=G))
    return order, bounds


def ranges(starts, lens) -> np.ndarray:
    """Flat indices of the ranges [starts[i], starts[i] + lens[i])."""
    starts = np.asarray(starts, np.int64)
    lens = np.asarray(lens, np.int64)
    total = int(lens.sum())
    if total == 0:
        return np.empty(0, np.int64)
    first = np.cumsum(lens) - lens
    return np.repeat(starts - first, lens) + np.arange(total, dtype=np.int64)


def _add_words(words, k, parts):
    """words[j][k] += parts[j] as one multiword unsigned integer (low word first)."""
    carry = np.zeros(k.shape[0], np.uint64)
    for w, x in zip(words, parts):
        old = w[k]
        s = old + x
        c1 = s < old
        s2 = s + carry
        c2 = s2 < s
        w[k] = s2
        carry = (c1 | c2).astype(np.uint64)
    assert not carry.any(), "multiword sum overflowed its top word"


def _mean_bits(count, lo, hi) -> np.ndarray:
    return np.array([float(int(l) | (int(h) << 64)) / float(int(c)) for c, l, h in zip(count, lo, hi)],
                    np.float64).view(np.uint64)


@dataclass
class GroupDfg:
    """The parts of one group's summary that add up to the whole log's."""
    src: np.ndarray
    dst: np.ndarray
    count: np.ndarray
    sum_lo: np.ndarray
    sum_hi: np.ndarray
    min: np.ndarray
    max: np.ndarray
    start: np.ndarray
    end: np.ndarray
    freq: np.ndarray
    n_events: int
    n_cases: int

    @staticmethod
    def of(R: oracle.Summary) -> "GroupDfg":
        return GroupDfg(R.src, R.dst, R.count, R.sum_lo, R.sum_hi, R.min, R.max, R.start, R.end, R.freq,
                        R.n_events, R.n_cases)


class DfgSum:
    """Performance DFG and endpoint counts of a union of disjoint case groups,
    on a dense |A| x |A| grid."""

    def __init__(self, A: int):
        self.A = A
        cells = A * A
        self.cnt = np.zeros(cells, np.uint64)
        self.lo = np.zeros(cells, np.uint64)
        self.hi = np.zeros(cells, np.uint64)
        self.mn = np.full(cells, U64_MAX, np.uint64)
        self.mx = np.zeros(cells, np.uint64)
        self.start = np.zeros(A, np.uint64)
        self.end = np.zeros(A, np.uint64)
        self.freq = np.zeros(A, np.uint64)
        self.n_events = 0
        self.n_cases = 0

    def add(self, g: GroupDfg) -> None:
        k = g.src.astype(np.int64) * self.A + g.dst
        assert np.unique(k).shape[0] == k.shape[0]
        self.cnt[k] += g.count
        _add_words((self.lo, self.hi), k, (g.sum_lo, g.sum_hi))
        self.mn[k] = np.minimum(self.mn[k], g.min)
        self.mx[k] = np.maximum(self.mx[k], g.max)
        self.start += g.start
        self.end += g.end
        self.freq += g.freq
        self.n_events += int(g.n_events)
        self.n_cases += int(g.n_cases)

    def edges(self) -> dict:
        k = np.flatnonzero(self.cnt)
        e = {"src": (k // self.A).astype(np.int32), "dst": (k % self.A).astype(np.int32), "count": self.cnt[k],
             "sum_lo": self.lo[k], "sum_hi": self.hi[k], "min": self.mn[k], "max": self.mx[k]}
        e["mean_bits"] = _mean_bits(e["count"], e["sum_lo"], e["sum_hi"])
        return e

    def assert_equal(self, perf, start, end, freq, n_events=None, n_cases=None, what="") -> None:
        """Bit-exact comparison with a whole-log result (PerfDfg or oracle.Summary fields)."""
        e = self.edges()
        for name in ("src", "dst", "count", "sum_lo", "sum_hi", "min", "max"):
            assert np.array_equal(np.asarray(getattr(perf, name)), e[name]), f"{what}{name} differs"
        assert np.array_equal(np.asarray(perf.mean).view(np.uint64), e["mean_bits"]), f"{what}mean differs"
        assert np.array_equal(start, self.start), f"{what}start counts differ"
        assert np.array_equal(end, self.end), f"{what}end counts differ"
        assert np.array_equal(freq, self.freq), f"{what}activity counts differ"
        if n_events is not None:
            assert n_events == self.n_events, f"{what}n_events differs"
        if n_cases is not None:
            assert n_cases == self.n_cases, f"{what}n_cases differs"


def variants_of(R: oracle.Summary):
    """An oracle summary's variant table in the binding's field names."""
    return SimpleNamespace(n_variants=R.n_variants, count=R.var_count, min_case=R.var_min_case, off=R.var_off,
                           acts=R.var_acts, case_ids=R.case_ids, case_variant=R.case_variant)


def check_case_variants(var, R: oracle.Summary, what="") -> None:
    """Each case of the oracle summary R has, under the whole table `var`, the
    same activity sequence as under R."""
    pos = np.searchsorted(var.case_ids, R.case_ids)
    assert np.all(pos < var.case_ids.shape[0]), f"{what}cases missing"
    assert np.array_equal(var.case_ids[pos], R.case_ids), f"{what}cases missing"
    gv = var.case_variant[pos].astype(np.int64)
    ov = R.case_variant.astype(np.int64)
    off = np.asarray(var.off, np.int64)
    glen = off[gv + 1] - off[gv]
    olen = R.var_off[ov + 1] - R.var_off[ov]
    assert np.array_equal(glen, olen), f"{what}case sequence lengths differ"
    assert np.array_equal(var.acts[ranges(off[gv], glen)], R.var_acts[ranges(R.var_off[ov], olen)]), \
        f"{what}case sequences differ"


def check_variant_table(var) -> None:
    """The whole variant table, with every case's rank, obeys the definitions:
    a rank's count is its number of cases and its smallest case the smallest of
    them; ranks order by (count descending, smallest case ascending); no two
    ranks share a sequence (64-bit sequence hashes; equal hashes are compared
    element by element)."""
    V = int(var.n_variants)
    count = np.asarray(var.count)
    assert count.shape[0] == V and var.min_case.shape[0] == V and var.off.shape[0] == V + 1
    cv = np.asarray(var.case_variant)
    assert cv.shape[0] == var.case_ids.shape[0]
    assert np.all(np.diff(var.case_ids) > 0), "case ids not ascending"
    if V == 0:
        assert cv.shape[0] == 0
        return
    assert cv.min() >= 0 and cv.max() < V
    assert np.array_equal(np.bincount(cv, minlength=V).astype(np.uint64), count), "counts differ from the cases"
    ranks, first = np.unique(cv, return_index=True)
    assert ranks.shape[0] == V, "a rank has no case"
    assert np.array_equal(var.case_ids[first], var.min_case), "smallest cases differ"
    c = count.astype(np.int64)
    assert np.all(c[:-1] >= c[1:]), "counts not descending"
    tie = c[:-1] == c[1:]
    assert np.all(var.min_case[:-1][tie] < var.min_case[1:][tie]), "ties not ordered by smallest case"
    off = np.asarray(var.off, np.int64)
    lens = np.diff(off)
    assert lens.min() >= 1
    pos = np.arange(off[-1], dtype=np.int64) - np.repeat(off[:-1], lens)
    pw = np.cumprod(np.full(int(lens.max()), 0x9E3779B97F4A7C15, np.uint64))
    h = np.add.reduceat((var.acts[:off[-1]].astype(np.uint64) + np.uint64(1)) * pw[pos], off[:-1])
    h ^= lens.astype(np.uint64) * np.uint64(0xD6E8FEB86659FD93)
    del pos
    srt = np.argsort(h, kind="stable")
    hs = h[srt]
    dup = np.flatnonzero(hs[1:] == hs[:-1])
    for i in dup:
        a, b = int(srt[i]), int(srt[i + 1])
        assert not np.array_equal(var.acts[off[a]:off[a + 1]], var.acts[off[b]:off[b + 1]]), \
            f"variants {a} and {b} have the same sequence"


def check_summaries_by_case_groups(case_id, activity, ts_ns, A: int, perf, start, end, freq, info, var,
                                   rows=None, rows_case=None, G: int = 64) -> None:
    """A whole log's performance DFG, endpoint counts, sizes, variants (with
    every case's rank) and, if given, formatted order (`rows`, and the case id
    of each formatted position `rows_case`) against the oracle on G groups of
    cases."""
    order, bounds = case_groups(case_id, G)
    if rows is not None:
        e_order, e_bounds = case_groups(rows_case if rows_case is not None else case_id[rows], G)

    def one(g):
        r = order[bounds[g]:bounds[g + 1]]
        R = oracle.summarize(case_id[r], activity[r], ts_ns[r], A)
        if rows is not None:
            mine = rows[e_order[e_bounds[g]:e_bounds[g + 1]]]
            assert np.array_equal(mine, r[R.sorted_rows]), f"group {g}: formatted order differs"
        check_case_variants(var, R, f"group {g}: ")
        return GroupDfg.of(R)

    acc = DfgSum(A)
    for part in pool_map(one, range(G)):
        acc.add(part)
    acc.assert_equal(perf, start, end, freq, info[0], info[1])
    assert var.case_ids.shape[0] == acc.n_cases
    check_variant_table(var)


def check_filter_by_case_groups(case_id, activity, ts_ns, A: int, kind: str, kw: dict, perf, start, end, freq,
                                info, G: int = 64) -> None:
    """A filter whose decision is local to each case (a paths filter, or case
    filters without a variant set) on the whole log, then summarised, against
    the oracle's filter and summary on G groups of cases."""
    assert kind in ("paths", "cases") and not kw.get("variant_set")
    order, bounds = case_groups(case_id, G)

    def one(g):
        r = order[bounds[g]:bounds[g + 1]]
        c, a, t = case_id[r], activity[r], ts_ns[r]
        keep = oracle.filter_paths(c, a, t, A, **kw) if kind == "paths" else oracle.filter_cases(c, a, t, A, **kw)
        return GroupDfg.of(oracle.summarize(c[keep], a[keep], t[keep], A))

    acc = DfgSum(A)
    for part in pool_map(one, range(G)):
        acc.add(part)
    acc.assert_equal(perf, start, end, freq, info[0], info[1], what=f"{kind} {kw}: ")


class EfgSum:
    """Eventually-follows counts, exact sums and exact sums of squares of a
    union of disjoint case groups, on a dense |A| x |A| grid."""

    def __init__(self, A: int):
        self.A = A
        cells = A * A
        self.cnt = np.zeros(cells, np.uint64)
        self.s = [np.zeros(cells, np.uint64) for _ in range(2)]
        self.q = [np.zeros(cells, np.uint64) for _ in range(3)]

    def add(self, F) -> None:
        k = F.src.astype(np.int64) * self.A + F.dst
        self.cnt[k] += F.count
        _add_words(self.s, k, (F.sum_lo, F.sum_hi))
        _add_words(self.q, k, (F.sq0, F.sq1, F.sq2))

    def assert_equal(self, got, what="") -> None:
        k = np.flatnonzero(self.cnt)
        want = {"src": (k // self.A).astype(np.int32), "dst": (k % self.A).astype(np.int32), "count": self.cnt[k],
                "sum_lo": self.s[0][k], "sum_hi": self.s[1][k], "sq0": self.q[0][k], "sq1": self.q[1][k],
                "sq2": self.q[2][k]}
        for name, w in want.items():
            assert np.array_equal(np.asarray(getattr(got, name)), w), f"{what}{name} differs"
        mean, sd = [], []
        for c, s0, s1, q0, q1, q2 in zip(*(want[x] for x in ("count", "sum_lo", "sum_hi", "sq0", "sq1", "sq2"))):
            n = int(c)
            S1 = int(s0) | (int(s1) << 64)
            S2 = int(q0) | (int(q1) << 64) | (int(q2) << 128)
            mean.append(float(S1) / float(n))
            sd.append(math.sqrt(float(n * S2 - S1 * S1) / float(n) / float(n)))
        assert np.array_equal(np.asarray(got.mean).view(np.uint64), np.array(mean, np.float64).view(np.uint64)), \
            f"{what}mean differs"
        assert np.array_equal(np.asarray(got.stdev).view(np.uint64), np.array(sd, np.float64).view(np.uint64)), \
            f"{what}stdev differs"


def check_efg_by_case_groups(case_id, activity, ts_ns, A: int, got, G: int = 64) -> None:
    """A whole log's eventually-follows graph and temporal profile against the
    oracle on G groups of cases."""
    order, bounds = case_groups(case_id, G)

    def one(g):
        r = order[bounds[g]:bounds[g + 1]]
        return oracle.efg(case_id[r], activity[r], ts_ns[r], A)

    acc = EfgSum(A)
    for part in pool_map(one, range(G)):
        acc.add(part)
    acc.assert_equal(got)
