"""Checks that pin the CPU oracle to something other than itself.

Each check takes an oracle library handle (the real one, or a mutated copy) and
raises AssertionError on a mismatch. The pins are: the definitional brute force
on exhaustively enumerated and random tiny logs; invariants fixed by the
definitions; a closed form for the duration sums; the paper's case replication
(Section 4) as a metamorphic relation; row shuffles and tied-row swaps; special
cases that reduce to hand-known answers; filter identities; hand-derived golden
fixtures.
"""

from __future__ import annotations

import itertools
import json
import os

import numpy as np

import oracle
import pm4g_synth as synth
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
U64 = 1 << 64


def summarize(lib, case, act, ts, A):
    return oracle.summarize(np.asarray(case, np.int32), np.asarray(act, np.int32),
                            np.asarray(ts, np.int64), A, lib=lib)


def as_dict(R):
    """Oracle summary in the brute force's plain-Python form."""
    sums = R.edge_sums()
    edges = {}
    for k in range(R.n_edges):
        edges[(int(R.src[k]), int(R.dst[k]))] = (int(R.count[k]), sums[k], int(R.min[k]), int(R.max[k]))
    seqs = R.variant_seqs()
    return {
        "edges": edges,
        "start": [int(x) for x in R.start],
        "end": [int(x) for x in R.end],
        "freq": [int(x) for x in R.freq],
        "variants": [(seqs[v], int(R.var_count[v]), int(R.var_min_case[v])) for v in range(R.n_variants)],
        "cases": [int(c) for c in R.case_ids],
        "case_variant": [int(v) for v in R.case_variant],
        "case_len": [int(x) for x in R.case_len],
    }


def check_against_bruteforce(lib, case, act, ts, A):
    R = summarize(lib, case, act, ts, A)
    got = as_dict(R)
    want = bf.summary(list(case), list(act), list(ts), A)
    assert got == want, f"mismatch on log case={case} act={act} ts={ts}:\n got={got}\n want={want}"
    assert [int(r) for r in R.sorted_rows] == bf.sorted_rows(list(case), list(ts))
    for k in range(R.n_edges):
        s = int(R.sum_lo[k]) + (int(R.sum_hi[k]) << 64)
        assert R.mean[k] == float(s) / float(int(R.count[k])) or \
            R.mean[k] == np.float64(s) / np.float64(int(R.count[k]))


def check_bruteforce_exhaustive(lib, max_n=4, cases=(-2, 1), acts=(0, 1, 2), tss=(-1, 1)):
    """Every log with up to ``max_n`` rows over the given value sets (forces
    timestamp ties and negative ids)."""
    A = max(acts) + 1
    rows = list(itertools.product(cases, acts, tss))
    n_logs = 0
    for n in range(0, max_n + 1):
        for log in itertools.product(rows, repeat=n):
            case = [r[0] for r in log]
            act = [r[1] for r in log]
            ts = [r[2] for r in log]
            check_against_bruteforce(lib, case, act, ts, A)
            n_logs += 1
    return n_logs


def check_bruteforce_random(lib, n_logs=300, seed=7, max_n=12):
    rng = np.random.default_rng(seed)
    extremes = np.array([-2**63, -2**62, -1, 0, 1, 2**62, 2**63 - 1], dtype=np.int64)
    for t in range(n_logs):
        n = int(rng.integers(0, max_n + 1))
        A = int(rng.integers(1, 5))
        case = rng.choice([-2**31, -5, 0, 3, 2**31 - 1], size=n).tolist()
        act = rng.integers(0, A, size=n).tolist()
        if t % 3 == 0:
            ts = rng.choice(extremes, size=n).tolist()
        else:
            ts = rng.integers(0, 4, size=n).tolist()
        check_against_bruteforce(lib, case, act, [int(x) for x in ts], A)


def check_invariants(lib, log):
    R = oracle.summarize(log.case_id, log.activity, log.ts_ns, log.n_activities, lib=lib)
    N, C, A = log.n_events, R.n_cases, log.n_activities
    # cases: distinct ids ascending, lengths sum to N
    ids = np.unique(log.case_id)
    assert np.array_equal(R.case_ids, ids)
    assert int(R.case_len.sum()) == N
    assert np.array_equal(R.case_len, np.bincount(np.searchsorted(ids, log.case_id), minlength=C))
    # DFG edge total = events - cases
    assert int(R.count.sum()) == N - C
    # per-activity out-edges + end = freq; in-edges + start = freq
    out_ = np.zeros(A, np.uint64)
    in_ = np.zeros(A, np.uint64)
    np.add.at(out_, R.src, R.count)
    np.add.at(in_, R.dst, R.count)
    assert np.array_equal(out_ + R.end, R.freq)
    assert np.array_equal(in_ + R.start, R.freq)
    assert np.array_equal(R.freq, np.bincount(log.activity, minlength=A).astype(np.uint64))
    assert int(R.start.sum()) == C and int(R.end.sum()) == C
    # edges strictly ascending by (src, dst) and nonzero
    key = R.src.astype(np.int64) * A + R.dst
    assert np.all(np.diff(key) > 0) and np.all(R.count > 0)
    # min <= mean <= max; single-pair edges have min = max = mean
    assert np.all(R.min <= R.max)
    assert np.all(R.min.astype(np.float64) <= R.mean) and np.all(R.mean <= R.max.astype(np.float64))
    one = R.count == 1
    assert np.all(R.min[one] == R.max[one])
    assert np.all(R.mean[one] == R.min[one].astype(np.float64))
    # variants: counts sum to C, count x length sums to N, bijective ids, order
    V = R.n_variants
    lens = np.diff(R.var_off)
    assert int(R.var_count.sum()) == C
    assert int((R.var_count * lens.astype(np.uint64)).sum()) == N
    assert np.array_equal(np.sort(np.unique(R.case_variant)), np.arange(V))
    assert np.array_equal(np.bincount(R.case_variant, minlength=V).astype(np.uint64), R.var_count)
    assert np.all(np.diff(R.var_count.astype(np.int64)) <= 0)
    tie = np.diff(R.var_count.astype(np.int64)) == 0
    assert np.all(np.diff(R.var_min_case)[tie] > 0)
    # each variant's smallest case id really is the smallest case with that variant
    mins = np.full(V, np.iinfo(np.int32).max, np.int64)
    np.minimum.at(mins, R.case_variant, R.case_ids.astype(np.int64))
    assert np.array_equal(mins, R.var_min_case.astype(np.int64))
    assert np.array_equal(lens[R.case_variant], R.case_len)
    return R


def check_closed_form_sums(lib, log, R=None):
    """Sum over edges of the duration sums = sum over cases of (last - first),
    computed from the unsorted columns with per-case max/min."""
    R = R or oracle.summarize(log.case_id, log.activity, log.ts_ns, log.n_activities, lib=lib)
    ids, inv = np.unique(log.case_id, return_inverse=True)
    tmax = np.full(ids.shape[0], np.iinfo(np.int64).min, np.int64)
    tmin = np.full(ids.shape[0], np.iinfo(np.int64).max, np.int64)
    np.maximum.at(tmax, inv, log.ts_ns)
    np.minimum.at(tmin, inv, log.ts_ns)
    want = sum(int(a) - int(b) for a, b in zip(tmax.tolist(), tmin.tolist()))
    got = sum(R.edge_sums())
    assert got == want, (got, want)


def check_replication(lib, log, k=3):
    """The paper replicates every case k times (Section 4): counts and sums
    scale by k, min/max and the variant set and order stay."""
    R = oracle.summarize(log.case_id, log.activity, log.ts_ns, log.n_activities, lib=lib)
    shift = int(log.case_id.max()) + 1
    case = np.concatenate([log.case_id + i * shift for i in range(k)]).astype(np.int32)
    act = np.tile(log.activity, k)
    ts = np.tile(log.ts_ns, k)
    Rk = oracle.summarize(case, act, ts, log.n_activities, lib=lib)
    assert np.array_equal(Rk.src, R.src) and np.array_equal(Rk.dst, R.dst)
    assert np.array_equal(Rk.count, R.count * np.uint64(k))
    assert [s * k for s in R.edge_sums()] == Rk.edge_sums()
    assert np.array_equal(Rk.min, R.min) and np.array_equal(Rk.max, R.max)
    assert Rk.variant_seqs() == R.variant_seqs()
    assert np.array_equal(Rk.var_count, R.var_count * np.uint64(k))
    assert np.array_equal(Rk.var_min_case, R.var_min_case)
    assert np.array_equal(Rk.start, R.start * np.uint64(k))
    assert np.array_equal(Rk.end, R.end * np.uint64(k))


def check_shuffle(lib, log, seed=3):
    """Without tied timestamps inside a case, row order is irrelevant."""
    key = log.case_id.astype(np.int64) * (1 << 32)
    order = np.lexsort((log.ts_ns, log.case_id))
    c, t = log.case_id[order], log.ts_ns[order]
    tied = np.any((c[1:] == c[:-1]) & (t[1:] == t[:-1]))
    assert not tied, "log has ties; pick one without"
    del key
    R = oracle.summarize(log.case_id, log.activity, log.ts_ns, log.n_activities, lib=lib)
    p = np.random.default_rng(seed).permutation(log.n_events)
    Rp = oracle.summarize(log.case_id[p], log.activity[p], log.ts_ns[p], log.n_activities, lib=lib)
    for f in ("src", "dst", "count", "sum_lo", "sum_hi", "min", "max", "mean", "start", "end",
              "freq", "var_count", "var_min_case", "var_off", "var_acts", "case_ids", "case_variant"):
        assert np.array_equal(getattr(R, f), getattr(Rp, f)), f


def check_tie_swap(lib):
    """Two events of one case with equal timestamps: the earlier row comes
    first, so swapping the rows swaps their order in the sequence."""
    case = [7, 7, 7]
    ts = [5, 5, 1]
    R1 = summarize(lib, case, [0, 1, 2], ts, 3)
    R2 = summarize(lib, case, [1, 0, 2], ts, 3)
    assert R1.variant_seqs() == [(2, 0, 1)]
    assert R2.variant_seqs() == [(2, 1, 0)]
    assert list(R1.sorted_rows) == [2, 0, 1]


def check_specials(lib):
    rng = np.random.default_rng(11)
    # A = 1: one edge (0, 0) with count N - C
    case = rng.integers(0, 50, 400).astype(np.int32)
    ts = rng.integers(0, 1000, 400)
    R = summarize(lib, case, np.zeros(400, np.int32), ts, 1)
    C = len(np.unique(case))
    assert list(R.src) == [0] and list(R.dst) == [0] and int(R.count[0]) == 400 - C
    assert R.n_variants == len(np.unique(np.bincount(case)[np.bincount(case) > 0]))
    # every case of length 1: no edges, V = number of distinct activities
    case = np.arange(300, dtype=np.int32)[::-1].copy()
    act = rng.integers(0, 7, 300).astype(np.int32)
    R = summarize(lib, case, act, rng.integers(-5, 5, 300), 9)
    assert R.n_edges == 0
    assert R.n_variants == len(np.unique(act))
    assert np.array_equal(R.start, R.end) and np.array_equal(R.start, R.freq)
    # empty log
    R = summarize(lib, [], [], [], 4)
    assert R.n_cases == 0 and R.n_edges == 0 and R.n_variants == 0
    assert int(R.start.sum()) == 0 and int(R.freq.sum()) == 0
    # errors: activity out of range, bad alphabet
    for act_bad in ([0, 3], [-1, 0]):
        try:
            summarize(lib, [1, 1], act_bad, [0, 1], 3)
            raise AssertionError("expected ERANGE")
        except oracle.OracleError as e:
            assert e.status == oracle.ERANGE
    try:
        summarize(lib, [1], [0], [0], 0)
        raise AssertionError("expected EINVAL")
    except oracle.OracleError as e:
        assert e.status == oracle.EINVAL


def check_big_durations(lib):
    """Durations near 2^64 and sums beyond 2^64 stay exact."""
    lo, hi = -2**63, 2**63 - 1
    case = [1, 1, 2, 2, 3, 3, 3]
    act = [0, 1, 0, 1, 0, 1, 0]
    ts = [lo, hi, lo, hi, lo, hi, hi]
    R = summarize(lib, case, act, ts, 2)
    sums = dict(zip(zip(R.src.tolist(), R.dst.tolist()), R.edge_sums()))
    assert sums[(0, 1)] == 3 * (U64 - 1)
    assert sums[(1, 0)] == 0
    k = list(zip(R.src.tolist(), R.dst.tolist())).index((0, 1))
    assert int(R.min[k]) == U64 - 1 and int(R.max[k]) == U64 - 1
    assert R.mean[k] == float(U64 - 1)
    # many large durations: the 64-bit sum overflows, the exact one does not
    n = 5000
    case = np.repeat(np.arange(n, dtype=np.int32), 2)
    ts = np.tile(np.array([0, 2**62 + 12345], np.int64), n)
    R = summarize(lib, case, np.zeros(2 * n, np.int32), ts, 1)
    assert R.edge_sums() == [n * (2**62 + 12345)]
    assert R.mean[0] == float(n * (2**62 + 12345)) / float(n)


def check_filters(lib, log, seed=5):
    rng = np.random.default_rng(seed)
    n = log.n_events
    attr = log.case_attr if log.case_attr is not None else (log.case_id % 13).astype(np.int32)
    t0, t1 = int(log.ts_ns.min()), int(log.ts_ns.max())
    args = (log.case_id, log.activity, log.ts_ns, attr, log.n_activities)
    for mode in range(4):
        rows = oracle.filter_rows(*args, [], t0, t1, mode, lib=lib)
        assert np.array_equal(rows, np.arange(n)), f"identity failed for mode {mode}"
    aset = np.unique(rng.choice(attr, size=5))
    lo = t0 + (t1 - t0) // 4
    hi = t0 + 3 * (t1 - t0) // 4
    cont = oracle.filter_rows(*args, aset, lo, hi, 2, lib=lib)
    inter = oracle.filter_rows(*args, aset, lo, hi, 3, lib=lib)
    assert set(cont.tolist()) <= set(inter.tolist())
    ev = oracle.filter_rows(*args, aset, lo, hi, 1, lib=lib)
    none = oracle.filter_rows(*args, aset, lo, hi, 0, lib=lib)
    inwin = (log.ts_ns[none] >= lo) & (log.ts_ns[none] <= hi)
    assert np.array_equal(ev, none[inwin])
    # contained cases lie inside the window; intersecting ones overlap it
    for rows, m in ((cont, 2), (inter, 3)):
        if rows.size == 0:
            continue
        ids, inv = np.unique(log.case_id[rows], return_inverse=True)
        tmin = np.full(ids.shape[0], np.iinfo(np.int64).max)
        tmax = np.full(ids.shape[0], np.iinfo(np.int64).min)
        np.minimum.at(tmin, inv, log.ts_ns[rows])
        np.maximum.at(tmax, inv, log.ts_ns[rows])
        if m == 2:
            assert np.all(tmin >= lo) and np.all(tmax <= hi)
        else:
            assert np.all(tmin <= hi) and np.all(tmax >= lo)


def check_filters_bruteforce(lib, n_logs=200, seed=9):
    rng = np.random.default_rng(seed)
    for _ in range(n_logs):
        n = int(rng.integers(0, 10))
        case = rng.integers(0, 3, n).tolist()
        act = rng.integers(0, 2, n).tolist()
        ts = rng.integers(0, 5, n).tolist()
        attr = rng.integers(0, 3, n).tolist()  # may vary within a case
        aset = sorted(set(rng.integers(0, 3, int(rng.integers(0, 3))).tolist()))
        t_lo = int(rng.integers(0, 5))
        t_hi = t_lo + int(rng.integers(0, 3))
        for mode in range(4):
            got = oracle.filter_rows(case, act, ts, attr, 2, aset, t_lo, t_hi, mode, lib=lib)
            want = bf.filter_rows(case, act, ts, attr, aset, t_lo, t_hi, mode)
            assert got.tolist() == want, (case, ts, attr, aset, t_lo, t_hi, mode, got, want)


def check_derived_filters_bruteforce(lib, n_logs=150, seed=13):
    """Paths and case filters against their definitions on random tiny logs."""
    rng = np.random.default_rng(seed)
    for _ in range(n_logs):
        n = int(rng.integers(0, 10))
        case = rng.integers(0, 3, n).tolist()
        act = rng.integers(0, 3, n).tolist()
        ts = rng.integers(0, 6, n).tolist()
        pairs = [tuple(rng.integers(0, 3, 2).tolist()) for _ in range(int(rng.integers(0, 4)))]
        for ex in (False, True):
            got = oracle.filter_paths(case, act, ts, 3, pairs, exclude=ex, lib=lib)
            want = bf.filter_paths(case, act, ts, pairs, exclude=ex)
            assert got.tolist() == want, ("paths", case, act, ts, pairs, ex, got, want)
        spec = {}
        for k, hi in (("min_events", 4), ("max_events", 4), ("min_duration", 6), ("max_duration", 6)):
            if rng.random() < 0.4:
                spec[k] = int(rng.integers(0, hi))
        for k in ("start_set", "end_set", "act_set", "variant_set"):
            if rng.random() < 0.4:
                spec[k] = sorted(set(rng.integers(0, 3, int(rng.integers(1, 3))).tolist()))
        for ex in (False, True):
            got = oracle.filter_cases(case, act, ts, 3, exclude=ex, lib=lib, **spec)
            want = bf.filter_cases(case, act, ts, exclude=ex, **spec)
            assert got.tolist() == want, ("cases", case, act, ts, spec, ex, got, want)


def check_derived_filters(lib, log, seed=11):
    """Identities of the paths and case filters on a workload-shaped log."""
    rng = np.random.default_rng(seed)
    n, A = log.n_events, log.n_activities
    args = (log.case_id, log.activity, log.ts_ns, A)
    R = oracle.summarize(*args, lib=lib)
    everything = np.arange(n)
    # exclude is the complement; no criterion keeps every row
    pairs = [tuple(p) for p in rng.integers(0, A, (5, 2)).tolist()]
    kp, kx = (oracle.filter_paths(*args, pairs, exclude=e, lib=lib) for e in (False, True))
    assert np.array_equal(np.sort(np.concatenate([kp, kx])), everything) and np.intersect1d(kp, kx).size == 0
    assert np.array_equal(oracle.filter_cases(*args, lib=lib), everything)
    assert oracle.filter_cases(*args, exclude=True, lib=lib).size == 0
    # every pair keeps exactly the events that have a previous event in their case
    allp = [(a, b) for a in range(A) for b in range(A)] if A <= 40 else [tuple(e) for e in zip(R.src, R.dst)]
    rows = oracle.filter_paths(*args, allp, lib=lib)
    assert rows.size == n - R.n_cases
    first = R.sorted_rows[np.concatenate([[0], np.cumsum(R.case_len)[:-1]]).astype(np.int64)]
    assert np.intersect1d(rows, first).size == 0
    # a path's kept events are as many as the edge's count
    for k in range(min(5, R.src.size)):
        assert oracle.filter_paths(*args, [(int(R.src[k]), int(R.dst[k]))], lib=lib).size == int(R.count[k])
    # exact case sizes; a variant keeps its count of cases
    L = int(R.case_len[R.case_len.size // 2])
    kept = oracle.filter_cases(*args, min_events=L, max_events=L, lib=lib)
    assert kept.size == L * int(np.sum(R.case_len == L))
    for v in range(min(3, R.n_variants)):
        kept = oracle.filter_cases(*args, variant_set=[v], lib=lib)
        assert np.unique(log.case_id[kept]).size == int(R.var_count[v])
    # start set = every activity keeps everything; the start counts split the cases
    assert np.array_equal(oracle.filter_cases(*args, start_set=list(range(A)), lib=lib), everything)
    a0 = int(np.argmax(R.start))
    assert np.unique(log.case_id[oracle.filter_cases(*args, start_set=[a0], lib=lib)]).size == int(R.start[a0])


def check_golden_filters(lib, name):
    g = load_golden(name)
    base = load_golden(g["log"])
    lg = base["log"]
    args = (lg["case"], lg["activity"], lg["ts"], base["n_activities"])
    for chk in g["checks"]:
        if chk["kind"] == "paths":
            got = oracle.filter_paths(*args, chk["pairs"], exclude=chk["exclude"], lib=lib)
        else:
            got = oracle.filter_cases(*args, lib=lib, **chk["spec"])
        assert got.tolist() == chk["rows"], (chk, got)


def _ulps(x, y):
    """Distance between two doubles in units of the larger one's last place."""
    import math
    if x == y:
        return 0.0
    return abs(x - y) / math.ulp(max(abs(x), abs(y)))


def check_efg_bruteforce(lib, n_logs=150, seed=17):
    """Eventually-follows pairs against their definition on random tiny logs:
    exact counts, sums and sums of squares; the mean within one unit in the last
    place of the exact quotient, the standard deviation within four of the
    correctly rounded population deviation."""
    import statistics
    from fractions import Fraction
    rng = np.random.default_rng(seed)
    for it in range(n_logs):
        n = int(rng.integers(0, 12))
        case = rng.integers(0, 3, n).tolist()
        act = rng.integers(0, 3, n).tolist()
        big = it % 3 == 0  # durations near 2^62: squares need the third word
        ts = (rng.integers(0, 2**62, n) if big else rng.integers(0, 7, n)).tolist()
        E = oracle.efg(case, act, ts, 3, lib=lib)
        want = bf.efg(case, act, ts)
        got = {(int(a), int(b)): (int(c), s, q) for a, b, c, s, q in
               zip(E.src, E.dst, E.count, E.sums(), E.squares())}
        assert got == want, (case, act, ts, got, want)
        for k, (key, (c, sm, sq)) in enumerate(want.items()):
            assert _ulps(float(E.mean[k]), float(Fraction(sm, c))) <= 1.0, (key, E.mean[k], sm, c)
            durs = [ts[j] - ts[i] for i in range(n) for j in range(n)
                    if i != j and case[i] == case[j] and (ts[i], i) < (ts[j], j) and (act[i], act[j]) == key]
            ref = statistics.pstdev(durs) if len(durs) > 1 else 0.0
            assert _ulps(float(E.stdev[k]), ref) <= 4.0 or abs(E.stdev[k] - ref) <= 1e-300, (key, E.stdev[k], ref)


def check_efg_invariants(lib, log, seed=19):
    """Identities of the eventually-follows graph on a workload-shaped log."""
    rng = np.random.default_rng(seed)
    A = log.n_activities
    E = oracle.efg(log.case_id, log.activity, log.ts_ns, A, lib=lib)
    R = oracle.summarize(log.case_id, log.activity, log.ts_ns, A, lib=lib)
    L = R.case_len.astype(np.int64)
    assert int(E.count.astype(np.int64).sum()) == int(np.sum(L * (L - 1) // 2))
    ef = {(int(a), int(b)): int(c) for a, b, c in zip(E.src, E.dst, E.count)}
    for a, b, c in zip(R.src, R.dst, R.count):  # every directly-follows pair eventually follows
        assert ef[(int(a), int(b))] >= int(c)
    assert np.all(E.stdev[E.count == 1] == 0.0) and np.all(E.mean >= 0)
    # shifting one case's timestamps changes nothing; shuffling rows neither
    shift = rng.integers(-10**9, 10**9, int(log.case_id.max()) + 1)
    E2 = oracle.efg(log.case_id, log.activity, log.ts_ns + shift[log.case_id], A, lib=lib)
    for f in ("src", "dst", "count", "sum_lo", "sum_hi", "sq0", "sq1", "sq2", "mean", "stdev"):
        assert np.array_equal(getattr(E, f), getattr(E2, f)), f
    pairs = np.stack([log.case_id.astype(np.int64), log.ts_ns], axis=1)
    if np.unique(pairs, axis=0).shape[0] == log.n_events:  # no tied timestamps in a case: rows do not matter
        p = rng.permutation(log.n_events)
        E3 = oracle.efg(log.case_id[p], log.activity[p], log.ts_ns[p], A, lib=lib)
        for f in ("src", "dst", "count", "sum_lo", "sq0", "sq1", "stdev"):
            assert np.array_equal(getattr(E, f), getattr(E3, f)), f"shuffle: {f}"


def check_golden_efg(lib, name):
    from fractions import Fraction
    import math
    g = load_golden(name)
    base = load_golden(g["log"])
    lg = base["log"]
    E = oracle.efg(lg["case"], lg["activity"], lg["ts"], base["n_activities"], lib=lib)
    assert [(int(a), int(b)) for a, b in zip(E.src, E.dst)] == [(p["src"], p["dst"]) for p in g["pairs"]]
    for k, p in enumerate(g["pairs"]):
        assert int(E.count[k]) == p["count"] and E.sums()[k] == p["sum"] and E.squares()[k] == p["sumsq"], p
        if isinstance(p["mean"], str):
            num, den = (int(x) for x in p["mean"].split("/"))
            assert _ulps(float(E.mean[k]), float(Fraction(num, den))) <= 1.0, p
        else:
            assert float(E.mean[k]) == p["mean"], p
        var = Fraction(*p["var"])
        if p["stdev"] is not None:
            assert float(E.stdev[k]) == p["stdev"], p
        else:
            assert _ulps(float(E.stdev[k]), math.sqrt(float(var))) <= 2.0, p


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def check_golden(lib, name):
    g = load_golden(name)
    log = g["log"]
    R = summarize(lib, log["case"], log["activity"], log["ts"], g["n_activities"])
    got = as_dict(R)
    exp = g["expected"]
    want_edges = {(e[0], e[1]): (e[2], e[3], e[4], e[5]) for e in exp["edges"]}
    assert got["edges"] == want_edges, (got["edges"], want_edges)
    assert R.mean.tolist() == exp["means"]
    assert R.sorted_rows.tolist() == exp["sorted_rows"]
    assert got["start"] == exp["start"] and got["end"] == exp["end"] and got["freq"] == exp["freq"]
    assert [[list(s), c, m] for s, c, m in got["variants"]] == exp["variants"]
    assert got["cases"] == exp["case_ids"]
    assert got["case_variant"] == exp["case_variant"]
    return g


def small_logs():
    """Seeded workload-shaped logs small enough for every CPU check."""
    return [
        synth.generate(synth.single_log(2000)),
        synth.generate(synth.large_log(3000)),
        synth.generate(synth.very_large_log(3000)),
        synth.generate(synth.drilldown_log(2000)),
    ]


def run_all(lib, quick=True):
    """Every pin, in a compact form (used to show planted mistakes are caught)."""
    check_bruteforce_exhaustive(lib, max_n=3)
    check_bruteforce_random(lib, n_logs=150 if quick else 600)
    check_tie_swap(lib)
    check_specials(lib)
    check_big_durations(lib)
    check_filters_bruteforce(lib, n_logs=60 if quick else 300)
    check_derived_filters_bruteforce(lib, n_logs=60 if quick else 300)
    check_efg_bruteforce(lib, n_logs=60 if quick else 300)
    for name in sorted(os.listdir(GOLDEN)):
        if name.endswith(".json"):
            check = check_golden_filters if name.startswith("filters_") else (
                check_golden_efg if name.startswith("efg_") else check_golden)
            check(lib, name)
    for log in small_logs():
        R = check_invariants(lib, log)
        check_closed_form_sums(lib, log, R)
        check_replication(lib, log, k=2)
        check_filters(lib, log)
        check_derived_filters(lib, log)
    check_efg_invariants(lib, small_logs()[0])
