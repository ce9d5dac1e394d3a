"""The case-group checks (tests/case_groups.py) on the CPU: the oracle's
whole-log results pass them (the sums over case groups, extremes, per-case
values and the FP64 means and deviations recombine exactly), and a planted
mistake in a whole-log result (a sum, an extreme, a formatted position, a
case's rank, a duplicated variant, a square) is caught. The full-size GPU
tests rest on these checks."""

import copy

import numpy as np
import pytest

import oracle
import pm4g_synth as synth

from .case_groups import (check_efg_by_case_groups, check_filter_by_case_groups, check_summaries_by_case_groups,
                          check_variant_table, variants_of)


@pytest.fixture(scope="module")
def logs(oracle_lib):
    out = []
    for spec in (synth.very_large_log(6000), synth.large_log(4000)):
        L = synth.generate(spec)
        out.append((L, oracle.summarize(L.case_id, L.activity, L.ts_ns, L.n_activities)))
    return out


def _check(L, R, var=None, rows=None, perf=None, G=8):
    check_summaries_by_case_groups(L.case_id, L.activity, L.ts_ns, L.n_activities, perf or R, R.start, R.end,
                                   R.freq, (R.n_events, R.n_cases), var or variants_of(R),
                                   rows=R.sorted_rows if rows is None else rows, G=G)


@pytest.mark.parametrize("G", [1, 8, 64])
def test_whole_oracle_result_recombines(logs, G):
    for L, R in logs:
        _check(L, R, G=G)


def test_planted_mistakes_are_caught(logs):
    L, R = logs[0]
    bad = copy.deepcopy(R)
    bad.sum_lo[3] += np.uint64(1)
    with pytest.raises(AssertionError, match="sum_lo"):
        _check(L, R, perf=bad)
    bad = copy.deepcopy(R)
    bad.max[5] += np.uint64(1)
    with pytest.raises(AssertionError, match="max"):
        _check(L, R, perf=bad)
    bad = copy.deepcopy(R)
    bad.mean[7] = np.nextafter(bad.mean[7], np.inf)
    with pytest.raises(AssertionError, match="mean"):
        _check(L, R, perf=bad)
    # two events of one case trade places in the formatted order
    rows = R.sorted_rows.copy()
    i = int(np.flatnonzero(L.case_id[rows][1:] == L.case_id[rows][:-1])[0])
    rows[i], rows[i + 1] = rows[i + 1], rows[i]
    with pytest.raises(AssertionError, match="formatted order"):
        _check(L, R, rows=rows)
    # a case moved to another variant
    var = variants_of(R)
    cv = var.case_variant.copy()
    cv[np.flatnonzero(cv == 0)[0]] = 1
    var.case_variant = cv
    with pytest.raises(AssertionError, match="case sequence"):
        _check(L, R, var=var)


def test_variant_table_mistakes_are_caught(logs):
    L, R = logs[0]
    check_variant_table(variants_of(R))
    # a later rank given rank 0's sequence: two ranks share a sequence
    var = variants_of(R)
    lens = np.diff(var.off)
    r = int(np.flatnonzero(lens[1:] == lens[0])[0]) + 1
    acts = var.acts.copy()
    acts[var.off[r]:var.off[r + 1]] = var.acts[var.off[0]:var.off[1]]
    var.acts = acts
    with pytest.raises(AssertionError, match="same sequence"):
        check_variant_table(var)
    var = variants_of(R)
    mc = var.min_case.copy()
    mc[0] += 1
    var.min_case = mc
    with pytest.raises(AssertionError, match="smallest cases"):
        check_variant_table(var)
    var = variants_of(R)
    var.count = var.count[::-1].copy()
    with pytest.raises(AssertionError):
        check_variant_table(var)


def test_efg_recombines_and_catches_mistakes(logs):
    for L, _ in logs:
        F = oracle.efg(L.case_id, L.activity, L.ts_ns, L.n_activities)
        check_efg_by_case_groups(L.case_id, L.activity, L.ts_ns, L.n_activities, F, G=8)
    bad = copy.deepcopy(F)
    bad.sq1[np.argmax(bad.sq1)] += np.uint64(1)
    with pytest.raises(AssertionError, match="sq1"):
        check_efg_by_case_groups(L.case_id, L.activity, L.ts_ns, L.n_activities, bad, G=8)
    bad = copy.deepcopy(F)
    bad.stdev[0] = np.nextafter(bad.stdev[0], 0)
    with pytest.raises(AssertionError, match="stdev"):
        check_efg_by_case_groups(L.case_id, L.activity, L.ts_ns, L.n_activities, bad, G=8)


def test_case_local_filters_recombine(logs):
    L, R = logs[0]
    A = L.n_activities
    top = np.argsort(-R.count.astype(np.int64), kind="stable")[:5]
    for kind, kw in (("paths", {"pairs": [(int(R.src[i]), int(R.dst[i])) for i in top]}),
                     ("cases", {"min_events": int(np.median(R.case_len))}),
                     ("cases", {"end_set": [int(np.argmax(R.end))], "exclude": True})):
        keep = (oracle.filter_paths(L.case_id, L.activity, L.ts_ns, A, **kw) if kind == "paths"
                else oracle.filter_cases(L.case_id, L.activity, L.ts_ns, A, **kw))
        S = oracle.summarize(L.case_id[keep], L.activity[keep], L.ts_ns[keep], A)
        check_filter_by_case_groups(L.case_id, L.activity, L.ts_ns, A, kind, kw, S, S.start, S.end, S.freq,
                                    (S.n_events, S.n_cases), G=8)
