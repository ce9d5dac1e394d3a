"""Filters on derived results on the GPU (paths filter, case filters) against
the oracle, bit-exact: the kept rows (the sub-log's exported rows) and every
summary of the sub-log. All calls go through the C ABI (libpm4g.so)."""

import numpy as np
import pytest

import oracle
import pm4g_synth as synth
from tests.gpu_util import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm4g():
    from paper_2204_04898_b300 import pm4g as m
    return m


@pytest.fixture()
def ctx(pm4g):
    c = pm4g.pm4g_ctx_create(0)
    yield c
    pm4g.pm4g_ctx_destroy(c)


def _load(pm4g, ctx, L):
    import torch
    cols = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns)]
    return pm4g.pm4g_load_log(ctx, *cols, n_activities=L.n_activities)


def _check_sub(pm4g, f, L, rows):
    """The sub-log f holds exactly `rows` of L (ascending) and summarises as
    the oracle does on them."""
    sub = L.take(rows)
    R = oracle.summarize(sub.case_id, sub.activity, sub.ts_ns, L.n_activities)
    got = {"info": pm4g.pm4g_log_info(f), "dfg": pm4g.pm4g_dfg(f), "perf": pm4g.pm4g_perf_dfg(f),
           "var": pm4g.pm4g_variants(f, cases=True)}
    got["start"], got["end"], got["freq"] = pm4g.pm4g_start_end(f, L.n_activities)
    e = pm4g.pm4g_log_export(f)
    assert np.array_equal(np.sort(e["row"]), rows), "kept rows differ"
    got["export"] = dict(e, row=np.searchsorted(rows, e["row"]))
    assert_same(got, R, sub.case_id, sub.activity, sub.ts_ns)


@pytest.mark.parametrize("spec", [synth.drilldown_log(5000), synth.large_log(4000), synth.single_log(3000)],
                         ids=lambda s: s.name)
def test_paths_filter(pm4g, ctx, spec):
    L = synth.generate(spec)
    A = L.n_activities
    log = _load(pm4g, ctx, L)
    try:
        R = oracle.summarize(L.case_id, L.activity, L.ts_ns, A)
        rng = np.random.default_rng(3)
        order = np.argsort(-R.count.astype(np.int64), kind="stable")
        cases = [[], [(int(R.src[order[0]]), int(R.dst[order[0]]))]]
        for _ in range(3):
            k = rng.choice(R.src.size, size=min(R.src.size, int(rng.integers(1, 40))), replace=False)
            pairs = [(int(R.src[i]), int(R.dst[i])) for i in k]
            pairs += [tuple(int(x) for x in rng.integers(0, A, 2)) for _ in range(3)]  # maybe absent pairs
            cases.append(pairs)
        for pairs in cases:
            for ex in (False, True):
                rows = oracle.filter_paths(L.case_id, L.activity, L.ts_ns, A, pairs, exclude=ex)
                f = pm4g.pm4g_filter_paths(log, pairs, exclude=ex)
                try:
                    _check_sub(pm4g, f, L, rows)
                finally:
                    pm4g.pm4g_log_free(f)
    finally:
        pm4g.pm4g_log_free(log)


@pytest.mark.parametrize("spec", [synth.drilldown_log(5000), synth.large_log(4000)], ids=lambda s: s.name)
def test_case_filters(pm4g, ctx, spec):
    L = synth.generate(spec)
    A = L.n_activities
    log = _load(pm4g, ctx, L)
    try:
        R = oracle.summarize(L.case_id, L.activity, L.ts_ns, A)
        lens = R.case_len
        L50 = int(np.median(lens))
        first = L.ts_ns[R.sorted_rows[np.concatenate([[0], np.cumsum(lens)[:-1]])]]
        last = L.ts_ns[R.sorted_rows[np.cumsum(lens) - 1]]
        dur = (last.astype(np.uint64) - first.astype(np.uint64)).astype(np.int64)
        d25, d75 = int(np.percentile(dur, 25)), int(np.percentile(dur, 75))
        top_start = [int(a) for a in np.argsort(-R.start.astype(np.int64))[:2]]
        top_end = [int(a) for a in np.argsort(-R.end.astype(np.int64))[:3]]
        rare = [int(a) for a in np.argsort(R.freq.astype(np.int64))[:5]]
        specs = [
            {},
            {"min_events": L50},
            {"max_events": L50},
            {"min_events": L50, "max_events": L50},
            {"min_duration": d25, "max_duration": d75},
            {"max_duration": 0},
            {"start_set": top_start},
            {"end_set": top_end},
            {"act_set": rare},
            {"variant_set": [0, 1, 2, R.n_variants - 1, R.n_variants + 5]},
            {"min_events": L50, "end_set": top_end, "act_set": rare + top_end},
        ]
        for sp in specs:
            for ex in (False, True):
                rows = oracle.filter_cases(L.case_id, L.activity, L.ts_ns, A, exclude=ex, **sp)
                f = pm4g.pm4g_filter_cases(log, exclude=ex, **sp)
                try:
                    _check_sub(pm4g, f, L, rows)
                finally:
                    pm4g.pm4g_log_free(f)
    finally:
        pm4g.pm4g_log_free(log)


def test_derived_filter_errors_and_empty(pm4g, ctx):
    L = synth.generate(synth.large_log(500))
    log = _load(pm4g, ctx, L)
    try:
        with pytest.raises(pm4g.Pm4gError):
            pm4g.pm4g_filter_paths(log, [(0, L.n_activities)])
        with pytest.raises(pm4g.Pm4gError):
            pm4g.pm4g_filter_cases(log, act_set=[-1])
        # nothing kept: an empty log that still answers
        f = pm4g.pm4g_filter_paths(log, [])
        try:
            assert pm4g.pm4g_log_info(f) == (0, 0)
            assert pm4g.pm4g_perf_dfg(f).n_edges == 0
        finally:
            pm4g.pm4g_log_free(f)
        # a filtered log filters again
        f1 = pm4g.pm4g_filter_cases(log, min_events=3)
        try:
            f2 = pm4g.pm4g_filter_paths(f1, [(0, 1), (1, 2)], exclude=True)
            try:
                r1 = oracle.filter_cases(L.case_id, L.activity, L.ts_ns, L.n_activities, min_events=3)
                s1 = L.take(r1)
                r2 = oracle.filter_paths(s1.case_id, s1.activity, s1.ts_ns, L.n_activities, [(0, 1), (1, 2)],
                                         exclude=True)
                _check_sub(pm4g, f2, L, r1[r2])
            finally:
                pm4g.pm4g_log_free(f2)
        finally:
            pm4g.pm4g_log_free(f1)
    finally:
        pm4g.pm4g_log_free(log)
