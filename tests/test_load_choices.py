"""The single-log pass's launch choices (bucket width, second-level partition
units, streaming-pass warps, streaming pass on or off, dense or hashed global
edge table, records a thread stages per partition tile, coarse fan-out) never change a result: every output of pm4g_load_log and the
summaries is bit-identical across choice sets and equal to the oracle's, and
a context the autotuner tuned keeps giving the oracle's results."""

import numpy as np
import pytest

import oracle
import pm4g_synth as synth
from tests.gpu_util import assert_same, collect

pytestmark = pytest.mark.gpu

CHOICES = [
    {},                                                              # defaults
    {"clb": 6, "splits": 2},
    {"stream_warps": 12, "edge_table": 1},
    {"stream_off": 1, "clb": 7},
    {"clb": 8, "splits": 16, "stream_warps": 20},
    {"clb": 3, "stream_off": 1, "edge_table": 1},
    {"part1_items": 4},
    {"part1_items": 4, "part2_items": 8, "clb": 7, "splits": 4},
    {"part_fbits": 9},
    {"part_fbits": 8, "clb": 6, "part2_items": 8},
]


def _run(pm4g, ctx, L, choice):
    import torch
    from paper_2204_04898_b300 import autotune
    autotune.Tuner.apply(ctx, {**autotune.LOAD_DEFAULTS, **choice}, autotune.LOAD_KNOBS)
    cols = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (L.case_id, L.activity, L.ts_ns)]
    log = pm4g.pm4g_load_log(ctx, *cols, n_activities=L.n_activities)
    try:
        return collect(pm4g, log, L.n_activities)
    finally:
        pm4g.pm4g_log_free(log)


def _same(a, b):
    assert a["info"] == b["info"]
    for k in ("src", "dst", "count"):
        assert np.array_equal(a["dfg"][k], b["dfg"][k]), k
    for k in ("src", "dst", "count", "sum_lo", "sum_hi", "min", "max"):
        assert np.array_equal(getattr(a["perf"], k), getattr(b["perf"], k)), k
    assert np.array_equal(a["perf"].mean.view(np.uint64), b["perf"].mean.view(np.uint64))
    for k in ("start", "end", "freq"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("count", "min_case", "off", "acts", "case_ids", "case_variant"):
        assert np.array_equal(getattr(a["var"], k), getattr(b["var"], k)), k
    for k in a["export"]:
        assert np.array_equal(a["export"][k], b["export"][k]), k


@pytest.mark.parametrize("law", ["very_large_log", "large_log"])
def test_results_do_not_depend_on_load_choices(law):
    from paper_2204_04898_b300 import pm4g
    L = synth.generate(synth.WORKLOADS[law]().scaled(30000, law))
    R = oracle.summarize(L.case_id, L.activity, L.ts_ns, L.n_activities)
    ctx = pm4g.pm4g_ctx_create(0)
    try:
        runs = [_run(pm4g, ctx, L, c) for c in CHOICES]
    finally:
        pm4g.pm4g_ctx_destroy(ctx)
    assert_same(runs[0], R, L.case_id, L.activity, L.ts_ns)
    for r in runs[1:]:
        _same(runs[0], r)


def test_tuned_context_keeps_the_oracle_results():
    import torch
    from paper_2204_04898_b300 import autotune, pm4g
    L = synth.generate(synth.very_large_log(20000))
    cols = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (L.case_id, L.activity, L.ts_ns)]
    ctx = pm4g.pm4g_ctx_create(0)
    try:
        small = {"clb": (0, 6), "splits": (0, 4), "stream_warps": (0, 12), "stream_off": (0, 1),
                 "edge_table": (0, 1), "part1_items": (0, 4), "part2_items": (0,), "part_fbits": (0, 9)}
        choice = autotune.Tuner(cache_path="").tune_load(ctx, cols, L.n_activities, top_k=10, reps=1, space=small)
        assert set(choice) == set(autotune.LOAD_KNOBS)
        assert all(choice[k] in small[k] for k in choice)
        log = pm4g.pm4g_load_log(ctx, *cols, n_activities=L.n_activities)
        try:
            got = collect(pm4g, log, L.n_activities)
        finally:
            pm4g.pm4g_log_free(log)
        assert_same(got, oracle.summarize(L.case_id, L.activity, L.ts_ns, L.n_activities), L.case_id, L.activity,
                    L.ts_ns)
    finally:
        pm4g.pm4g_ctx_destroy(ctx)
