"""The multi-GPU merge fed by the CUDA path: a log is split into case-disjoint
shards by `shard_of`, every shard is loaded and summarised by the engine on
the one GPU (as each rank of a sharded run would on its own GPU), the
engine's outputs (128-bit sums as lo/hi words, the full variant tables and
every case's variant rank) go through `ShardSummary.from_arrays` and `merge`,
and the result must equal the oracle's whole-log summary exactly."""

import numpy as np
import pytest

import oracle
import pm4g_synth as synth
from paper_2204_04898_b300.merge import ShardSummary, merge, shard_of
from tests.test_merge_gloo import _check

pytestmark = pytest.mark.gpu


def _engine_summary(pm4g, ctx, L, rows):
    import torch
    cols = [torch.from_numpy(np.ascontiguousarray(x[rows])).cuda() for x in (L.case_id, L.activity, L.ts_ns)]
    log = pm4g.pm4g_load_log(ctx, *cols, n_activities=L.n_activities)
    try:
        p = pm4g.pm4g_perf_dfg(log)
        st, en, fr = pm4g.pm4g_start_end(log, L.n_activities)
        v = pm4g.pm4g_variants(log, top_k=-1, cases=True)
        assert v.count.shape[0] == v.n_variants  # the full table: merging needs every variant
        return ShardSummary.from_arrays(L.n_activities, p.src, p.dst, p.count, p.sum_lo, p.sum_hi, p.min, p.max,
                                        st, en, fr, v.count, v.min_case, v.off, v.acts, v.case_ids,
                                        v.case_variant)
    finally:
        pm4g.pm4g_log_free(log)


@pytest.mark.parametrize("law,k", [("very_large_log", 2), ("large_log", 3), ("single_log", 4)])
def test_engine_shards_merge_to_whole_log(law, k):
    from paper_2204_04898_b300 import pm4g
    L = synth.generate(synth.WORKLOADS[law]().scaled(6000, law))
    ctx = pm4g.pm4g_ctx_create(0)
    try:
        sh = shard_of(L.case_id, k)
        parts = [_engine_summary(pm4g, ctx, L, np.nonzero(sh == r)[0]) for r in range(k)]
    finally:
        pm4g.pm4g_ctx_destroy(ctx)
    _check(merge(parts), oracle.summarize(L.case_id, L.activity, L.ts_ns, L.n_activities))


def test_engine_shards_merge_with_sums_beyond_64_bits():
    """Two shards whose edge sums each pass 2^64, so the merged sums carry the
    engine's high words."""
    from paper_2204_04898_b300 import pm4g
    n = 4000
    case_id = np.repeat(np.arange(n, dtype=np.int32), 2)
    act = np.tile(np.array([0, 1], np.int32), n)
    ts = np.zeros(2 * n, np.int64)
    ts[1::2] = (1 << 62) + np.arange(n, dtype=np.int64)  # each pair lasts about 2^62 ns
    ctx = pm4g.pm4g_ctx_create(0)

    class _L:
        pass
    L = _L()
    L.case_id, L.activity, L.ts_ns, L.n_activities = case_id, act, ts, 2
    try:
        sh = shard_of(case_id, 2)
        parts = [_engine_summary(pm4g, ctx, L, np.nonzero(sh == r)[0]) for r in range(2)]
    finally:
        pm4g.pm4g_ctx_destroy(ctx)
    assert all(p.edges[(0, 1)][1] >= (1 << 64) for p in parts)
    _check(merge(parts), oracle.summarize(case_id, act, ts, 2))
