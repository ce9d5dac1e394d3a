"""Large activity alphabets against the CPU oracle, bit-exact.

Up to 4,096 activities the engine aggregates directly-follows pairs into a
global table dense over the A x A pairs; above that, into an open-addressing
table keyed by src * A + dst (Section 3: the DFG of large alphabets goes to a
hashed global table). A context option forces the hashed table at any size, so
both tables are checked on the same logs. All calls go through the C ABI.
"""

from dataclasses import replace

import numpy as np
import pytest

import oracle
import pm4g_synth as synth
from tests.gpu_util import assert_same, gpu_run

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


def _log(law, n_cases, n_activities):
    spec = replace(synth.WORKLOADS[law]().scaled(n_cases, law), n_activities=n_activities)
    return synth.generate(spec)


def _parity(pm4g, ctx, L, A):
    got, log = gpu_run(pm4g, ctx, L.case_id, L.activity, L.ts_ns, A)
    try:
        R = oracle.summarize(L.case_id, L.activity, L.ts_ns, A)
        assert_same(got, R, L.case_id, L.activity, L.ts_ns)
        return R
    finally:
        pm4g.pm4g_log_free(log)


@pytest.mark.parametrize("law", ["very_large_log", "large_log"])
def test_alphabet_4096(pm4g, ctx, law):
    """The largest dense table, above the shared-memory endpoint counters'
    2,048 (time-ordered and shuffled rows)."""
    L = _log(law, 30000, 4096)
    R = _parity(pm4g, ctx, L, 4096)
    assert R.n_edges > 4096  # more edges than the shared table holds


def test_alphabet_65536(pm4g, ctx):
    """The hashed global table, with the last activity following itself (the
    pair whose key is 2^32 - 1) and codes at both ends of the alphabet."""
    L = _log("very_large_log", 20000, 65536)
    n0 = int(L.case_id.max()) + 1
    extra_case = np.array([n0, n0, n0, n0 + 1, n0 + 1], np.int32)
    extra_act = np.array([65535, 65535, 0, 0, 65535], np.int32)
    t0 = int(L.ts_ns.max())
    extra_ts = np.array([t0 + 1, t0 + 2, t0 + 3, t0 + 4, t0 + 5], np.int64)
    case_id = np.concatenate([L.case_id, extra_case])
    act = np.concatenate([L.activity, extra_act])
    ts = np.concatenate([L.ts_ns, extra_ts])
    got, log = gpu_run(pm4g, ctx, case_id, act, ts, 65536)
    try:
        R = oracle.summarize(case_id, act, ts, 65536)
        assert_same(got, R, case_id, act, ts)
        assert ((R.src == 65535) & (R.dst == 65535)).any()
    finally:
        pm4g.pm4g_log_free(log)


@pytest.mark.parametrize("law", ["very_large_log", "large_log", "single_log"])
def test_forced_hashed_table(pm4g, law):
    """The hashed global table at small alphabets gives the dense table's
    results (the time-ordered law then takes the sorting segment pass)."""
    L = synth.generate(synth.WORKLOADS[law]().scaled(20000, law))
    ctx = pm4g.pm4g_ctx_create(0)
    try:
        pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_EDGE_TABLE, 1)
        _parity(pm4g, ctx, L, L.n_activities)
    finally:
        pm4g.pm4g_ctx_destroy(ctx)


def test_large_alphabet_drilldown_and_filter(pm4g, ctx):
    """Batched drill-down views and a filter of a 65,536-activity log: the
    drill-down index finds edge ids by searching the hashed table's keys."""
    import torch
    from tests.test_batch_drilldown import _check_batch, _random_specs
    spec = replace(synth.drilldown_log(4000), n_activities=65536)
    L = synth.generate(spec)
    cols = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (L.case_id, L.activity, L.ts_ns, L.case_attr)]
    log = pm4g.pm4g_load_log(ctx, *cols[:3], case_attr=cols[3], n_activities=65536)
    try:
        specs = _random_specs(L, np.random.default_rng(31), 12)
        B = pm4g.pm4g_batch_dfg(log, [s[0] for s in specs], [s[1] for s in specs], [s[2] for s in specs],
                                [s[3] for s in specs], var_top_k=3)
        _check_batch(B, L, specs, top_k=3)
        t0, t1 = int(L.ts_ns.min()), int(L.ts_ns.max())
        aset = np.arange(0, 4096, 5, dtype=np.int32)
        sub = pm4g.pm4g_filter(log, aset, t0, (t0 + t1) // 2, pm4g.TW_EVENTS)
        try:
            rows = oracle.filter_rows(L.case_id, L.activity, L.ts_ns, L.case_attr, 65536, aset, t0, (t0 + t1) // 2,
                                      oracle.TW_EVENTS)
            S = L.take(rows)
            R = oracle.summarize(S.case_id, S.activity, S.ts_ns, 65536)
            from tests.gpu_util import collect
            assert_same(collect(pm4g, sub, 65536, export=False), R, export=False)
        finally:
            pm4g.pm4g_log_free(sub)
    finally:
        pm4g.pm4g_log_free(log)


def test_alphabet_limits(pm4g, ctx):
    c = np.array([0, 0, 1], np.int32)
    t = np.array([1, 2, 3], np.int64)
    with pytest.raises(pm4g.Pm4gError) as e:
        pm4g.pm4g_load_log(ctx, c, np.array([0, 1, 2], np.int32), t, n_activities=65537)
    assert e.value.status == pm4g.EINVAL
    with pytest.raises(pm4g.Pm4gError) as e:
        pm4g.pm4g_load_log(ctx, c, np.array([0, 65536, 2], np.int32), t, n_activities=65536)
    assert e.value.status == pm4g.ERANGE
    # the eventually-follows graph's dense 65,536 x 65,536 table cannot fit: a clear error
    log = pm4g.pm4g_load_log(ctx, c, np.array([0, 65535, 2], np.int32), t, n_activities=65536)
    try:
        with pytest.raises(pm4g.Pm4gError) as e:
            pm4g.pm4g_efg(log)
        assert e.value.status == pm4g.ENOMEM
        d = pm4g.pm4g_perf_dfg(log)
        assert list(d.src) == [0] and list(d.dst) == [65535] and list(d.count) == [1]
    finally:
        pm4g.pm4g_log_free(log)
