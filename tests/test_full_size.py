"""Parity at the full sizes of the benchmarked workloads, in the launch
configuration the benchmark times: device-resident columns, a context on its
own stream, top-1000 variants.

- Large log (1M cases, about 20.6M events): every output against the oracle
  run on the whole log, bit-exact; the eventually-follows graph against the
  oracle on 16 groups of cases.
- Very large log (10M cases, about 206.6M events): the summaries, the
  formatted order, the whole variant table with every case's rank, the
  eventually-follows graph and the benchmark's filters on derived results,
  bit-exact against the oracle run on 64 groups of cases (tests/case_groups.py
  states why the groups fix the whole-log result), plus the invariants of the
  definitions against plain counts of the input.
- Drill-down (4,096 views of the 100M-event log in one batched call, plus
  four edge views: the largest attribute value alone, every value, an empty
  window and an absent value): the invariants of the definitions on every
  view; the view of every value equals the log's own summary; the other edge
  views and 32 more (the largest, the smallest and random ones) bit-exact
  against the oracle's filter and summary.
- Serving (the resident 10M-case log with attributes, views, variants and uploads of about
  10k, 1M and 20M events): alone equals the shuffled mix; uploads and 8 views bit-exact
  against the oracle.
"""

from types import SimpleNamespace

import numpy as np
import pytest

import oracle
import pm4g_synth as synth

from .case_groups import (check_efg_by_case_groups, check_filter_by_case_groups, check_summaries_by_case_groups,
                          pool_map)
from .gpu_util import assert_same, collect

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm4g():
    from paper_2204_04898_b300 import pm4g as m
    return m


def _resident(pm4g, L, with_attr=False):
    """The log's columns on the device and a context on its own stream, as
    the benchmark sets them up."""
    import torch
    stream = torch.cuda.Stream()
    ctx = pm4g.pm4g_ctx_create(0, stream=stream.cuda_stream)
    cols = [L.case_id, L.activity, L.ts_ns] + ([L.case_attr] if with_attr else [])
    dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in cols]
    torch.cuda.synchronize()
    log = pm4g.pm4g_load_log(ctx, *dev[:3], case_attr=dev[3] if with_attr else None, n_activities=L.n_activities)
    return SimpleNamespace(L=L, log=log, ctx=ctx, dev=dev, stream=stream)


def _release(pm4g, r):
    pm4g.pm4g_log_free(r.log)
    pm4g.pm4g_ctx_destroy(r.ctx)
    r.dev.clear()


def _per_activity(src, dst, count, A):
    out_deg = np.bincount(src, weights=count.astype(np.float64), minlength=A)
    in_deg = np.bincount(dst, weights=count.astype(np.float64), minlength=A)
    return out_deg.astype(np.uint64), in_deg.astype(np.uint64)


def test_large_log_whole(pm4g):
    L = synth.generate(synth.large_log())
    A = L.n_activities
    r = _resident(pm4g, L)
    try:
        R = oracle.summarize(L.case_id, L.activity, L.ts_ns, A)
        for k in (1000, -1):
            got = collect(pm4g, r.log, A, export=(k == 1000), top_k=k)
            assert_same(got, R, L.case_id, L.activity, L.ts_ns, export=(k == 1000), top_k=k)
        check_efg_by_case_groups(L.case_id, L.activity, L.ts_ns, A, pm4g.pm4g_efg(r.log), G=16)
    finally:
        _release(pm4g, r)


@pytest.fixture(scope="module")
def very_large(pm4g):
    r = _resident(pm4g, synth.generate(synth.very_large_log()))
    yield r
    _release(pm4g, r)


def test_very_large_log_summaries(pm4g, very_large):
    L, log = very_large.L, very_large.log
    A = L.n_activities
    info = pm4g.pm4g_log_info(log)
    d = pm4g.pm4g_dfg(log)
    perf = pm4g.pm4g_perf_dfg(log)
    start, end, freq = pm4g.pm4g_start_end(log, A)
    top = pm4g.pm4g_variants(log, top_k=1000)
    var = pm4g.pm4g_variants(log, top_k=-1, cases=True)
    # invariants of the definitions, against plain counts of the input
    per_case = np.bincount(L.case_id)
    C = int(np.count_nonzero(per_case))
    assert info == (L.n_events, C)
    assert np.array_equal(freq, np.bincount(L.activity, minlength=A).astype(np.uint64))
    for k in ("src", "dst", "count"):
        assert np.array_equal(d[k], getattr(perf, k))
    assert int(perf.count.sum()) == L.n_events - C
    assert int(start.sum()) == C and int(end.sum()) == C
    out_deg, in_deg = _per_activity(perf.src, perf.dst, perf.count, A)
    assert np.array_equal(out_deg + end, freq) and np.array_equal(in_deg + start, freq)
    assert int(var.count.sum()) == C
    k = min(1000, var.n_variants)
    assert top.n_variants == var.n_variants
    assert np.array_equal(top.count, var.count[:k]) and np.array_equal(top.min_case, var.min_case[:k])
    assert np.array_equal(top.off, var.off[:k + 1]) and np.array_equal(top.acts, var.acts[:var.off[k]])
    # the formatted log carries the input's values
    ex = pm4g.pm4g_log_export(log)
    rows = ex["row"]
    assert np.array_equal(ex["case_id"], L.case_id[rows])
    assert np.array_equal(ex["activity"], L.activity[rows])
    assert np.array_equal(ex["ts_ns"], L.ts_ns[rows])
    check_summaries_by_case_groups(L.case_id, L.activity, L.ts_ns, A, perf, start, end, freq, info, var,
                                   rows=rows, rows_case=ex["case_id"], G=64)


def test_very_large_log_efg(pm4g, very_large):
    L = very_large.L
    F = pm4g.pm4g_efg(very_large.log)
    per_case = np.bincount(L.case_id).astype(np.int64)
    assert int(F.count.sum()) == int((per_case * (per_case - 1) // 2).sum())
    check_efg_by_case_groups(L.case_id, L.activity, L.ts_ns, L.n_activities, F, G=64)


def _filter_mix(pm4g, log, A):
    """The benchmark's filters, with their arguments from the log's own
    summaries: the 20 most frequent paths, cases of at least the median size,
    durations within the quartiles, the 3 most frequent end activities, the 5
    rarest activities, the 10 most frequent variants."""
    perf = pm4g.pm4g_perf_dfg(log)
    _, end, freq = pm4g.pm4g_start_end(log, A)
    e = pm4g.pm4g_log_export(log)
    starts = np.flatnonzero(np.r_[True, e["case_id"][1:] != e["case_id"][:-1]])
    ends = np.r_[starts[1:], e["case_id"].size] - 1
    lens = ends - starts + 1
    dur = e["ts_ns"][ends] - e["ts_ns"][starts]
    del e
    order = np.argsort(-perf.count.astype(np.int64), kind="stable")[:20]
    return [
        ("paths", {"pairs": [(int(perf.src[i]), int(perf.dst[i])) for i in order]}),
        ("cases", {"min_events": int(np.median(lens))}),
        ("cases", {"min_duration": int(np.percentile(dur, 25)), "max_duration": int(np.percentile(dur, 75))}),
        ("cases", {"end_set": [int(a) for a in np.argsort(-end.astype(np.int64))[:3]]}),
        ("cases", {"act_set": [int(a) for a in np.argsort(freq.astype(np.int64))[:5]]}),
        ("cases", {"variant_set": list(range(10))}),
    ]


def test_very_large_log_filters(pm4g, very_large):
    L, log = very_large.L, very_large.log
    A = L.n_activities
    var = pm4g.pm4g_variants(log, top_k=10)
    for kind, kw in _filter_mix(pm4g, log, A):
        f = pm4g.pm4g_filter_paths(log, **kw) if kind == "paths" else pm4g.pm4g_filter_cases(log, **kw)
        try:
            info = pm4g.pm4g_log_info(f)
            perf = pm4g.pm4g_perf_dfg(f)
            start, end, freq = pm4g.pm4g_start_end(f, A)
        finally:
            pm4g.pm4g_log_free(f)
        if kw.get("variant_set"):
            # ranks are global: the kept cases are those of the 10 top variants
            lens = np.diff(var.off)
            assert info == (int((var.count * lens.astype(np.uint64)).sum()), int(var.count.sum()))
            continue
        check_filter_by_case_groups(L.case_id, L.activity, L.ts_ns, A, kind, kw, perf, start, end, freq, info,
                                    G=64)


def test_drilldown_views(pm4g):
    L = synth.generate(synth.drilldown_log())
    A = L.n_activities
    views = synth.drilldown_specs(L, n_views=4096)
    sets = [v.attr_set for v in views]
    lo = [v.t_lo for v in views]
    hi = [v.t_hi for v in views]
    # edge views, pinned below with the sample: the largest attribute value
    # alone over the whole log; every attribute value over the whole log; a
    # window before the first event (empty); an attribute value no case has
    # (empty)
    t0, t1 = int(L.ts_ns.min()), int(L.ts_ns.max())
    amax = int(L.case_attr.max())
    missing = int(np.setdiff1d(np.arange(amax + 2), L.case_attr)[-1])
    edge = [(np.array([amax], np.int32), t0, t1), (np.unique(L.case_attr).astype(np.int32), t0, t1),
            (np.array([amax], np.int32), t0 - 10, t0 - 1), (np.array([missing], np.int32), t0, t1)]
    for a_, l_, h_ in edge:
        sets.append(a_)
        lo.append(l_)
        hi.append(h_)
    Q = len(sets)
    r = _resident(pm4g, L, with_attr=True)
    try:
        buf = pm4g.BatchBuffers(Q, A, 0)
        bspec = pm4g.BatchSpec(sets, lo, hi, [pm4g.TW_EVENTS] * Q)
        B = pm4g.pm4g_batch_dfg(r.log, out=buf, var_top_k=1000, spec=bspec)
        # the whole log's own summary, for the view of every attribute value
        whole_perf = pm4g.pm4g_perf_dfg(r.log)
        whole_se = pm4g.pm4g_start_end(r.log, A)
        whole_var = pm4g.pm4g_variants(r.log, top_k=1000)
    finally:
        _release(pm4g, r)
    # invariants on every view
    eo = B.edge_off.astype(np.int64)
    view = np.repeat(np.arange(Q), np.diff(eo))
    cs = np.r_[0, np.cumsum(B.count.astype(np.int64))]
    assert np.array_equal(cs[eo[1:]] - cs[eo[:-1]], B.n_events - B.n_cases)
    assert np.array_equal(B.start.sum(1).astype(np.int64), B.n_cases)
    assert np.array_equal(B.end.sum(1).astype(np.int64), B.n_cases)
    assert np.array_equal(B.freq.sum(1).astype(np.int64), B.n_events)
    out_deg, in_deg = _per_activity(view * A + B.src, view * A + B.dst, B.count, Q * A)
    assert np.array_equal(out_deg.reshape(Q, A) + B.end, B.freq)
    assert np.array_equal(in_deg.reshape(Q, A) + B.start, B.freq)
    assert np.all(B.min <= B.max)
    vo = B.var_off.astype(np.int64)
    vc = np.r_[0, np.cumsum(B.var_count.astype(np.int64))]
    per_view = vc[vo[1:]] - vc[vo[:-1]]
    assert np.all(per_view <= B.n_cases)
    whole = B.n_variants <= 1000
    assert np.array_equal(per_view[whole], B.n_cases[whole])
    # a sample of views, bit-exact
    by_size = np.argsort(B.n_events, kind="stable")
    rng = np.random.default_rng(2204)
    pick = sorted(set(by_size[:4].tolist()) | set(by_size[-4:].tolist()) |
                  set(rng.choice(Q, 24, replace=False).tolist()) | {Q - 4, Q - 2, Q - 1})
    assert B.n_events[Q - 2] == 0 and B.n_events[Q - 1] == 0  # the empty edge views
    # every attribute value over the whole log: the log's own summary (the
    # single-log pass, against the oracle in the tests above)
    w = Q - 3
    assert B.n_events[w] == L.n_events
    sw = B.sub(w)
    for name in ("src", "dst", "count", "sum_lo", "sum_hi", "min", "max"):
        assert np.array_equal(sw[name], getattr(whole_perf, name)), f"whole-log view: {name}"
    assert np.array_equal(sw["mean"].view(np.uint64), whole_perf.mean.view(np.uint64))
    for name, x in zip(("start", "end", "freq"), whole_se):
        assert np.array_equal(getattr(B, name)[w], x), f"whole-log view: {name}"
    a, b = int(B.var_off[w]), int(B.var_off[w + 1])
    assert B.n_variants[w] == whole_var.n_variants
    assert np.array_equal(B.var_count[a:b], whole_var.count) and np.array_equal(B.var_min_case[a:b],
                                                                                 whole_var.min_case)

    def one(i):
        # The oracle filters the events of the cases whose attribute is in the
        # view's set (the attribute is a case's, so no kept event is left out).
        pre = np.flatnonzero(np.isin(L.case_attr, sets[i]))
        rows = pre[oracle.filter_rows(L.case_id[pre], L.activity[pre], L.ts_ns[pre], L.case_attr[pre], A, sets[i],
                                      lo[i], hi[i], pm4g.TW_EVENTS)]
        R = oracle.summarize(L.case_id[rows], L.activity[rows], L.ts_ns[rows], A)
        assert B.n_events[i] == rows.shape[0] and B.n_cases[i] == R.n_cases, f"view {i}: sizes"
        s = B.sub(i)
        for name in ("src", "dst", "count", "sum_lo", "sum_hi", "min", "max"):
            assert np.array_equal(s[name], getattr(R, name)), f"view {i}: {name} differs"
        assert np.array_equal(s["mean"].view(np.uint64), R.mean.view(np.uint64)), f"view {i}: mean differs"
        for name in ("start", "end", "freq"):
            assert np.array_equal(getattr(B, name)[i], getattr(R, name)), f"view {i}: {name} differs"
        assert B.n_variants[i] == R.n_variants, f"view {i}: n_variants"
        k = min(1000, R.n_variants)
        a, b = int(vo[i]), int(vo[i + 1])
        assert b - a == k
        assert np.array_equal(B.var_count[a:b], R.var_count[:k]), f"view {i}: variant counts"
        assert np.array_equal(B.var_min_case[a:b], R.var_min_case[:k]), f"view {i}: variant smallest cases"
        so = B.var_seq_off[a:b + 1].astype(np.int64)
        assert np.array_equal(so - so[0], R.var_off[:k + 1]), f"view {i}: variant lengths"
        assert np.array_equal(B.var_acts[so[0]:so[-1]], R.var_acts[:R.var_off[k]]), f"view {i}: variant sequences"
        return rows.shape[0]

    assert sum(pool_map(one, pick)) == int(B.n_events[pick].sum())


def _same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        x, y = a[k], b[k]
        if isinstance(x, np.ndarray):
            assert x.dtype == y.dtype and np.array_equal(x.view(np.uint8), y.view(np.uint8)), k
        else:
            assert x == y, k


def test_serving_full_size(pm4g):
    """The serving workload at full size: a resident 10M-case log with case
    attributes answers filter+DFG views, top-10 variants and uploads of about
    10k, 1M and 20M events; every result is the same alone and in the mix,
    and matches the oracle (views, uploads) or the plain call (variants)."""
    from paper_2204_04898_b300.serve import GpuEngine, Request, Server
    L = synth.generate(synth.serving_log())
    A = L.n_activities
    views = synth.drilldown_specs(L, n_views=48, seed=20220417)
    ups = [synth.generate(synth.very_large_log(c).scaled(c, f"upload{c}")) for c in (500, 50_000, 1_000_000)]
    r = _resident(pm4g, L, with_attr=True)
    eng = GpuEngine(pm4g, 0, r.log, r.ctx, upload_slots=2)
    try:
        def make():
            reqs = [Request("dfg", attr_set=v.attr_set, t_lo=v.t_lo, t_hi=v.t_hi, mode=pm4g.TW_EVENTS) for v in views]
            reqs += [Request("variants", top_k=10) for _ in range(4)]
            reqs += [Request("upload", columns=(u.case_id, u.activity, u.ts_ns), n_activities=u.n_activities,
                             top_k=10) for u in ups]
            return reqs

        srv = Server(eng, upload_slots=2)
        try:
            alone = make()
            for q in alone:
                srv.submit(q)
                assert q.done.wait(300)
                assert q.error is None, q.error
            mix = make()
            for i in np.random.default_rng(23).permutation(len(mix)):
                srv.submit(mix[i])
            for q in mix:
                assert q.done.wait(300)
                assert q.error is None, q.error
            assert max(srv.batches) > 1, "the mix must have been batched"
        finally:
            srv.close()
        for a, b in zip(alone, mix):
            _same(a.result, b.result)
        plain = pm4g.pm4g_variants(r.log, top_k=10)
        for q in alone[len(views):len(views) + 4]:
            v = q.result
            assert v["n_variants"] == plain.n_variants
            for k in ("count", "min_case", "off", "acts"):
                assert np.array_equal(v[k], getattr(plain, k))
    finally:
        eng.close()
        _release(pm4g, r)

    def check(job):
        kind, i = job
        if kind == "dfg":
            q = alone[i]
            pre = np.flatnonzero(np.isin(L.case_attr, q.attr_set))
            rows = pre[oracle.filter_rows(L.case_id[pre], L.activity[pre], L.ts_ns[pre], L.case_attr[pre], A,
                                          q.attr_set, q.t_lo, q.t_hi, q.mode)]
            R = oracle.summarize(L.case_id[rows], L.activity[rows], L.ts_ns[rows], A)
            n_events = rows.shape[0]
        else:
            q, u = alone[len(views) + 4 + i], ups[i]
            R = oracle.summarize(u.case_id, u.activity, u.ts_ns, u.n_activities)
            n_events = u.n_events
        got = q.result
        assert got["n_events"] == n_events and got["n_cases"] == R.n_cases, f"{job}: sizes"
        for name in ("src", "dst", "count", "sum_lo", "sum_hi", "min", "max", "start", "end", "freq"):
            assert np.array_equal(got[name], getattr(R, name)), f"{job}: {name} differs"
        assert np.array_equal(got["mean"].view(np.uint64), R.mean.view(np.uint64)), f"{job}: mean differs"
        if kind == "upload":
            k = min(10, R.n_variants)
            assert got["n_variants"] == R.n_variants
            assert np.array_equal(got["var_count"], R.var_count[:k])
            assert np.array_equal(got["var_min_case"], R.var_min_case[:k])
            assert np.array_equal(got["var_off"], R.var_off[:k + 1])
            assert np.array_equal(got["var_acts"], R.var_acts[:R.var_off[k]])

    pool_map(check, [("upload", i) for i in range(len(ups))] + [("dfg", i) for i in range(0, len(views), 6)])
