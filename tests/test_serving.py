"""Serving on the GPU: a resident log answers filter+DFG, variants and upload
requests through the continuous-batching server; every result is identical
alone (one request at a time) and in the mix (all submitted at once, batched
and overlapping), and matches the oracle."""

import numpy as np
import pytest

import oracle
import pm4g_synth as synth
from paper_2204_04898_b300.serve import GpuEngine, Request, Server

pytestmark = pytest.mark.gpu


def _same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        x, y = a[k], b[k]
        if isinstance(x, np.ndarray):
            assert x.dtype == y.dtype and np.array_equal(x.view(np.uint8), y.view(np.uint8)), k
        else:
            assert x == y, k


def test_alone_equals_mix_and_oracle():
    import torch
    from paper_2204_04898_b300 import pm4g
    L = synth.generate(synth.drilldown_log(8000))
    A = L.n_activities
    ctx = pm4g.pm4g_ctx_create(0)
    cols = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns, L.case_attr)]
    log = pm4g.pm4g_load_log(ctx, *cols[:3], case_attr=cols[3], n_activities=A)
    eng = GpuEngine(pm4g, 0, log, ctx, upload_slots=2)
    try:
        rng = np.random.default_rng(21)
        views = synth.drilldown_specs(L, n_views=40, lo_events=200, hi_events=L.n_events / 3)
        ups = [synth.generate(synth.large_log(n)) for n in (500, 3000, 20000)]

        def make():
            reqs = [Request("dfg", attr_set=v.attr_set, t_lo=v.t_lo, t_hi=v.t_hi, mode=int(rng.integers(0, 4)))
                    for v in views]
            reqs += [Request("variants", top_k=k) for k in (1, 10, 10)]
            reqs += [Request("upload", columns=(u.case_id, u.activity, u.ts_ns), n_activities=u.n_activities,
                             top_k=5) for u in ups]
            return reqs

        alone = make()
        srv = Server(eng, upload_slots=2)
        try:
            for r in alone:                       # one at a time
                srv.submit(r)
                assert r.done.wait(120)
                assert r.error is None, r.error
            rng = np.random.default_rng(21)
            mix = make()
            order = np.random.default_rng(22).permutation(len(mix))
            for i in order:                       # all at once, shuffled
                srv.submit(mix[i])
            for r in mix:
                assert r.done.wait(120)
                assert r.error is None, r.error
            assert max(srv.batches) > 1, "the mix must have been batched"
        finally:
            srv.close()
        for a, b in zip(alone, mix):
            _same(a.result, b.result)
        # a few against the oracle
        for r in alone[:6]:
            rows = oracle.filter_rows(L.case_id, L.activity, L.ts_ns, L.case_attr, A, r.attr_set, r.t_lo, r.t_hi,
                                      r.mode)
            R = oracle.summarize(L.case_id[rows], L.activity[rows], L.ts_ns[rows], A)
            got = r.result
            assert got["n_events"] == rows.shape[0] and got["n_cases"] == R.n_cases
            assert np.array_equal(got["count"], R.count) and np.array_equal(got["sum_lo"], R.sum_lo)
            assert np.array_equal(got["start"], R.start) and np.array_equal(got["freq"], R.freq)
        for r, u in zip(alone[-3:], ups):
            R = oracle.summarize(u.case_id, u.activity, u.ts_ns, u.n_activities)
            got = r.result
            assert got["n_events"] == u.n_events and got["n_cases"] == R.n_cases
            assert np.array_equal(got["count"], R.count) and np.array_equal(got["max"], R.max)
            assert np.array_equal(got["var_count"], R.var_count[:5])
        R = oracle.summarize(L.case_id, L.activity, L.ts_ns, A)
        v = alone[len(views) + 1].result
        assert v["n_variants"] == R.n_variants and np.array_equal(v["count"], R.var_count[:10])
    finally:
        eng.close()
        pm4g.pm4g_log_free(log)
        pm4g.pm4g_ctx_destroy(ctx)


def test_concurrent_contexts_in_threads():
    """Loads of differently sized logs (different bucket widths, table modes and
    shared-memory sizes) on two contexts from two threads at once give the
    results each gives alone."""
    import threading
    from paper_2204_04898_b300 import pm4g
    logs = [synth.generate(s) for s in (synth.single_log(3000), synth.large_log(30000), synth.very_large_log(20000),
                                        synth.drilldown_log(15000), synth.large_log(2000), synth.single_log(40000))]

    def summary(ctx, L):
        log = pm4g.pm4g_load_log(ctx, L.case_id, L.activity, L.ts_ns, n_activities=L.n_activities)
        try:
            p = pm4g.pm4g_perf_dfg(log)
            v = pm4g.pm4g_variants(log, top_k=20)
            return (p.src.tobytes(), p.count.tobytes(), p.sum_lo.tobytes(), p.max.tobytes(), v.count.tobytes(),
                    v.acts.tobytes())
        finally:
            pm4g.pm4g_log_free(log)

    ctxs = [pm4g.pm4g_ctx_create(0) for _ in range(2)]
    try:
        alone = [summary(ctxs[0], L) for L in logs]
        got = [[None] * len(logs) for _ in range(2)]
        errs = []

        def worker(t):
            try:
                for rep in range(3):
                    for i in (range(len(logs)) if t == 0 else reversed(range(len(logs)))):
                        got[t][i] = summary(ctxs[t], logs[i])
            except BaseException as e:
                errs.append(e)

        th = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
        for x in th:
            x.start()
        for x in th:
            x.join(600)
        assert not errs, errs
        for t in range(2):
            for i in range(len(logs)):
                assert got[t][i] == alone[i], (t, i)
    finally:
        for c in ctxs:
            pm4g.pm4g_ctx_destroy(c)
