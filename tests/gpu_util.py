"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare its outputs with the oracle's, element by element (tolerance 0)."""

from __future__ import annotations

import numpy as np

import oracle


def to_device(log):
    import torch
    cols = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (log.case_id, log.activity, log.ts_ns)]
    attr = None if log.case_attr is None else torch.from_numpy(np.ascontiguousarray(log.case_attr)).cuda()
    return cols, attr


def gpu_run(pm4g, ctx, case_id, activity, ts_ns, n_activities, case_attr=None, device=True, export=True,
            top_k=-1):
    """Load a log through the C ABI and collect every output."""
    import torch
    if device:
        cols = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (case_id, activity, ts_ns)]
        attr = None if case_attr is None else torch.from_numpy(np.ascontiguousarray(case_attr)).cuda()
    else:
        cols = [np.ascontiguousarray(case_id, np.int32), np.ascontiguousarray(activity, np.int32),
                np.ascontiguousarray(ts_ns, np.int64)]
        attr = None if case_attr is None else np.ascontiguousarray(case_attr, np.int32)
    log = pm4g.pm4g_load_log(ctx, *cols, case_attr=attr, n_activities=n_activities)
    try:
        return collect(pm4g, log, n_activities, export=export, top_k=top_k), log
    except BaseException:
        pm4g.pm4g_log_free(log)
        raise


def collect(pm4g, log, n_activities, export=True, top_k=-1):
    out = {}
    out["info"] = pm4g.pm4g_log_info(log)
    out["dfg"] = pm4g.pm4g_dfg(log)
    out["perf"] = pm4g.pm4g_perf_dfg(log)
    out["start"], out["end"], out["freq"] = pm4g.pm4g_start_end(log, n_activities)
    out["var"] = pm4g.pm4g_variants(log, top_k=top_k, cases=True)
    if export:
        out["export"] = pm4g.pm4g_log_export(log)
    return out


def assert_same(got, R, case_id=None, activity=None, ts_ns=None, export=True, top_k=-1):
    """Bit-exact comparison of GPU outputs with an oracle Summary."""
    n_events, n_cases = got["info"]
    assert n_events == R.n_events and n_cases == R.n_cases
    d, p = got["dfg"], got["perf"]
    for name, g, w in (("src", d["src"], R.src), ("dst", d["dst"], R.dst), ("count", d["count"], R.count),
                       ("perf.src", p.src, R.src), ("perf.dst", p.dst, R.dst), ("perf.count", p.count, R.count),
                       ("sum_lo", p.sum_lo, R.sum_lo), ("sum_hi", p.sum_hi, R.sum_hi), ("min", p.min, R.min),
                       ("max", p.max, R.max)):
        assert np.array_equal(g, w), f"{name} differs"
    # means: same formula on the same integers, so identical bits
    assert np.array_equal(p.mean.view(np.uint64), R.mean.view(np.uint64)), "mean differs"
    assert np.array_equal(got["start"], R.start) and np.array_equal(got["end"], R.end)
    assert np.array_equal(got["freq"], R.freq)
    v = got["var"]
    assert v.n_variants == R.n_variants
    k = R.n_variants if top_k < 0 else min(top_k, R.n_variants)
    assert np.array_equal(v.count, R.var_count[:k]), "variant counts differ"
    assert np.array_equal(v.min_case, R.var_min_case[:k]), "variant smallest cases differ"
    assert np.array_equal(v.off, R.var_off[:k + 1]), "variant offsets differ"
    assert np.array_equal(v.acts, R.var_acts[:R.var_off[k]]), "variant sequences differ"
    assert np.array_equal(v.case_ids, R.case_ids), "case ids differ"
    assert np.array_equal(v.case_variant, R.case_variant), "case variants differ"
    if export and "export" in got:
        e = got["export"]
        rows = R.sorted_rows
        assert np.array_equal(e["row"], rows), "formatted order differs"
        assert np.array_equal(e["case_id"], np.asarray(case_id)[rows])
        assert np.array_equal(e["activity"], np.asarray(activity)[rows])
        assert np.array_equal(e["ts_ns"], np.asarray(ts_ns)[rows])


def check_log(pm4g, ctx, case_id, activity, ts_ns, A, case_attr=None, device=True, export=True, top_k=-1):
    R = oracle.summarize(case_id, activity, ts_ns, A)
    got, log = gpu_run(pm4g, ctx, case_id, activity, ts_ns, A, case_attr=case_attr, device=device,
                       export=export, top_k=top_k)
    try:
        assert_same(got, R, case_id, activity, ts_ns, export=export, top_k=top_k)
    finally:
        pm4g.pm4g_log_free(log)
    return R
