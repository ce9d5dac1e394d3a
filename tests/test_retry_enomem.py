"""Requests that run out of device memory part way through their allocations,
through the context's allocator hook: every point of failure is tried, from a
request's first allocation on. The failed call returns PM4G_ENOMEM, the same
request on the same log then gives the result a fresh log gives, and once the
log is freed no buffer of the hook is left (a buffer the log already held is
given back before it is allocated again; an array that a failed call left
unfilled is never taken as formed)."""

import dataclasses

import numpy as np
import pytest

import pm4g_synth as synth

pytestmark = pytest.mark.gpu

KINDS = ["variants", "filter_window", "filter_cases", "filter_paths", "efg", "batch"]
LOG_KINDS = {"filter_window", "filter_cases", "filter_paths"}


@pytest.fixture(scope="module")
def pm4g():
    from paper_2204_04898_b300 import pm4g as m
    return m


class Hook:
    """Device memory from torch's pool; after `budget` more allocations every
    request fails. The library frees in stream order and this pool reuses
    memory at once, so a free waits for the device first."""

    def __init__(self):
        import torch
        self.torch = torch
        self.budget = None
        self.live = {}

    def alloc(self, nbytes, stream):
        if self.budget is not None:
            if self.budget == 0:
                return 0
            self.budget -= 1
        t = self.torch.empty(nbytes, dtype=self.torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr, nbytes, stream):
        self.torch.cuda.synchronize()
        self.live.pop(ptr, None)


def _flat(x):
    if dataclasses.is_dataclass(x):
        return [(f.name, getattr(x, f.name)) for f in dataclasses.fields(x)]
    if isinstance(x, tuple):
        return [(str(i), v) for i, v in enumerate(x)]
    return [("value", x)]


def _same(a, b, where="result"):
    fa, fb = _flat(a), _flat(b)
    assert [n for n, _ in fa] == [n for n, _ in fb], where
    for (n, va), (_, vb) in zip(fa, fb):
        w = f"{where}.{n}"
        if va is None or vb is None:
            assert va is None and vb is None, w
        elif isinstance(va, np.ndarray):
            assert va.dtype == vb.dtype and va.shape == vb.shape, w
            assert np.array_equal(va, vb, equal_nan=va.dtype.kind == "f"), w
        elif dataclasses.is_dataclass(va) or isinstance(va, tuple):
            _same(va, vb, w)
        else:
            assert va == vb, w


def _request(pm4g, kind, log, ctx_data):
    if kind == "variants":
        return pm4g.pm4g_variants(log, top_k=-1, cases=True)
    if kind == "filter_window":
        return pm4g.pm4g_filter(log, None, ctx_data["t_lo"], ctx_data["t_hi"], pm4g.TW_CASES_CONTAINED)
    if kind == "filter_cases":
        return pm4g.pm4g_filter_cases(log, min_events=3)
    if kind == "filter_paths":
        return pm4g.pm4g_filter_paths(log, ctx_data["pairs"])
    if kind == "efg":
        return pm4g.pm4g_efg(log)
    return pm4g.pm4g_batch_dfg(log, spec=ctx_data["spec"], var_top_k=5)


def _materialise(pm4g, kind, raw, A):
    """A plain value of a request's result (a returned log's summaries, the
    log then freed)."""
    if kind not in LOG_KINDS:
        return raw
    try:
        return (pm4g.pm4g_log_info(raw), pm4g.pm4g_perf_dfg(raw), pm4g.pm4g_start_end(raw, A),
                pm4g.pm4g_variants(raw, top_k=-1))
    finally:
        pm4g.pm4g_log_free(raw)


@pytest.mark.parametrize("kind", KINDS)
def test_retry_after_enomem(pm4g, kind):
    hook = Hook()
    torch = hook.torch
    L = synth.generate(synth.drilldown_log(3000))
    A = L.n_activities
    cols = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns, L.case_attr)]
    ctx = pm4g.pm4g_ctx_create(0, allocator=(hook.alloc, hook.free))
    try:
        def load():
            return pm4g.pm4g_load_log(ctx, *cols[:3], case_attr=cols[3], n_activities=A)

        lo, hi = (int(v) for v in np.quantile(L.ts_ns, [0.2, 0.8]))
        vals = np.unique(L.case_attr)
        data = {"t_lo": lo, "t_hi": hi,
                "spec": pm4g.BatchSpec([[], vals[:1], vals[1:4], []], [lo, lo, -2**63, lo], [hi, hi, 2**63 - 1, hi],
                                       [pm4g.TW_CASES_CONTAINED, pm4g.TW_EVENTS, pm4g.TW_NONE,
                                        pm4g.TW_CASES_INTERSECTING])}
        log = load()
        try:
            d = pm4g.pm4g_perf_dfg(log)
            data["pairs"] = [(int(d.src[0]), int(d.dst[0])), (int(d.src[-1]), int(d.dst[-1]))]
            expected = _materialise(pm4g, kind, _request(pm4g, kind, log, data), A)
        finally:
            pm4g.pm4g_log_free(log)
        torch.cuda.synchronize()
        assert not hook.live
        failed = 0
        done = False
        for k in range(400):
            log = load()
            try:
                hook.budget = k
                try:
                    raw = _request(pm4g, kind, log, data)
                    done = True
                except pm4g.Pm4gError as e:
                    assert e.status == pm4g.ENOMEM, e
                    failed += 1
                hook.budget = None
                if done:
                    _same(_materialise(pm4g, kind, raw, A), expected)
                _same(_materialise(pm4g, kind, _request(pm4g, kind, log, data), A), expected)
            finally:
                hook.budget = None
                pm4g.pm4g_log_free(log)
            torch.cuda.synchronize()
            assert not hook.live, f"{len(hook.live)} device buffers left after a failure at allocation {k}"
            if done:
                break
        assert done and failed >= 2, (done, failed)
    finally:
        pm4g.pm4g_ctx_destroy(ctx)
