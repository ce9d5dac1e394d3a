"""The allocation-free DFG entry point against the regular path.

pm4g_dfg_noalloc serves callers that cannot allocate device memory when they
need a summary (code under CUDA graph capture, serving processes with a fixed
memory budget, hosts whose device memory belongs to another framework's pool):
its only working memory is a fixed array inside the library, shared by all
calls. Two calls in a row, on different logs (the second smaller, so stale data
from the first would show), must each equal the regular C-ABI path exactly.
This file is collected last so that a run stopping at the first failure has
already run every other test."""

import numpy as np
import pytest

import pm4g_synth as synth

pytestmark = pytest.mark.gpu


def _dense_from_regular(pm4g, ctx, cols, A):
    log = pm4g.pm4g_load_log(ctx, *cols, n_activities=A)
    try:
        p = pm4g.pm4g_perf_dfg(log)
        s, e, _ = pm4g.pm4g_start_end(log, A)
    finally:
        pm4g.pm4g_log_free(log)
    cells = A * A
    want = {"count": np.zeros(cells, np.uint64), "sum_lo": np.zeros(cells, np.uint64),
            "sum_hi": np.zeros(cells, np.uint64), "min": np.full(cells, np.iinfo(np.uint64).max, np.uint64),
            "max": np.zeros(cells, np.uint64)}
    k = p.src.astype(np.int64) * A + p.dst
    for name, v in (("count", p.count), ("sum_lo", p.sum_lo), ("sum_hi", p.sum_hi), ("min", p.min),
                    ("max", p.max)):
        want[name][k] = v
    want["start"], want["end"] = s, e
    return want


def test_noalloc_matches_regular_path_on_two_calls_in_a_row():
    import torch
    from paper_2204_04898_b300 import pm4g

    ctx = pm4g.pm4g_ctx_create(0)
    try:
        for spec in (synth.large_log(8000), synth.very_large_log(3000)):
            L = synth.generate(spec)
            cols = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns)]
            got = pm4g.pm4g_dfg_noalloc(*cols, n_activities=L.n_activities)
            torch.cuda.synchronize()
            want = _dense_from_regular(pm4g, ctx, cols, L.n_activities)
            for name, w in want.items():
                g = got[name].cpu().numpy().view(np.uint64)
                assert np.array_equal(g, w), f"{spec.name}: {name} differs"
    finally:
        pm4g.pm4g_ctx_destroy(ctx)


def test_noalloc_rejects_oversized_input():
    import torch
    from paper_2204_04898_b300 import pm4g

    n = (1 << 18) + 1
    z = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(pm4g.Pm4gError) as e:
        pm4g.pm4g_dfg_noalloc(z, z, torch.zeros(n, dtype=torch.int64, device="cuda"), n_activities=1)
    assert e.value.status == pm4g.EINVAL


def test_captured_graph_replays_for_logs_of_any_size():
    """pm4g_dfg_noalloc_async captured once in a CUDA graph: replays on three
    logs of different sizes (the largest first, so stale data would show)
    each equal the regular path exactly."""
    import torch
    from paper_2204_04898_b300 import pm4g

    logs = [synth.generate(synth.large_log(n)) for n in (8000, 700, 3)]
    A = logs[0].n_activities
    g = pm4g.NoallocGraph(A)
    ctx = pm4g.pm4g_ctx_create(0)
    try:
        for L in logs:
            assert L.n_events <= pm4g.NOALLOC_MAX_EVENTS and L.n_activities == A
            got, status = g.run(L.case_id, L.activity, L.ts_ns)
            assert status == 0
            cols = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns)]
            want = _dense_from_regular(pm4g, ctx, cols, A)
            for name, w in want.items():
                assert np.array_equal(got[name].cpu().numpy().view(np.uint64), w), f"{L.n_events}: {name} differs"
    finally:
        pm4g.pm4g_ctx_destroy(ctx)


def test_captured_graph_reports_input_errors():
    """Input errors come back in the status word and no kernel reads or
    writes outside its arrays: an activity outside the alphabet (bit 0), a
    case longer than 512 events (bit 1), case ids spanning more than 2^18
    values (bit 2), an event count beyond the buffers (bit 3)."""
    import torch
    from paper_2204_04898_b300 import pm4g

    g = pm4g.NoallocGraph(4)
    ts = np.arange(10, dtype=np.int64)
    _, st = g.run(np.zeros(10, np.int32), np.array([0, 1, 2, 3, 4, 0, 1, 2, 3, 0], np.int32), ts)
    assert st & 1
    out, st = g.run(np.zeros(600, np.int32), np.zeros(600, np.int32), np.arange(600, dtype=np.int64))
    assert st == 2
    out, st = g.run(np.array([0, 300_000], np.int32), np.zeros(2, np.int32), np.arange(2, dtype=np.int64))
    assert st == 4 and int(out["count"].sum().item()) == 0
    with torch.cuda.stream(g.stream):
        g.n.fill_(pm4g.NOALLOC_MAX_EVENTS + 1)
        g.graph.replay()
    g.stream.synchronize()
    assert int(g.status.item()) == 8 and int(g.out["start"].sum().item()) == 0
    # and a good log afterwards is exact again
    out, st = g.run(np.array([5, 5, 6], np.int32), np.array([1, 2, 3], np.int32), np.array([10, 30, 5], np.int64))
    assert st == 0
    cnt = out["count"].cpu().numpy().reshape(4, 4)
    assert cnt[1, 2] == 1 and cnt.sum() == 1
    assert out["sum_lo"].cpu().numpy().reshape(4, 4)[1, 2] == 20
    assert list(out["start"].cpu().numpy()) == [0, 1, 0, 1] and list(out["end"].cpu().numpy()) == [0, 0, 1, 1]
