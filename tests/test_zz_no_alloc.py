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
