"""Batched drill-down (pm4g_batch_dfg) against the CPU oracle, bit-exact: for
every sub-log of a batch, the oracle filters the rows (attribute set, window,
mode) and summarises the sub-log; the batch's sizes, edges (count, 128-bit
sum, min, max, mean bits) and start/end/freq rows must equal it. All calls go
through the C ABI."""

import numpy as np
import pytest

import oracle
import pm4g_synth as synth

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


def _load(pm4g, ctx, L, with_attr=True):
    import torch
    cols = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (L.case_id, L.activity, L.ts_ns)]
    attr = torch.from_numpy(np.ascontiguousarray(L.case_attr)).cuda() if with_attr else None
    return pm4g.pm4g_load_log(ctx, *cols, case_attr=attr, n_activities=L.n_activities)


def _check_batch(B, L, specs, with_attr=True, top_k=0):
    A = L.n_activities
    assert B.edge_off.shape[0] == len(specs) + 1
    for i, (aset, lo, hi, mode) in enumerate(specs):
        rows = oracle.filter_rows(L.case_id, L.activity, L.ts_ns, L.case_attr if with_attr else None, A,
                                  aset, lo, hi, mode)
        R = oracle.summarize(L.case_id[rows], L.activity[rows], L.ts_ns[rows], A)
        assert B.n_events[i] == rows.shape[0], f"sub-log {i}: n_events"
        assert B.n_cases[i] == R.n_cases, f"sub-log {i}: n_cases"
        s = B.sub(i)
        for name, got, want in (("src", s["src"], R.src), ("dst", s["dst"], R.dst), ("count", s["count"], R.count),
                                ("sum_lo", s["sum_lo"], R.sum_lo), ("sum_hi", s["sum_hi"], R.sum_hi),
                                ("min", s["min"], R.min), ("max", s["max"], R.max)):
            assert np.array_equal(got, want), f"sub-log {i}: {name} differs"
        assert np.array_equal(s["mean"].view(np.uint64), R.mean.view(np.uint64)), f"sub-log {i}: mean"
        assert np.array_equal(B.start[i], R.start), f"sub-log {i}: start"
        assert np.array_equal(B.end[i], R.end), f"sub-log {i}: end"
        assert np.array_equal(B.freq[i], R.freq), f"sub-log {i}: freq"
        if top_k:
            assert B.n_variants[i] == R.n_variants, f"sub-log {i}: n_variants"
            k = R.n_variants if top_k < 0 else min(top_k, R.n_variants)
            cnt, mnc, seqs = B.sub_variants(i)
            assert np.array_equal(cnt, R.var_count[:k]), f"sub-log {i}: variant counts"
            assert np.array_equal(mnc, R.var_min_case[:k]), f"sub-log {i}: variant min case"
            assert seqs == R.variant_seqs()[:k], f"sub-log {i}: variant sequences"


def _random_specs(L, rng, n, max_attrs=200):
    t0, t1 = int(L.ts_ns.min()), int(L.ts_ns.max())
    specs = []
    for _ in range(n):
        k = int(rng.integers(0, max_attrs))
        aset = rng.integers(-5, 4100, k).astype(np.int32)  # values outside the log's range too
        if k and rng.random() < 0.3:
            aset = np.concatenate([aset, aset[: k // 2]])  # repeats
        lo = t0 + int(rng.uniform(-0.1, 0.8) * (t1 - t0))
        hi = lo + int(rng.uniform(-0.05, 0.7) * (t1 - t0))  # sometimes hi < lo
        specs.append((aset, lo, hi, int(rng.integers(0, 4))))
    return specs


def _run(pm4g, log, specs, top_k=0):
    return pm4g.pm4g_batch_dfg(log, [s[0] for s in specs], [s[1] for s in specs], [s[2] for s in specs],
                               [s[3] for s in specs], var_top_k=top_k)


def test_batch_random_subsets(pm4g, ctx):
    L = synth.generate(synth.drilldown_log(8000))
    log = _load(pm4g, ctx, L)
    try:
        t0, t1 = int(L.ts_ns.min()), int(L.ts_ns.max())
        specs = [(np.empty(0, np.int32), t0, t1, m) for m in range(4)]       # whole log, every mode
        specs += [(np.empty(0, np.int32), t1 + 1, t1 + 10, 1)]               # window after the log
        specs += [(np.array([5000], np.int32), t0, t1, 0)]                    # absent attribute
        specs += _random_specs(L, np.random.default_rng(11), 60)
        _check_batch(_run(pm4g, log, specs), L, specs)
    finally:
        pm4g.pm4g_log_free(log)


def test_batch_equals_plain_filter_calls(pm4g, ctx):
    """The batch gives what pm4g_filter + the DFG queries give, sub-log by sub-log."""
    L = synth.generate(synth.drilldown_log(5000))
    log = _load(pm4g, ctx, L)
    try:
        specs = _random_specs(L, np.random.default_rng(12), 12)
        B = _run(pm4g, log, specs)
        for i, (aset, lo, hi, mode) in enumerate(specs):
            f = pm4g.pm4g_filter(log, np.unique(aset), lo, hi, mode)
            try:
                p = pm4g.pm4g_perf_dfg(f)
                st, en, fr = pm4g.pm4g_start_end(f, L.n_activities)
                s = B.sub(i)
                assert pm4g.pm4g_log_info(f) == (B.n_events[i], B.n_cases[i])
                for k in ("src", "dst", "count", "sum_lo", "sum_hi", "min", "max"):
                    assert np.array_equal(getattr(p, k), s[k]), k
                assert np.array_equal(st, B.start[i]) and np.array_equal(en, B.end[i])
                assert np.array_equal(fr, B.freq[i])
            finally:
                pm4g.pm4g_log_free(f)
    finally:
        pm4g.pm4g_log_free(log)


def test_batch_large_subsets_split_into_items(pm4g, ctx):
    """Sub-logs far larger than one work item (the whole log, wide windows)
    are split across CTAs and merged exactly; long cases and the sorted-case
    path are in the mix."""
    L = synth.generate(synth.large_log(60_000))
    rng = np.random.default_rng(13)
    L.case_attr = (L.case_id.astype(np.int64) * 7919 % 50).astype(np.int32)
    log = _load(pm4g, ctx, L)
    try:
        t0, t1 = int(L.ts_ns.min()), int(L.ts_ns.max())
        specs = [(np.empty(0, np.int32), t0, t1, 0), (np.empty(0, np.int32), t0, (t0 + t1) // 2, 1),
                 (np.arange(0, 50, 2, dtype=np.int32), t0 + (t1 - t0) // 4, t1, 3)]
        specs += _random_specs(L, rng, 8, max_attrs=40)
        _check_batch(_run(pm4g, log, specs), L, specs)
    finally:
        pm4g.pm4g_log_free(log)


def test_batch_without_attributes(pm4g, ctx):
    L = synth.generate(synth.single_log(3000))
    log = _load(pm4g, ctx, L, with_attr=False)
    try:
        t0, t1 = int(L.ts_ns.min()), int(L.ts_ns.max())
        specs = [(np.empty(0, np.int32), t0 + (t1 - t0) // 3, t1 - (t1 - t0) // 3, m) for m in range(4)]
        _check_batch(_run(pm4g, log, specs), L, specs, with_attr=False)
        with pytest.raises(pm4g.Pm4gError) as e:
            _run(pm4g, log, [(np.array([1], np.int32), t0, t1, 0)])
        assert e.value.status == pm4g.EINVAL
    finally:
        pm4g.pm4g_log_free(log)


def test_batch_edge_cases(pm4g, ctx):
    L = synth.generate(synth.drilldown_log(500))
    log = _load(pm4g, ctx, L)
    try:
        B = _run(pm4g, log, [])
        assert B.edge_off.tolist() == [0] and B.src.size == 0
        with pytest.raises(pm4g.Pm4gError) as e:
            _run(pm4g, log, [(np.empty(0, np.int32), 0, 1, 7)])
        assert e.value.status == pm4g.EINVAL
    finally:
        pm4g.pm4g_log_free(log)
    # an empty log: every sub-log is empty
    e = np.empty(0, np.int32)
    L0 = synth.EventLog(e, e, np.empty(0, np.int64), e, 3)
    log = _load(pm4g, ctx, L0)
    try:
        B = _run(pm4g, log, [(np.empty(0, np.int32), 0, 10, 1), (np.empty(0, np.int32), 0, 10, 0)])
        assert B.n_events.tolist() == [0, 0] and B.edge_off.tolist() == [0, 0, 0]
        assert B.start.shape == (2, 3) and not B.start.any()
    finally:
        pm4g.pm4g_log_free(log)


def test_batch_means_of_sums_beyond_64_bits(pm4g, ctx):
    """Edge (0, 0) sums above 2^64 whose low bits sit at, just below and just
    above the rounding boundary of the double conversion (round to nearest,
    ties to even, carry into a new bit): the batch's means are computed on the
    device and must have the oracle's (host) bits."""
    rng = np.random.default_rng(14)
    spans = []
    for d in (0, 1, 2, 3, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097):
        spans.append((1 << 63) + d)
        spans.append((1 << 64) - 1 - d)
    spans += [int(x) for x in rng.integers(1 << 62, (1 << 63) - 1, 20, dtype=np.int64)]
    K = len(spans)
    case = np.repeat(np.arange(K, dtype=np.int32), 2)
    ts = np.empty(2 * K, np.int64)
    for k, s in enumerate(spans):
        lo = -(1 << 63) + (k % 3)  # span < 2^64 fits between the int64 extremes
        ts[2 * k] = lo
        ts[2 * k + 1] = lo + s if lo + s < (1 << 63) else (1 << 63) - 1
    act = np.zeros(2 * K, np.int32)
    attr = np.repeat(np.arange(K, dtype=np.int32), 2)
    L = synth.EventLog(case, act, ts, attr, 1)
    log = _load(pm4g, ctx, L)
    try:
        specs = []
        for _ in range(40):
            k = int(rng.integers(2, 12))
            specs.append((rng.choice(K, k, replace=False).astype(np.int32), -(1 << 63), (1 << 63) - 1, 0))
        specs.append((np.arange(K, dtype=np.int32), -(1 << 63), (1 << 63) - 1, 0))
        _check_batch(_run(pm4g, log, specs), L, specs)
    finally:
        pm4g.pm4g_log_free(log)


def test_batch_into_reused_buffers(pm4g, ctx):
    """Caller-owned buffers: identical results, a too-small edge capacity
    reports PM4G_ERANGE with the size needed (the binding then grows and
    retries), and buffers are reused across calls."""
    L = synth.generate(synth.drilldown_log(4000))
    log = _load(pm4g, ctx, L)
    try:
        specs = _random_specs(L, np.random.default_rng(15), 20)
        args = ([s[0] for s in specs], [s[1] for s in specs], [s[2] for s in specs], [s[3] for s in specs])
        B1 = pm4g.pm4g_batch_dfg(log, *args)
        buf = pm4g.BatchBuffers(1, 1, 8)
        for _ in range(2):
            B2 = pm4g.pm4g_batch_dfg_into(log, *args, out=buf)
            for k in ("n_events", "n_cases", "edge_off", "src", "dst", "count", "sum_lo", "sum_hi", "min", "max",
                      "start", "end", "freq"):
                assert np.array_equal(getattr(B1, k), getattr(B2, k)), k
            assert np.array_equal(B1.mean.view(np.uint64), B2.mean.view(np.uint64))
        # the raw call with room for one edge
        import ctypes
        Q, A = len(specs), L.n_activities
        small = pm4g.BatchBuffers(Q, A, 1)
        small.edges = 1
        off = np.zeros(Q + 1, np.int64)
        off[1:] = np.cumsum([s[0].size for s in specs])
        vals = np.ascontiguousarray(np.concatenate([s[0] for s in specs]), np.int32)
        tl, th = np.array(args[1], np.int64), np.array(args[2], np.int64)
        md = np.array(args[3], np.int32)
        spec = pm4g._BatchSpec(Q, off.ctypes.data, vals.ctypes.data, tl.ctypes.data, th.ctypes.data, md.ctypes.data)
        r = pm4g._BatchDfg(Q, A, *(x.ctypes.data for x in (small.n_events, small.n_cases, small.edge_off, small.src,
                                                             small.dst, small.count, small.sum_lo, small.sum_hi,
                                                             small.min, small.max, small.mean, small.start,
                                                             small.end, small.freq)))
        st = pm4g.lib.pm4g_batch_dfg_into(log, ctypes.byref(spec), ctypes.byref(r), 1)
        assert st == pm4g.ERANGE
        assert int(small.edge_off[Q]) == int(B1.edge_off[-1]) > 1
        assert np.array_equal(small.n_events[:Q], B1.n_events)
    finally:
        pm4g.pm4g_log_free(log)


@pytest.mark.parametrize("top_k", [-1, 1, 3])
def test_batch_variants(pm4g, ctx, top_k):
    """Per-sub-log variants (counts, smallest case ids, sequences, order, top-k)
    computed in the same batch."""
    L = synth.generate(synth.drilldown_log(6000))
    log = _load(pm4g, ctx, L)
    try:
        t0, t1 = int(L.ts_ns.min()), int(L.ts_ns.max())
        specs = [(np.empty(0, np.int32), t0, t1, 0), (np.empty(0, np.int32), t0, (t0 + t1) // 2, 1)]
        specs += _random_specs(L, np.random.default_rng(16), 30)
        _check_batch(_run(pm4g, log, specs, top_k), L, specs, top_k=top_k)
    finally:
        pm4g.pm4g_log_free(log)


def test_batch_variants_repeated_sequences(pm4g, ctx):
    """Few activities, so many cases share sequences within and across
    sub-logs (a variant must never merge two sub-logs); forced hash collisions
    take the verification rounds."""
    L = synth.generate(synth.single_log(4000))
    L.case_attr = (L.case_id.astype(np.int64) % 7).astype(np.int32)
    log = _load(pm4g, ctx, L)
    try:
        t0, t1 = int(L.ts_ns.min()), int(L.ts_ns.max())
        specs = [(np.array([a], np.int32), t0, t1, 0) for a in range(7)]
        specs += [(np.array([0, 1], np.int32), t0 + (t1 - t0) // 5, t1, 1), (np.empty(0, np.int32), t0, t1, 3)]
        _check_batch(_run(pm4g, log, specs, -1), L, specs, top_k=-1)
        pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TEST_HASH_BITS, 3)
        _check_batch(_run(pm4g, log, specs, 5), L, specs, top_k=5)
    finally:
        pm4g.pm4g_log_free(log)


def test_batch_variants_into_buffers(pm4g, ctx):
    """Variants through caller buffers, starting too small (grow and retry)."""
    L = synth.generate(synth.drilldown_log(3000))
    log = _load(pm4g, ctx, L)
    try:
        specs = _random_specs(L, np.random.default_rng(17), 15)
        args = ([s[0] for s in specs], [s[1] for s in specs], [s[2] for s in specs], [s[3] for s in specs])
        B1 = pm4g.pm4g_batch_dfg(log, *args, var_top_k=-1)
        buf = pm4g.BatchBuffers(1, 1, 4, 2, 2)
        B2 = pm4g.pm4g_batch_dfg_into(log, *args, out=buf, var_top_k=-1)
        for k in ("n_variants", "var_off", "var_count", "var_min_case", "var_seq_off", "var_acts", "edge_off",
                  "count"):
            assert np.array_equal(getattr(B1, k), getattr(B2, k)), k
        _check_batch(B2, L, specs, top_k=-1)
    finally:
        pm4g.pm4g_log_free(log)


def _same_batch(A, B):
    for k in ("n_events", "n_cases", "edge_off", "src", "dst", "count", "sum_lo", "sum_hi", "min", "max", "start",
              "end", "freq", "n_variants", "var_off", "var_count", "var_min_case", "var_seq_off", "var_acts"):
        x, y = getattr(A, k), getattr(B, k)
        assert np.array_equal(np.asarray(x), np.asarray(y)), k
    assert np.array_equal(A.mean.view(np.uint64), B.mean.view(np.uint64))


def test_launch_choices_do_not_change_results(pm4g, ctx):
    """Every launch choice of the batch (cases per warp chunk, items per SM,
    pipeline groups into caller-owned buffers) gives the same results, bit
    for bit; the default choice is checked against the oracle."""
    L = synth.generate(synth.drilldown_log(8000))
    log = _load(pm4g, ctx, L)
    try:
        specs = _random_specs(L, np.random.default_rng(17), 80)
        spec = pm4g.BatchSpec([s[0] for s in specs], [s[1] for s in specs], [s[2] for s in specs],
                              [s[3] for s in specs])
        ref = pm4g.pm4g_batch_dfg(log, spec=spec, var_top_k=5)
        _check_batch(ref, L, specs, top_k=5)
        for chunk, items, stages in ((8, 2, 1), (32, 8, 2), (16, 1, 3), (8, 32, 16), (32, 4, 4)):
            for knob, v in ((pm4g.OPT_BATCH_CHUNK, chunk), (pm4g.OPT_BATCH_ITEMS_PER_SM, items),
                            (pm4g.OPT_BATCH_STAGES, stages)):
                pm4g.pm4g_ctx_set_option(ctx, knob, v)
            _same_batch(pm4g.pm4g_batch_dfg(log, spec=spec, var_top_k=5), ref)
            buf = pm4g.BatchBuffers(len(specs), L.n_activities, 0)  # caller-owned: the pipelined path
            _same_batch(pm4g.pm4g_batch_dfg(log, spec=spec, out=buf, var_top_k=5), ref)
        for knob in (pm4g.OPT_BATCH_CHUNK, pm4g.OPT_BATCH_ITEMS_PER_SM, pm4g.OPT_BATCH_STAGES):
            with pytest.raises(pm4g.Pm4gError):
                pm4g.pm4g_ctx_set_option(ctx, knob, 7 if knob == pm4g.OPT_BATCH_CHUNK else 99)
            pm4g.pm4g_ctx_set_option(ctx, knob, 0)
    finally:
        pm4g.pm4g_log_free(log)


def test_autotuner_applies_a_choice_that_keeps_results(pm4g, ctx, tmp_path):
    from paper_2204_04898_b300 import autotune
    L = synth.generate(synth.drilldown_log(8000))
    log = _load(pm4g, ctx, L)
    try:
        specs = _random_specs(L, np.random.default_rng(19), 70)
        spec = pm4g.BatchSpec([s[0] for s in specs], [s[1] for s in specs], [s[2] for s in specs],
                              [s[3] for s in specs])
        ref = pm4g.pm4g_batch_dfg(log, spec=spec, var_top_k=3)
        buf = pm4g.BatchBuffers(len(specs), L.n_activities, 0)
        tuner = autotune.Tuner(cache_path=str(tmp_path / "tune.json"))
        choice = tuner.tune_batch(ctx, log, spec, var_top_k=3, out=buf, reps=1)
        assert all(choice[k] in autotune.SPACE[k] for k in autotune.SPACE)
        _same_batch(pm4g.pm4g_batch_dfg(log, spec=spec, out=buf, var_top_k=3), ref)
        assert autotune.Tuner(cache_path=str(tmp_path / "tune.json")).cache  # persisted
        autotune.Tuner.apply(ctx, {})
    finally:
        pm4g.pm4g_log_free(log)


def test_efg_then_drilldown_shares_timestamps_without_leaking(pm4g):
    """The eventually-follows graph and the drill-down index both use the
    log's timestamps in formatted order. Running pm4g_efg first and then a
    batched drill-down on the same log must give the oracle's results and
    leave no device buffer behind once the log is freed, however often the
    pair is repeated (a counting allocator sees every block)."""
    import torch
    live = {}

    def alloc(nbytes, stream):
        t = torch.empty(max(1, nbytes), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, nbytes, stream):
        live.pop(ptr, None)

    ctx = pm4g.pm4g_ctx_create(0, allocator=(alloc, free))
    try:
        L = synth.generate(synth.drilldown_log(3000))
        specs = _random_specs(L, np.random.default_rng(21), 10)
        W = oracle.efg(L.case_id, L.activity, L.ts_ns, L.n_activities)
        held = []
        for rep in range(4):
            log = _load(pm4g, ctx, L)
            try:
                G = pm4g.pm4g_efg(log)
                for f in ("src", "dst", "count", "sum_lo", "sum_hi"):
                    assert np.array_equal(getattr(G, f), getattr(W, f)), f
                B = _run(pm4g, log, specs, top_k=3)
                if rep == 0:
                    _check_batch(B, L, specs, top_k=3)
            finally:
                pm4g.pm4g_log_free(log)
            torch.cuda.synchronize()
            held.append(sum(t.numel() for t in live.values()))
        assert held[0] == 0, f"{held[0]} bytes still held after the log was freed"
        assert held == [held[0]] * len(held), f"device bytes held after each repeat: {held}"
    finally:
        pm4g.pm4g_ctx_destroy(ctx)
