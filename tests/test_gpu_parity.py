"""CUDA path against the CPU oracle, bit-exact (tolerance 0): counts, 128-bit
duration sums, min/max, FP64 means formed from the exact sums, start/end and
frequency counts, variant ids, counts, sequences and order, the case-to-variant
map and the formatted (case, timestamp, row) order. All calls go through the C
ABI (libpm4g.so)."""

import numpy as np
import pytest

import oracle
import pm4g_synth as synth
from tests import oracle_pins as pins
from tests.gpu_util import check_log, gpu_run, assert_same

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


@pytest.mark.parametrize("name", ["fine_process_example.json", "signed_ties_example.json"])
def test_golden(pm4g, ctx, name):
    g = pins.load_golden(name)
    lg = g["log"]
    check_log(pm4g, ctx, np.array(lg["case"], np.int32), np.array(lg["activity"], np.int32),
              np.array(lg["ts"], np.int64), g["n_activities"])


def test_random_tiny_logs(pm4g, ctx):
    rng = np.random.default_rng(1)
    for t in range(120):
        n = int(rng.integers(1, 40))
        A = int(rng.integers(1, 6))
        case = rng.choice([-2**31, -7, 0, 5, 9, 2**31 - 1], size=n).astype(np.int32)
        act = rng.integers(0, A, n).astype(np.int32)
        if t % 3 == 0:
            ts = rng.choice(np.array([-2**63, -1, 0, 1, 2**62, 2**63 - 1], np.int64), size=n)
        else:
            ts = rng.integers(0, 5, n).astype(np.int64)
        check_log(pm4g, ctx, case, act, ts, A)


def test_empty_log(pm4g, ctx):
    e = np.empty(0, np.int32)
    check_log(pm4g, ctx, e, e, np.empty(0, np.int64), 3, device=False)


@pytest.mark.parametrize("spec", [synth.single_log(), synth.large_log(40_000), synth.very_large_log(40_000),
                                  synth.drilldown_log(20_000)], ids=lambda s: s.name)
def test_workloads(pm4g, ctx, spec):
    L = synth.generate(spec)
    check_log(pm4g, ctx, L.case_id, L.activity, L.ts_ns, L.n_activities, case_attr=L.case_attr)


@pytest.mark.parametrize("spec", [synth.large_log(300_000), synth.very_large_log(300_000)], ids=lambda s: s.name)
def test_two_level_partition(pm4g, ctx, spec):
    """Logs with more than 512 buckets are partitioned in two levels."""
    L = synth.generate(spec)
    check_log(pm4g, ctx, L.case_id, L.activity, L.ts_ns, L.n_activities, export=False)


def test_host_pointers(pm4g, ctx):
    L = synth.generate(synth.large_log(5_000))
    check_log(pm4g, ctx, L.case_id, L.activity, L.ts_ns, L.n_activities, device=False)


def test_sparse_case_ids(pm4g, ctx):
    """Case ids spread over the whole int32 range take the renumbering path."""
    L = synth.generate(synth.single_log(3000))
    rng = np.random.default_rng(5)
    ids = np.unique(rng.integers(-2**31, 2**31 - 1, 6000))[:3000]
    rng.shuffle(ids)
    case = ids[L.case_id].astype(np.int32)
    check_log(pm4g, ctx, case, L.activity, L.ts_ns, L.n_activities)


def test_special_cases(pm4g, ctx):
    rng = np.random.default_rng(2)
    case = rng.integers(0, 300, 5000).astype(np.int32)
    ts = rng.integers(0, 50, 5000).astype(np.int64)
    check_log(pm4g, ctx, case, np.zeros(5000, np.int32), ts, 1)           # A = 1
    case = rng.permutation(4000).astype(np.int32)
    check_log(pm4g, ctx, case, rng.integers(0, 9, 4000).astype(np.int32), ts[:4000], 9)  # all L = 1


def test_long_cases_take_global_path(pm4g, ctx):
    """Cases longer than the on-chip sort limit (512 events) and buckets larger
    than shared memory go through the global-memory path."""
    rng = np.random.default_rng(3)
    lens = np.array([1, 600, 3, 2000, 513, 7, 40000], np.int64)
    case = np.repeat(np.arange(lens.size, dtype=np.int32) * 3, lens)
    n = case.size
    p = rng.permutation(n)
    case = case[p]
    act = rng.integers(0, 7, n).astype(np.int32)
    ts = rng.integers(0, 10**6, n).astype(np.int64)
    check_log(pm4g, ctx, case, act, ts, 7)


@pytest.mark.parametrize("ts_range", [8, 10**9])
def test_on_chip_sort_lengths(pm4g, ctx, ts_range):
    """Shuffled cases of every on-chip sort size class (1..32, ..64, ..128 in
    registers; 129..512 merged from 128-event chunks), with timestamp ties
    broken by row when the range is small."""
    rng = np.random.default_rng(7)
    base = np.array([1, 2, 31, 32, 33, 64, 65, 127, 128, 129, 130, 200, 255, 256, 257, 300, 383, 384, 385,
                     450, 511, 512], np.int64)
    lens = np.concatenate([base, rng.integers(100, 513, 60)])
    case = np.repeat(rng.permutation(lens.size).astype(np.int32) * 5, lens)
    n = case.size
    p = rng.permutation(n)
    case = case[p]
    act = rng.integers(0, 11, n).astype(np.int32)
    ts = rng.integers(-ts_range, ts_range, n).astype(np.int64)
    check_log(pm4g, ctx, case, act, ts, 11)


def test_forced_small_buckets(pm4g, ctx):
    """A tiny on-chip capacity sends most buckets down the global path."""
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TEST_BUCKET_CAP, 64)
    L = synth.generate(synth.large_log(3000))
    check_log(pm4g, ctx, L.case_id, L.activity, L.ts_ns, L.n_activities)


@pytest.mark.parametrize("bits", [1, 4, 8])
def test_forced_hash_collisions(pm4g, ctx, bits):
    """Truncated variant keys collide constantly; the full-sequence check must
    still give the exact variant table."""
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TEST_HASH_BITS, bits)
    L = synth.generate(synth.single_log(3000))
    check_log(pm4g, ctx, L.case_id, L.activity, L.ts_ns, L.n_activities)


def test_top_k(pm4g, ctx):
    L = synth.generate(synth.large_log(4000))
    for k in (0, 1, 10, 10**9):
        check_log(pm4g, ctx, L.case_id, L.activity, L.ts_ns, L.n_activities, export=False, top_k=k)


def test_errors(pm4g, ctx):
    c = np.array([1, 1], np.int32)
    t = np.array([0, 1], np.int64)
    with pytest.raises(pm4g.Pm4gError) as e:
        pm4g.pm4g_load_log(ctx, c, np.array([0, 3], np.int32), t, n_activities=3)
    assert e.value.status == pm4g.ERANGE
    with pytest.raises(pm4g.Pm4gError) as e:
        pm4g.pm4g_load_log(ctx, c, np.array([-1, 0], np.int32), t, n_activities=3)
    assert e.value.status == pm4g.ERANGE
    with pytest.raises(pm4g.Pm4gError) as e:
        pm4g.pm4g_load_log(ctx, c, np.array([0, 0], np.int32), t, n_activities=0)
    assert e.value.status == pm4g.EINVAL
    with pytest.raises(pm4g.Pm4gError) as e:
        pm4g.pm4g_ctx_set_option(ctx, 99, 1)
    assert e.value.status == pm4g.EINVAL
    # the context still works after errors
    check_log(pm4g, ctx, c, np.array([0, 1], np.int32), t, 3)


def test_allocator_hook_failure_is_enomem(pm4g):
    import torch
    calls = {"n": 0}
    live = {}

    def alloc(nbytes, stream):
        calls["n"] += 1
        if calls["n"] >= 6:
            return 0
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, nbytes, stream):
        live.pop(ptr, None)

    ctx = pm4g.pm4g_ctx_create(0, allocator=(alloc, free))
    try:
        L = synth.generate(synth.single_log(2000))
        with pytest.raises(pm4g.Pm4gError) as e:
            pm4g.pm4g_load_log(ctx, *[torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns)],
                               n_activities=L.n_activities)
        assert e.value.status == pm4g.ENOMEM
        torch.cuda.synchronize()
        assert not live, "a failed load leaked device buffers"
    finally:
        pm4g.pm4g_ctx_destroy(ctx)


# ---------------- drill-down filters ----------------
def _filter_parity(pm4g, ctx, L, aset, t_lo, t_hi, mode):
    rows = oracle.filter_rows(L.case_id, L.activity, L.ts_ns, L.case_attr, L.n_activities, aset, t_lo, t_hi, mode)
    sub = L.take(rows)
    R = oracle.summarize(sub.case_id, sub.activity, sub.ts_ns, L.n_activities)
    return rows, sub, R


def test_filters(pm4g, ctx):
    L = synth.generate(synth.drilldown_log(6000))
    import torch
    cols = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns, L.case_attr)]
    log = pm4g.pm4g_load_log(ctx, *cols[:3], case_attr=cols[3], n_activities=L.n_activities)
    try:
        t0, t1 = int(L.ts_ns.min()), int(L.ts_ns.max())
        rng = np.random.default_rng(4)
        specs = [([], t0, t1, 0), ([], t0, t1, 1), ([], t0, t1, 2), ([], t0, t1, 3)]
        for _ in range(6):
            aset = np.unique(rng.integers(0, 4096, int(rng.integers(1, 2000))))
            lo = t0 + int(rng.uniform(0, 0.5) * (t1 - t0))
            hi = lo + int(rng.uniform(0.1, 0.5) * (t1 - t0))
            for mode in range(4):
                specs.append((aset, lo, hi, mode))
        for aset, lo, hi, mode in specs:
            rows, sub, R = _filter_parity(pm4g, ctx, L, aset, lo, hi, mode)
            f = pm4g.pm4g_filter(log, aset, lo, hi, mode)
            try:
                got = {"info": pm4g.pm4g_log_info(f), "dfg": pm4g.pm4g_dfg(f), "perf": pm4g.pm4g_perf_dfg(f),
                       "var": pm4g.pm4g_variants(f, cases=True)}
                got["start"], got["end"], got["freq"] = pm4g.pm4g_start_end(f, L.n_activities)
                e = pm4g.pm4g_log_export(f)
                # exported rows are original rows; relabel the oracle's sub-log order
                got["export"] = dict(e, row=np.searchsorted(rows, e["row"]))
                assert np.array_equal(rows[got["export"]["row"]], e["row"])
                assert_same(got, R, sub.case_id, sub.activity, sub.ts_ns)
            finally:
                pm4g.pm4g_log_free(f)
    finally:
        pm4g.pm4g_log_free(log)


def test_filter_chain_and_reuse(pm4g, ctx):
    """A filtered log is a log: it can be queried repeatedly and filtered again."""
    L = synth.generate(synth.drilldown_log(3000))
    import torch
    cols = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns, L.case_attr)]
    log = pm4g.pm4g_load_log(ctx, *cols[:3], case_attr=cols[3], n_activities=L.n_activities)
    t0, t1 = int(L.ts_ns.min()), int(L.ts_ns.max())
    mid = (t0 + t1) // 2
    f1 = pm4g.pm4g_filter(log, [], t0, mid, pm4g.TW_CASES_INTERSECTING)
    f2 = pm4g.pm4g_filter(f1, [], mid - (mid - t0) // 2, t1, pm4g.TW_EVENTS)
    try:
        r1 = oracle.filter_rows(L.case_id, L.activity, L.ts_ns, None, L.n_activities, [], t0, mid, 3)
        s1 = L.take(r1)
        r2 = oracle.filter_rows(s1.case_id, s1.activity, s1.ts_ns, None, L.n_activities, [],
                                mid - (mid - t0) // 2, t1, 1)
        s2 = s1.take(r2)
        R = oracle.summarize(s2.case_id, s2.activity, s2.ts_ns, L.n_activities)
        for _ in range(2):
            got = {"info": pm4g.pm4g_log_info(f2), "dfg": pm4g.pm4g_dfg(f2), "perf": pm4g.pm4g_perf_dfg(f2),
                   "var": pm4g.pm4g_variants(f2, cases=True)}
            got["start"], got["end"], got["freq"] = pm4g.pm4g_start_end(f2, L.n_activities)
            assert_same(got, R, export=False)
    finally:
        for h in (f2, f1, log):
            pm4g.pm4g_log_free(h)


@pytest.mark.parametrize("where", ["first", "warp", "tile", "chunk", "last", "none"])
def test_time_sorted_input_fast_path(pm4g, ctx, where):
    """Rows sorted by timestamp take the streaming segment pass; one descent
    that puts a case out of order anywhere (at a warp, tile or row-chunk
    boundary of the partition, or at the ends) must be seen by that pass, whose
    partial sums are then cleared and the log redone by the sorting pass."""
    L = synth.generate(synth.very_large_log(20000))
    n = L.n_events
    case, act, ts = L.case_id.copy(), L.activity.copy(), L.ts_ns.copy()
    assert np.all(np.diff(ts) >= 0)
    chunk = ((n + 2 * 148 - 1) // (2 * 148) + 3) // 4 * 4
    target = {"first": 1, "warp": 256, "tile": 4096, "chunk": chunk, "last": n - 1, "none": None}[where]
    if target is not None:
        # the first row at or after target whose case has an earlier event: its
        # timestamp drops just below that earlier event's, so exactly one
        # descent appears (at that row) and its case is out of order
        first_row = {}
        for r in range(n):
            first_row.setdefault(int(case[r]), r)
        pos = next(r for r in range(target, n) if first_row[int(case[r])] < r)
        q = max(r for r in range(pos) if case[r] == case[pos])
        ts[pos] = ts[q] - 1
        d = np.nonzero(np.diff(ts) < 0)[0]
        assert d.tolist() == [pos - 1]
    check_log(pm4g, ctx, case, act, ts, L.n_activities)


def test_case_ordered_rows_take_the_streaming_pass(pm4g, ctx):
    """Rows grouped by case, each case's events in timestamp order, are not
    in global timestamp order, yet every case is: the streaming pass takes the
    log (the sorting pass sorts nothing). One event moved before its case's
    previous one sends the log to the sorting pass, with the same results as
    the oracle's."""
    L = synth.generate(synth.very_large_log(20000))
    o = np.lexsort((np.arange(L.n_events), L.ts_ns, L.case_id))
    case, act, ts = L.case_id[o].copy(), L.activity[o].copy(), L.ts_ns[o].copy()
    assert np.any(np.diff(ts) < 0)
    pm4g.pm4g_ctx_timing_reset(ctx)
    check_log(pm4g, ctx, case, act, ts, L.n_activities)
    assert pm4g.pm4g_ctx_timing(ctx, "sorted_windows")[0] == 0
    # the last event of a case of length >= 2, at the end of the rows, now
    # comes before its predecessor
    r = next(i for i in range(L.n_events - 1, 0, -1) if case[i] == case[i - 1])
    ts[r] = ts[r - 1] - 1
    pm4g.pm4g_ctx_timing_reset(ctx)
    check_log(pm4g, ctx, case, act, ts, L.n_activities)
    assert pm4g.pm4g_ctx_timing(ctx, "sorted_windows")[0] > 0


@pytest.mark.parametrize("device", [True, False], ids=["device", "host"])
def test_case_id_range_guess(pm4g, ctx, device):
    """The buckets are laid out for a case id range guessed from evenly spaced
    rows and widened by 1/256 of its span on each side; the bucket histogram
    confirms that every id lies inside. No column reduction runs when the
    guess holds (ids in row order either way round, or spread over the rows
    in time order); it runs, with the oracle's results all the same, when an
    id elsewhere falls outside the widened span (below, above, or far enough
    out to make the ids sparse) and when the guess itself looks sparse."""
    L = synth.generate(synth.large_log(6000))
    o = np.lexsort((np.arange(L.n_events), L.ts_ns, L.case_id))
    case, act, ts = L.case_id[o].astype(np.int64), L.activity[o].copy(), L.ts_ns[o].copy()
    n = len(case)
    span = int(case.max() - case.min())
    r = np.arange(n)
    t = np.argsort(ts, kind="stable")  # the same events in time order
    shapes = {
        "ascending": (case + 11, True),
        "descending": (case.max() - case - 5, True),
        "time_ordered": (case[t], True),
        "below_inside": (np.where(r == n // 2, case.min() - span // 8, case), False),
        "above_inside": (np.where(r == n // 3 + 1, case.max() + span // 8, case), False),
        "sparse_inside": (np.where(r == n // 4, 2**31 - 1, case), False),
        "sparse_ends": (np.where(r == n - 1, -2**31, case), False),
    }
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 1)
    try:
        for name, (c, no_reduction) in shapes.items():
            c = c.astype(np.int32)
            a, tt = (act[t], ts[t]) if name == "time_ordered" else (act, ts)
            pm4g.pm4g_ctx_timing_reset(ctx)
            check_log(pm4g, ctx, c, a, tt, L.n_activities, device=device)
            ran = pm4g.pm4g_ctx_timing(ctx, "stats")[0]
            assert (ran == 0) == no_reduction, name
    finally:
        pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 0)
    # one event: its id is the whole range
    check_log(pm4g, ctx, np.array([-9], np.int32), np.array([0], np.int32), np.array([5], np.int64), 1,
              device=device)
    # ids at both ends of the int32 range around dense ones are sparse
    check_log(pm4g, ctx, np.array([2**31 - 1, 3, 4, -2**31], np.int32), np.zeros(4, np.int32),
              np.arange(4, dtype=np.int64), 1, device=device)


@pytest.mark.parametrize("spec", [synth.single_log(), synth.very_large_log(40_000), synth.drilldown_log(20_000)],
                         ids=lambda s: s.name)
def test_workload_range_needs_no_reduction(pm4g, ctx, spec):
    """On the benchmark workloads' logs the sampled case-id range holds, so
    no column reduction runs (and the results are the oracle's)."""
    L = synth.generate(spec)
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 1)
    try:
        pm4g.pm4g_ctx_timing_reset(ctx)
        check_log(pm4g, ctx, L.case_id, L.activity, L.ts_ns, L.n_activities, case_attr=L.case_attr,
                  export=False)
        assert pm4g.pm4g_ctx_timing(ctx, "stats")[0] == 0
        assert pm4g.pm4g_ctx_timing(ctx, "bucket_hist")[0] >= 1
    finally:
        pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 0)


def test_one_pass_16bit_histogram(pm4g, ctx):
    """Between 57,856 and 115,712 buckets the bucket histogram runs once with
    16-bit counters (8M events, case ids spread over 16M slots)."""
    rng = np.random.default_rng(31)
    n = 8_000_000
    case = rng.integers(0, 16_000_000, n).astype(np.int32)
    act = rng.integers(0, 6, n).astype(np.int32)
    ts = rng.integers(0, 10**12, n).astype(np.int64)
    check_log(pm4g, ctx, case, act, ts, 6, export=False)


def test_16bit_histogram_overflow_recount(pm4g, ctx):
    """A row chunk holding more than 65,535 events of one bucket makes its CTA
    count again in 32 bits (24M rows: one 70,000-event case in consecutive rows
    among single-event cases)."""
    rng = np.random.default_rng(32)
    n_small = 24_000_000
    big = 70_000
    case = np.arange(n_small, dtype=np.int32)
    n = n_small + big
    chunk = ((n + 2 * 148 - 1) // (2 * 148) + 3) // 4 * 4  # the partition's row chunk
    at = 62 * chunk                                      # the whole run inside chunk 62
    case = np.concatenate([case[:at], np.full(big, 1_000_003, np.int32), case[at:]])
    act = rng.integers(0, 5, n).astype(np.int32)
    ts = rng.integers(0, 10**9, n).astype(np.int64)
    check_log(pm4g, ctx, case, act, ts, 5, export=False)


def test_unaligned_device_columns(pm4g, ctx):
    """Columns that start 4, 8 or 12 bytes past a 16-byte boundary (views into
    larger tensors): the tile prefetches cover only the aligned interior of
    each range, and the results are those of the aligned columns."""
    import torch
    from tests.gpu_util import collect
    L = synth.generate(synth.large_log(20000))
    R = oracle.summarize(L.case_id, L.activity, L.ts_ns, L.n_activities)
    for off in (1, 2, 3):
        cols = []
        for x in (L.case_id, L.activity, L.ts_ns):
            t = torch.from_numpy(x)
            buf = torch.zeros(x.size + 4, dtype=t.dtype, device="cuda")
            buf[off:off + x.size] = t.cuda()
            cols.append(buf[off:off + x.size])
        assert cols[0].data_ptr() % 16 != 0
        log = pm4g.pm4g_load_log(ctx, *cols, n_activities=L.n_activities)
        try:
            got = collect(pm4g, log, L.n_activities)
        finally:
            pm4g.pm4g_log_free(log)
        assert_same(got, R, L.case_id, L.activity, L.ts_ns)


def test_wide_coarse_partition(pm4g, ctx):
    """32,000 case slots in 32-slot buckets (forced by a small on-chip
    capacity): 1,000 buckets, a two-level partition with 500 coarse buckets,
    whose shared memory allows one CTA per SM; buckets over the capacity
    split into case ranges."""
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TEST_BUCKET_CAP, 1000)
    rng = np.random.default_rng(8)
    lens = rng.integers(10, 31, 32000)
    case = np.repeat(np.arange(32000, dtype=np.int32), lens)
    n = case.size
    act = rng.integers(0, 40, n).astype(np.int32)
    ts = rng.integers(0, 10**13, n).astype(np.int64)
    order = np.argsort(ts, kind="stable")  # a time-ordered log, cases interleaved
    check_log(pm4g, ctx, case[order], act[order], ts[order], 40)


@pytest.mark.parametrize("bits", [0, 4])
def test_variants_long_repeated_sequences(pm4g, ctx, bits):
    """Cases of 40 to 300 events that repeat a few sequences, some of which
    differ from another only at position 33, in the middle or at the last
    event: the grouped comparison with the representative has to read past
    its first steps (with truncated keys every case meets a foreign one)."""
    if bits:
        pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TEST_HASH_BITS, bits)
    rng = np.random.default_rng(5)
    base = rng.integers(0, 9, 300).astype(np.int32)
    seqs = []
    for n in (40, 100, 300):
        s0 = base[:n].copy()
        seqs.append(s0)
        for pos in (33, n // 2, n - 1):
            s1 = s0.copy()
            s1[pos] = (s1[pos] + 1) % 9
            seqs.append(s1)
    cases, acts, tss = [], [], []
    cid = 0
    for _ in range(6):
        for s in seqs:
            cases.append(np.full(s.size, cid, np.int32))
            acts.append(s)
            tss.append(np.sort(rng.integers(0, 10**12, s.size)))
            cid += 1
    case, act, ts = np.concatenate(cases), np.concatenate(acts), np.concatenate(tss).astype(np.int64)
    p = rng.permutation(case.size)
    check_log(pm4g, ctx, case[p], act[p], ts[p], 9)
