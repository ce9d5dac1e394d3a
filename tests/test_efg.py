"""Eventually-follows graph and temporal profile on the GPU against the
oracle, bit-exact: pairs, counts, 128-bit sums, 192-bit sums of squares, and
the bits of every mean and standard deviation. All calls go through the C ABI
(libpm4g.so)."""

import numpy as np
import pytest

import oracle
import pm4g_synth as synth
from tests import oracle_pins as pins

pytestmark = pytest.mark.gpu

FIELDS = ("src", "dst", "count", "sum_lo", "sum_hi", "sq0", "sq1", "sq2")


@pytest.fixture(scope="module")
def pm4g():
    from paper_2204_04898_b300 import pm4g as m
    return m


@pytest.fixture()
def ctx(pm4g):
    c = pm4g.pm4g_ctx_create(0)
    yield c
    pm4g.pm4g_ctx_destroy(c)


def check_efg(pm4g, ctx, case, act, ts, A, device=True):
    case, act, ts = np.asarray(case, np.int32), np.asarray(act, np.int32), np.asarray(ts, np.int64)
    W = oracle.efg(case, act, ts, A)
    if device:
        import torch
        cols = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (case, act, ts)]
    else:
        cols = [case, act, ts]
    log = pm4g.pm4g_load_log(ctx, *cols, n_activities=A)
    try:
        G = pm4g.pm4g_efg(log)
    finally:
        pm4g.pm4g_log_free(log)
    for f in FIELDS:
        assert np.array_equal(getattr(G, f), getattr(W, f)), f
    for f in ("mean", "stdev"):
        assert np.array_equal(getattr(G, f).view(np.uint64), getattr(W, f).view(np.uint64)), f
    return W


def test_golden(pm4g, ctx):
    g = pins.load_golden("fine_process_example.json")
    lg = g["log"]
    check_efg(pm4g, ctx, lg["case"], lg["activity"], lg["ts"], g["n_activities"], device=False)


def test_random_tiny_logs(pm4g, ctx):
    rng = np.random.default_rng(31)
    for it in range(40):
        n = int(rng.integers(0, 60))
        case = rng.integers(0, 6, n)
        act = rng.integers(0, 4, n)
        big = it % 2 == 0  # durations near 2^62: the squares carry into their third word
        ts = rng.integers(-(2**62), 2**62, n) if big else rng.integers(0, 9, n)
        check_efg(pm4g, ctx, case, act, ts, 4)


@pytest.mark.parametrize("spec", [synth.large_log(3000), synth.very_large_log(2000), synth.single_log(3000)],
                         ids=lambda s: s.name)
def test_workloads(pm4g, ctx, spec):
    L = synth.generate(spec)
    W = check_efg(pm4g, ctx, L.case_id, L.activity, L.ts_ns, L.n_activities)
    assert W.count.size > 0


def test_long_and_short_cases(pm4g, ctx):
    """Cases of 1, 2, 31, 32, 33, 64, 65 and 300 events (chunk edges of the
    warp walk), with ties in time."""
    rng = np.random.default_rng(7)
    lens = [1, 2, 31, 32, 33, 64, 65, 300, 1, 5]
    case = np.repeat(np.arange(len(lens), dtype=np.int32), lens)
    act = rng.integers(0, 7, case.size)
    ts = rng.integers(0, 40, case.size) * 1_000_000_007
    p = rng.permutation(case.size)
    check_efg(pm4g, ctx, case[p], act[p], ts[p], 7)


def test_empty_and_single_events(pm4g, ctx):
    check_efg(pm4g, ctx, [], [], [], 3, device=False)
    check_efg(pm4g, ctx, [5, 6, 7], [0, 1, 2], [1, 2, 3], 3, device=False)
