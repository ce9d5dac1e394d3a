"""Generator determinism and shapes (no GPU)."""

import numpy as np

import pm4g_synth as synth


def test_deterministic_and_thread_independent():
    a = synth.generate(synth.large_log(5000), n_threads=1)
    b = synth.generate(synth.large_log(5000), n_threads=7)
    for f in ("case_id", "activity", "ts_ns"):
        assert np.array_equal(getattr(a, f), getattr(b, f))


def test_shapes():
    L = synth.generate(synth.very_large_log(4000))
    assert np.all(np.diff(L.ts_ns) >= 0)  # rows sorted by timestamp only
    assert L.activity.min() >= 0 and L.activity.max() < 500
    assert np.array_equal(np.unique(L.case_id), np.arange(4000))
    L1 = synth.generate(synth.single_log())
    assert 90_000 < L1.n_events < 110_000
    L4 = synth.generate(synth.drilldown_log(3000))
    assert L4.case_attr is not None and L4.case_attr.max() < 4096
    # the attribute is constant per case
    order = np.argsort(L4.case_id, kind="stable")
    c, a = L4.case_id[order], L4.case_attr[order]
    same = c[1:] == c[:-1]
    assert np.all(a[1:][same] == a[:-1][same])


def test_drilldown_specs():
    L = synth.generate(synth.drilldown_log(3000))
    specs = synth.drilldown_specs(L, n_views=32)
    assert len(specs) == 32
    for s in specs:
        assert s.t_lo <= s.t_hi and 1 <= s.attr_set.size <= 4096
        assert np.all(np.diff(s.attr_set) > 0)
