"""Host side of the batched drill-down (no GPU): every result array grows to at
least twice its size, so a server seeing ever larger batches reallocates (and
page-locks) a few times only, and a smaller batch never shrinks them; the views
reach the C struct as CSR attribute lists, int64 windows and int32 modes."""

from paper_2204_04898_b300 import pm4g


def test_buffers_grow_geometrically():
    b = pm4g.BatchBuffers(0, 0, 0)
    sizes = []
    for q in range(1, 200):
        b.ensure(q, 8, 100 * q, var_rows=10 * q, var_acts=40 * q)
        assert b.n_sub >= q and b.start.shape[0] >= q * 8
        assert b.src.shape[0] >= 100 * q and b.var_count.shape[0] >= 10 * q and b.var_acts.shape[0] >= 40 * q
        sizes.append((b.n_sub, b.edges, b.var_rows, b.var_acts_cap))
    # distinct sizes of each array: logarithmic in the largest request
    for k in range(4):
        assert len({s[k] for s in sizes}) <= 9, k


def test_smaller_batches_keep_the_buffers():
    b = pm4g.BatchBuffers(64, 16, 5000, var_rows=100, var_acts=400)
    arrays = (b.start, b.src, b.var_count, b.var_acts)
    b.ensure(8, 16, 100, var_rows=10, var_acts=40)
    assert all(x is y for x, y in zip(arrays, (b.start, b.src, b.var_count, b.var_acts)))


def test_batch_spec_marshalling():
    """The views go to the C struct as CSR attribute lists (None and empty sets
    mean all cases), int64 windows and int32 modes, whatever the input types."""
    import ctypes

    import numpy as np
    import pytest

    spec = pm4g.BatchSpec([None, [3, 1], np.array([7], np.int64), []], [0, -5, 2**40, -(2**63)],
                          np.array([10, 5, 2**41, 2**63 - 1]), [pm4g.TW_NONE, pm4g.TW_EVENTS,
                                                                pm4g.TW_CASES_CONTAINED,
                                                                pm4g.TW_CASES_INTERSECTING])
    assert spec.Q == 4
    assert spec.off.tolist() == [0, 0, 2, 3, 3] and spec.off.dtype == np.int64
    assert spec.vals.tolist() == [3, 1, 7] and spec.vals.dtype == np.int32
    assert spec.tl.tolist() == [0, -5, 2**40, -(2**63)] and spec.th[-1] == 2**63 - 1
    assert spec.md.dtype == np.int32
    s = spec.struct(-1)
    assert s.n_sub == 4 and s.var_top_k == -1
    assert s.attr_off == spec.off.ctypes.data and s.attr_vals == spec.vals.ctypes.data
    assert list((ctypes.c_int64 * 5).from_address(s.attr_off)) == [0, 0, 2, 3, 3]
    assert list((ctypes.c_int32 * 3).from_address(s.attr_vals)) == [3, 1, 7]
    assert list((ctypes.c_int64 * 4).from_address(s.t_lo)) == [0, -5, 2**40, -(2**63)]
    assert list((ctypes.c_int32 * 4).from_address(s.mode)) == [pm4g.TW_NONE, pm4g.TW_EVENTS,
                                                                pm4g.TW_CASES_CONTAINED,
                                                                pm4g.TW_CASES_INTERSECTING]
    # an empty batch has no attribute values to point at
    empty = pm4g.BatchSpec([], [], [], [])
    assert empty.Q == 0 and empty.off.tolist() == [0] and empty.vals.size == 0
    assert not empty.struct(0).attr_vals
    with pytest.raises(ValueError):
        pm4g.BatchSpec([[1]], [0, 1], [2, 3], [0, 0])
