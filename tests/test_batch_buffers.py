"""Result buffers of the batched drill-down (host side, no GPU): every array
grows to at least twice its size, so a server seeing ever larger batches
reallocates (and page-locks) a few times only, and a smaller batch never
shrinks them."""

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
