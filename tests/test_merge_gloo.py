"""Sharding by case and merging, as a multi-GPU run would (CPU only): two gloo
ranks each summarise their case-disjoint shard (with the CPU oracle here), the
summaries are all-gathered and merged, and the merge must equal the whole-log
summary exactly."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import pm4g_synth as synth
from paper_2204_04898_b300.merge import ShardSummary, merge, shard_of


def _summary(L, rows):
    R = oracle.summarize(L.case_id[rows], L.activity[rows], L.ts_ns[rows], L.n_activities)
    return ShardSummary.from_arrays(L.n_activities, R.src, R.dst, R.count, R.sum_lo, R.sum_hi, R.min, R.max,
                                    R.start, R.end, R.freq, R.var_count, R.var_min_case, R.var_off, R.var_acts,
                                    R.case_ids, R.case_variant)


def _check(M, R):
    assert np.array_equal(M.src, R.src) and np.array_equal(M.dst, R.dst)
    assert np.array_equal(M.count, R.count)
    assert M.sums == R.edge_sums()
    assert np.array_equal(M.min, R.min) and np.array_equal(M.max, R.max)
    assert np.array_equal(M.start, R.start) and np.array_equal(M.end, R.end) and np.array_equal(M.freq, R.freq)
    assert np.array_equal(M.var_count, R.var_count) and np.array_equal(M.var_min_case, R.var_min_case)
    assert M.var_seqs == R.variant_seqs()
    assert np.array_equal(M.case_ids, R.case_ids) and np.array_equal(M.case_variant, R.case_variant)


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    from paper_2204_04898_b300.merge import gather_and_merge
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = synth.generate(synth.large_log(4000))
        rows = np.nonzero(shard_of(L.case_id, world) == rank)[0]
        M = gather_and_merge(_summary(L, rows))
        R = oracle.summarize(L.case_id, L.activity, L.ts_ns, L.n_activities)
        _check(M, R)
        q.put((rank, "ok"))
    except Exception as e:  # report to the parent
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_gloo_merge_equals_whole_log():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert results == {0: "ok", 1: "ok"}, results


@pytest.mark.parametrize("k", [1, 3, 7])
def test_merge_of_k_shards_equals_whole_log(k):
    L = synth.generate(synth.very_large_log(3000))
    sh = shard_of(L.case_id, k)
    parts = [_summary(L, np.nonzero(sh == r)[0]) for r in range(k)]
    _check(merge(parts), oracle.summarize(L.case_id, L.activity, L.ts_ns, L.n_activities))


def test_merge_rejects_overlapping_shards():
    L = synth.generate(synth.single_log(500))
    s = _summary(L, np.arange(L.n_events))
    with pytest.raises(ValueError):
        merge([s, s])
