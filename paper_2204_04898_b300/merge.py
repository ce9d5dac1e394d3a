"""Merging summaries of case-disjoint shards (host side).

The method shards naturally by case: every event of a case lives in one shard,
each shard computes its summaries independently, and the summaries combine
exactly (Section 3's definitions only ever relate events of the same case):

* directly-follows edges: counts and 128-bit duration sums add; minima and
  maxima take the minimum and maximum;
* start, end and frequency counts add;
* variants: shards' tables are united by the exact activity sequence, counts
  add, the smallest case id is the minimum, and the union is re-ranked by
  (count descending, smallest case id ascending); each case keeps the variant
  of its sequence.

Each shard contributes its full variant table (``pm4g_variants`` with
top_k = -1): a variant outside one shard's top-k can still rank inside the
merged top-k, so truncated tables do not merge exactly.

Shards are formed by a hash of the case id (``shard_of``). These functions are
the exchange and merge step of a multi-GPU run; ``gather_and_merge`` performs
the exchange over a torch.distributed process group.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MIX = 0x9E3779B97F4A7C15


def shard_of(case_id: np.ndarray, n_shards: int) -> np.ndarray:
    """Shard index of every event: a multiplicative hash of its case id."""
    c = np.asarray(case_id, dtype=np.int64).astype(np.uint64) & np.uint64(0xFFFFFFFF)
    with np.errstate(over="ignore"):
        h = c * np.uint64(MIX)  # wraps modulo 2^64
    return ((h >> np.uint64(32)) % np.uint64(n_shards)).astype(np.int64)


@dataclass
class ShardSummary:
    """The summaries of one shard, in plain Python containers."""

    n_activities: int
    edges: dict = field(default_factory=dict)        # (src, dst) -> [count, sum, min, max]
    start: np.ndarray | None = None                  # uint64[A]
    end: np.ndarray | None = None
    freq: np.ndarray | None = None
    variants: dict = field(default_factory=dict)     # sequence tuple -> [count, min_case]
    case_seq: dict = field(default_factory=dict)     # case id -> sequence tuple

    @classmethod
    def from_arrays(cls, n_activities, src, dst, count, sum_lo, sum_hi, mn, mx, start, end, freq, var_count,
                    var_min_case, var_off, var_acts, case_ids=None, case_variant=None):
        s = cls(n_activities)
        for k in range(len(src)):
            s.edges[(int(src[k]), int(dst[k]))] = [int(count[k]), int(sum_lo[k]) + (int(sum_hi[k]) << 64),
                                                   int(mn[k]), int(mx[k])]
        s.start = np.asarray(start, np.uint64).copy()
        s.end = np.asarray(end, np.uint64).copy()
        s.freq = np.asarray(freq, np.uint64).copy()
        seqs = [tuple(int(a) for a in var_acts[var_off[v]:var_off[v + 1]]) for v in range(len(var_count))]
        for v, q in enumerate(seqs):
            s.variants[q] = [int(var_count[v]), int(var_min_case[v])]
        if case_ids is not None:
            for c, v in zip(case_ids, case_variant):
                s.case_seq[int(c)] = seqs[int(v)]
        return s


@dataclass
class Merged:
    src: np.ndarray
    dst: np.ndarray
    count: np.ndarray
    sums: list            # exact Python ints
    min: np.ndarray
    max: np.ndarray
    start: np.ndarray
    end: np.ndarray
    freq: np.ndarray
    var_count: np.ndarray
    var_min_case: np.ndarray
    var_seqs: list
    case_ids: np.ndarray
    case_variant: np.ndarray


def merge(shards: list[ShardSummary]) -> Merged:
    """Exact merge of case-disjoint shard summaries."""
    if not shards:
        raise ValueError("nothing to merge")
    A = shards[0].n_activities
    edges: dict = {}
    start = np.zeros(A, np.uint64)
    end = np.zeros(A, np.uint64)
    freq = np.zeros(A, np.uint64)
    var: dict = {}
    case_seq: dict = {}
    for s in shards:
        if s.n_activities != A:
            raise ValueError("shards disagree on the activity alphabet")
        for k, (c, sm, mn, mx) in s.edges.items():
            e = edges.get(k)
            if e is None:
                edges[k] = [c, sm, mn, mx]
            else:
                e[0] += c
                e[1] += sm
                e[2] = min(e[2], mn)
                e[3] = max(e[3], mx)
        start += s.start
        end += s.end
        freq += s.freq
        for q, (c, m) in s.variants.items():
            v = var.get(q)
            if v is None:
                var[q] = [c, m]
            else:
                v[0] += c
                v[1] = min(v[1], m)
        for c, q in s.case_seq.items():
            if c in case_seq:
                raise ValueError(f"case {c} appears in two shards")
            case_seq[c] = q
    keys = sorted(edges)
    order = sorted(var.items(), key=lambda kv: (-kv[1][0], kv[1][1]))
    rank = {q: r for r, (q, _) in enumerate(order)}
    cids = np.array(sorted(case_seq), dtype=np.int32)
    return Merged(
        src=np.array([k[0] for k in keys], np.int32), dst=np.array([k[1] for k in keys], np.int32),
        count=np.array([edges[k][0] for k in keys], np.uint64), sums=[edges[k][1] for k in keys],
        min=np.array([edges[k][2] for k in keys], np.uint64), max=np.array([edges[k][3] for k in keys], np.uint64),
        start=start, end=end, freq=freq,
        var_count=np.array([v[0] for _, v in order], np.uint64),
        var_min_case=np.array([v[1] for _, v in order], np.int32),
        var_seqs=[q for q, _ in order],
        case_ids=cids, case_variant=np.array([rank[case_seq[int(c)]] for c in cids], np.int32))


def gather_and_merge(local: ShardSummary, group=None) -> Merged:
    """All-gather every rank's shard summary over torch.distributed and merge
    them (the one exchange step of a sharded run)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, local, group=group)
    return merge(parts)
