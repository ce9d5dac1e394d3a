"""Definitional brute force for tiny logs (pure Python, O(N^3)).

Independent of the oracle's code: instead of sorting, it applies the
definitions directly. Within one case, event i precedes event j iff
(ts_i, row_i) < (ts_j, row_j) (Section 3, the ordering by case, timestamp and
absolute index). Event j directly follows event i iff they share a case, i
precedes j, and no other event of that case lies strictly between them
(Section 3, the directly-follows level). A case's sequence places each event at
position = number of events of the case preceding it. Start (end) events have
no predecessor (successor) in their case.
"""

from __future__ import annotations


def _before(ts, i, j):
    return (ts[i], i) < (ts[j], j)


def summary(case, act, ts, n_activities):
    n = len(case)
    A = n_activities
    edges = {}
    start = [0] * A
    end = [0] * A
    freq = [0] * A
    for i in range(n):
        freq[act[i]] += 1
        same = [k for k in range(n) if case[k] == case[i] and k != i]
        if not any(_before(ts, k, i) for k in same):
            start[act[i]] += 1
        if not any(_before(ts, i, k) for k in same):
            end[act[i]] += 1
    for i in range(n):
        for j in range(n):
            if i == j or case[i] != case[j] or not _before(ts, i, j):
                continue
            if any(case[k] == case[i] and k not in (i, j) and _before(ts, i, k) and _before(ts, k, j)
                   for k in range(n)):
                continue
            d = ts[j] - ts[i]
            e = edges.setdefault((act[i], act[j]), [0, 0, None, None])
            e[0] += 1
            e[1] += d
            e[2] = d if e[2] is None else min(e[2], d)
            e[3] = d if e[3] is None else max(e[3], d)
    # sequences
    seqs = {}
    for c in sorted(set(case)):
        members = [k for k in range(n) if case[k] == c]
        pos = {k: sum(1 for q in members if _before(ts, q, k)) for k in members}
        seq = [None] * len(members)
        for k in members:
            seq[pos[k]] = act[k]
        seqs[c] = tuple(seq)
    var = {}
    for c, s in seqs.items():
        v = var.setdefault(s, [0, c])
        v[0] += 1
        v[1] = min(v[1], c)
    order = sorted(var.items(), key=lambda kv: (-kv[1][0], kv[1][1]))
    rank = {s: r for r, (s, _) in enumerate(order)}
    return {
        "edges": {k: tuple(v) for k, v in sorted(edges.items())},
        "start": start,
        "end": end,
        "freq": freq,
        "variants": [(s, v[0], v[1]) for s, v in order],
        "cases": sorted(seqs),
        "case_variant": [rank[seqs[c]] for c in sorted(seqs)],
        "case_len": [len(seqs[c]) for c in sorted(seqs)],
    }


def sorted_rows(case, ts):
    """Rows ordered by the definition: case id, then position within the case."""
    n = len(case)
    out = []
    for c in sorted(set(case)):
        members = [k for k in range(n) if case[k] == c]
        members_pos = sorted(members, key=lambda k: sum(1 for q in members if _before(ts, q, k)))
        out.extend(members_pos)
    return out


def filter_rows(case, act, ts, attr, attr_set, t_lo, t_hi, mode):
    """Rows kept by the drill-down filter, from the definitions: the case's
    attribute is its value at the case's first event; the window is closed."""
    n = len(case)
    keep = []
    aset = set(attr_set)
    for i in range(n):
        members = [k for k in range(n) if case[k] == case[i]]
        first = min(members, key=lambda k: (ts[k], k))
        last = max(members, key=lambda k: (ts[k], k))
        ok = (not aset) or (attr[first] in aset)
        if ok and mode == 2:
            ok = ts[first] >= t_lo and ts[last] <= t_hi
        if ok and mode == 3:
            ok = ts[first] <= t_hi and ts[last] >= t_lo
        if ok and mode == 1:
            ok = t_lo <= ts[i] <= t_hi
        if ok:
            keep.append(i)
    return keep


def _case_members(case, ts, c):
    """Events of case c in order (by the number of its events preceding each)."""
    n = len(case)
    members = [k for k in range(n) if case[k] == c]
    return sorted(members, key=lambda k: sum(1 for q in members if _before(ts, q, k)))


def filter_paths(case, act, ts, pairs, exclude=False):
    """Rows kept by the paths filter, from the definitions: event j matches iff
    some event i of its case directly precedes it (precedes it with no event of
    the case in between) and (act_i, act_j) is one of the pairs."""
    n = len(case)
    pset = {tuple(p) for p in pairs}
    keep = []
    for j in range(n):
        match = False
        for i in range(n):
            if i == j or case[i] != case[j] or not _before(ts, i, j):
                continue
            if any(case[k] == case[j] and k not in (i, j) and _before(ts, i, k) and _before(ts, k, j)
                   for k in range(n)):
                continue
            match = (act[i], act[j]) in pset
        if match != bool(exclude):
            keep.append(j)
    return keep


def filter_cases(case, act, ts, min_events=-1, max_events=-1, min_duration=-1, max_duration=-1,
                 start_set=(), end_set=(), act_set=(), variant_set=(), exclude=False):
    """Rows kept by the case filters, from the definitions (variant ids are the
    ranks of summary())."""
    s = summary(case, act, ts, max(act) + 1 if act else 1)
    rank = dict(zip(s["cases"], s["case_variant"]))
    keep = []
    for c in sorted(set(case)):
        m = _case_members(case, ts, c)
        dur = ts[m[-1]] - ts[m[0]]
        ok = True
        if min_events >= 0 and len(m) < min_events:
            ok = False
        if max_events >= 0 and len(m) > max_events:
            ok = False
        if min_duration >= 0 and dur < min_duration:
            ok = False
        if max_duration >= 0 and dur > max_duration:
            ok = False
        if start_set and act[m[0]] not in start_set:
            ok = False
        if end_set and act[m[-1]] not in end_set:
            ok = False
        if act_set and not any(act[k] in act_set for k in m):
            ok = False
        if variant_set and rank[c] not in variant_set:
            ok = False
        if ok != bool(exclude):
            keep.extend(m)
    return sorted(keep)


def efg(case, act, ts):
    """Eventually-follows pairs from the definitions, with Python integers:
    {(a, b): (count, sum of durations, sum of squared durations)} over pairs of
    distinct events i, j of one case with i preceding j."""
    n = len(case)
    out = {}
    for i in range(n):
        for j in range(n):
            if i == j or case[i] != case[j] or not _before(ts, i, j):
                continue
            d = ts[j] - ts[i]
            c = out.setdefault((act[i], act[j]), [0, 0, 0])
            c[0] += 1
            c[1] += d
            c[2] += d * d
    return {k: tuple(v) for k, v in sorted(out.items())}
