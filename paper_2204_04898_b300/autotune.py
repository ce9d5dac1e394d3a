"""Autotuner for the launch choices of the batched drill-down and of the
single-log pass.

Results never depend on launch choices. Times do, and they vary with the log's
activity alphabet, its case lengths, its row order and (for a batch) the
sizes of the views. The batched drill-down's choices are:

- the cases a warp takes at once (8, 16 or 32);
- the work items per SM that a batch's events are cut into;
- the groups a batch is pipelined in (copies of a group overlap the next
  group's kernels).

The single-log pass's choices (pm4g_load_log followed by the summaries) are:

- the bucket width (2^clb case slots a bucket; 0 = sized to the on-chip
  capacity of the sorting segment pass);
- the units each coarse bucket's second partition level is cut into;
- the warps per block of the streaming segment pass;
- whether logs whose cases come in timestamp order take the streaming pass
  or the sorting pass;
- the global edge table: dense over the A x A pairs or hashed (the
  histogram-versus-hash switch);
- the records a thread stages per tile in each partition level (8, or 4 for
  smaller tiles and one more resident block per SM);
- the coarse fan-out: final buckets per coarse bucket of the first partition
  level (fewer, larger coarse buckets).

The tuner times candidate choices on the caller's own batch or log: the wall
time of whole calls, which return with every result on the host; the best of a few
calls counts. It searches one choice at a time from the defaults (coordinate
descent), applies the fastest to the context and remembers it per workload
signature. The memory lasts for the process; it is also written to a JSON
file when `PM4G_AUTOTUNE_CACHE` names one.
"""

from __future__ import annotations

import json
import math
import os
import time

from . import pm4g as _pm4g

KNOBS = {
    "chunk": _pm4g.OPT_BATCH_CHUNK,
    "items_per_sm": _pm4g.OPT_BATCH_ITEMS_PER_SM,
    "stages": _pm4g.OPT_BATCH_STAGES,
}
DEFAULTS = {"chunk": 16, "items_per_sm": 4, "stages": 4}
SPACE = {"chunk": (8, 16, 32), "items_per_sm": (2, 4, 8), "stages": (1, 2, 4, 8)}

LOAD_KNOBS = {
    "clb": _pm4g.OPT_LOAD_CLB,
    "splits": _pm4g.OPT_LOAD_SPLITS,
    "stream_warps": _pm4g.OPT_STREAM_WARPS,
    "stream_off": _pm4g.OPT_STREAM_OFF,
    "edge_table": _pm4g.OPT_EDGE_TABLE,
    "part1_items": _pm4g.OPT_PART1_ITEMS,
    "part2_items": _pm4g.OPT_PART2_ITEMS,
    "part_fbits": _pm4g.OPT_PART_FBITS,
}
LOAD_DEFAULTS = {"clb": 0, "splits": 0, "stream_warps": 0, "stream_off": 0, "edge_table": 0, "part1_items": 0,
                 "part2_items": 0, "part_fbits": 0}
LOAD_SPACE = {"clb": (0, 6, 7, 8), "splits": (0, 2, 4, 8, 16), "stream_warps": (0, 12, 16, 24),
              "stream_off": (0, 1), "edge_table": (0, 1), "part1_items": (0, 4), "part2_items": (0, 8),
              "part_fbits": (0, 8, 9)}


def load_signature(n_events: int, n_cases: int, n_activities: int, time_ordered: bool, top_k: int,
                   device: str = "") -> str:
    """A single-log workload class: sizes rounded to powers of two, and
    whether the rows are time-ordered (which selects the segment pass)."""
    def p2(x):
        return int(round(math.log2(max(1, int(x)))))
    return (f"load|{device}|ev{p2(n_events)}|cs{p2(n_cases)}|A{p2(n_activities)}|t{int(bool(time_ordered))}"
            f"|k{int(top_k != 0)}")


def signature(n_events: int, n_cases: int, n_activities: int, n_views: int, sub_events: int, var_top_k: int,
              device: str = "") -> str:
    """A workload class: sizes rounded to powers of two (choices tuned on one
    batch carry over to batches of about the same shape)."""
    def p2(x):
        return int(round(math.log2(max(1, int(x)))))
    return (f"{device}|ev{p2(n_events)}|cs{p2(n_cases)}|A{p2(n_activities)}|Q{p2(n_views)}|sub{p2(sub_events)}"
            f"|k{int(var_top_k != 0)}")


def coordinate_descent(measure, space: dict = SPACE, start: dict = DEFAULTS) -> tuple[dict, float, list]:
    """Minimises measure(choice) -> seconds over the grid `space`, one
    coordinate at a time from `start`, until a full sweep changes nothing.
    Returns (best choice, its time, every (choice, time) measured)."""
    seen: dict[tuple, float] = {}
    trials = []

    def t_of(choice):
        key = tuple(sorted(choice.items()))
        if key not in seen:
            seen[key] = float(measure(dict(choice)))
            trials.append((dict(choice), seen[key]))
        return seen[key]

    best = dict(start)
    best_t = t_of(best)
    changed = True
    while changed:
        changed = False
        for knob, values in space.items():
            for v in values:
                if v == best[knob]:
                    continue
                cand = dict(best)
                cand[knob] = v
                t = t_of(cand)
                if t < best_t:
                    best, best_t, changed = cand, t, True
    return best, best_t, trials


class Tuner:
    """Tunes and applies the launch choices of the batched drill-down and of
    the single-log pass, with a cache keyed by workload signature."""

    def __init__(self, cache_path: str | None = None):
        self.cache_path = cache_path if cache_path is not None else os.environ.get("PM4G_AUTOTUNE_CACHE")
        self.cache: dict[str, dict] = {}
        if self.cache_path and os.path.exists(self.cache_path):
            with open(self.cache_path) as f:
                self.cache = json.load(f)

    @staticmethod
    def apply(ctx: int, choice: dict, knobs: dict = KNOBS) -> None:
        for knob, opt in knobs.items():
            _pm4g.pm4g_ctx_set_option(ctx, opt, int(choice.get(knob, 0)))

    def _save(self) -> None:
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)

    def tune(self, sig: str, measure, space: dict = SPACE, start: dict = DEFAULTS) -> dict:
        """The cached choice for `sig`, else the coordinate-descent minimum of
        measure(choice) -> seconds (remembered)."""
        if sig in self.cache:
            return dict(self.cache[sig]["choice"])
        best, best_t, trials = coordinate_descent(measure, space, start)
        self.cache[sig] = {"choice": best, "seconds": best_t, "trials": len(trials)}
        self._save()
        return dict(best)

    def tune_batch(self, ctx: int, log: int, spec, var_top_k: int = 0, out=None, reps: int = 2,
                   device: str = "", space: dict = SPACE) -> dict:
        """Tunes pm4g_batch_dfg(log, spec=spec, out=out, var_top_k=...) on the
        context and leaves the fastest choice applied. `spec` is a
        pm4g.BatchSpec; `out` the caller's reused buffers, if any."""
        first = _pm4g.pm4g_batch_dfg(log, spec=spec, out=out, var_top_k=var_top_k)
        n_events, n_cases = _pm4g.pm4g_log_info(log)
        sig = signature(n_events, n_cases, _pm4g.pm4g_log_activities(log), int(first.n_events.shape[0]),
                        int(first.n_events.sum()), var_top_k, device)

        def measure(choice):
            self.apply(ctx, choice)
            ts = []
            for _ in range(reps):
                t = time.perf_counter()
                _pm4g.pm4g_batch_dfg(log, spec=spec, out=out, var_top_k=var_top_k)
                ts.append(time.perf_counter() - t)
            return min(ts)

        choice = self.tune(sig, measure, space)
        self.apply(ctx, choice)
        return choice

    def tune_load(self, ctx: int, columns, n_activities: int, top_k: int = 1000, reps: int = 2,
                  time_ordered: bool | None = None, device: str = "", space: dict = LOAD_SPACE) -> dict:
        """Tunes the single-log pass on the context (pm4g_load_log of
        `columns` = (case_id, activity, ts_ns), then the frequency and
        performance DFG, start/end counts and pm4g_variants(top_k), then
        pm4g_log_free) and leaves the fastest choice applied."""
        import numpy as np

        def step():
            log = _pm4g.pm4g_load_log(ctx, *columns, n_activities=n_activities)
            try:
                _pm4g.pm4g_dfg(log)
                _pm4g.pm4g_perf_dfg(log)
                _pm4g.pm4g_start_end(log, n_activities)
                _pm4g.pm4g_variants(log, top_k=top_k)
                return _pm4g.pm4g_log_info(log)
            finally:
                _pm4g.pm4g_log_free(log)

        self.apply(ctx, LOAD_DEFAULTS, LOAD_KNOBS)
        n_events, n_cases = step()
        if time_ordered is None:
            ts = columns[2]
            ts = ts.cpu().numpy() if hasattr(ts, "cpu") else np.asarray(ts)
            time_ordered = bool(np.all(ts[1:] >= ts[:-1]))
        sig = load_signature(n_events, n_cases, n_activities, time_ordered, top_k, device)

        def measure(choice):
            self.apply(ctx, choice, LOAD_KNOBS)
            ts_ = []
            for _ in range(reps):
                t = time.perf_counter()
                step()
                ts_.append(time.perf_counter() - t)
            return min(ts_)

        choice = self.tune(sig, measure, space, LOAD_DEFAULTS)
        self.apply(ctx, choice, LOAD_KNOBS)
        return choice
