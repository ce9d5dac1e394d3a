"""Autotuner for the launch choices of the batched drill-down.

The results of pm4g_batch_dfg never depend on its launch choices. Its time
does, and it varies with the log's activity alphabet, its case lengths and the
sizes of the views. The choices are:

- the cases a warp takes at once (8, 16 or 32);
- the work items per SM that a batch's events are cut into;
- the groups a batch is pipelined in (copies of a group overlap the next
  group's kernels).

The tuner times candidate choices on the caller's own batch: the wall time of
whole calls, which return with every result on the host; the best of a few
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
    """Tunes and applies the batched drill-down's launch choices, with a cache
    keyed by workload signature."""

    def __init__(self, cache_path: str | None = None):
        self.cache_path = cache_path if cache_path is not None else os.environ.get("PM4G_AUTOTUNE_CACHE")
        self.cache: dict[str, dict] = {}
        if self.cache_path and os.path.exists(self.cache_path):
            with open(self.cache_path) as f:
                self.cache = json.load(f)

    @staticmethod
    def apply(ctx: int, choice: dict) -> None:
        for knob, opt in KNOBS.items():
            _pm4g.pm4g_ctx_set_option(ctx, opt, int(choice.get(knob, 0)))

    def _save(self) -> None:
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)

    def tune(self, sig: str, measure, space: dict = SPACE) -> dict:
        """The cached choice for `sig`, else the coordinate-descent minimum of
        measure(choice) -> seconds (remembered)."""
        if sig in self.cache:
            return dict(self.cache[sig]["choice"])
        best, best_t, trials = coordinate_descent(measure, space)
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
