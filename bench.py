#!/usr/bin/env python
"""Throughput of the single-log pass: load and format a columnar event log,
then frequency DFG, performance DFG, start/end activities and the variant
table, on one B300 per process.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload very_large_log]
    python bench.py --impl reference ...    # the CPU oracle on host cores

One step = pm4g_load_log (device-resident columns) + pm4g_dfg + pm4g_perf_dfg +
pm4g_start_end + pm4g_variants(top_k) + pm4g_log_free. Prints one JSON line.
Under torchrun every rank processes its own copy of the workload (replicas;
weak scaling); value = events of all ranks / max rank time.

    python bench.py --mode drilldown [--views 4096] [--plain-views 4096]
    python bench.py --mode filters
    python bench.py --mode efg

Drill-down: a resident drilldown_log (100M events, A = 2000, case attributes)
and 4096 drill-down views (attribute set + time window, EVENTS mode). One step
= one pm4g_batch_dfg call over all views (filter + frequency/performance DFG +
start/end per view, results on the host); value = sub-log events / step time.
The same views through plain calls (pm4g_filter + pm4g_perf_dfg +
pm4g_start_end + pm4g_log_free per view) are timed once beside it.

Filters on derived results: the resident very_large_log and a fixed mix of six
filters (the 20 most frequent paths; cases of at least the median size; cases
whose throughput time lies between its quartiles; cases ending in one of the
three most frequent end activities; cases containing one of the five rarest
activities; cases of the ten most frequent variants). One step = each filter,
then pm4g_perf_dfg of its sub-log and pm4g_log_free; value = input events of
the six filters / step time.

Eventually-follows graph / temporal profile: the resident very_large_log; one
step = pm4g_efg (every ordered pair of events of a case, exact count, sum and
sum of squares per activity pair, means and deviations, results on the host);
value = pairs / step time (and events / step time beside it).
"""

from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pm4g_synth as synth  # noqa: E402

METRIC = "events/s for DFG+perf-DFG+variants (single-log pass)"
UNIT = "events/s"
FALLBACK_HBM_GBS = 6400.0
# Algorithmic bytes (the byte model of the method, not of this implementation):
# read case+activity+timestamp once (16 B/event), write activity+timestamp once
# in case-grouped order (12 B/event), read them back (12 B/event), write the
# case-to-variant id (4 B/case). Split by the kernel that does each part.
ALG_BYTES = {
    "partition": (28.0, 0.0),  # (per event, per case), over the kernel's launches in one step
    "bucket_scatter": (28.0, 0.0),
    "segment": (12.0, 0.0),
    "segment_sort": (12.0, 0.0),
    "variants": (0.0, 4.0),
}
# Source file of each timed kernel: a DRAM-traffic figure recorded under
# profiles/ is used only while this file is unchanged since the capture.
KERNEL_SOURCE = {"segment": "stream.cu", "segment_sort": "segment.cu", "partition": "format.cu",
                 "bucket_scatter": "format.cu",
                 "variants": "summaries.cu"}


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary
    (profiles/<kernel>_<workload>.md, lines 'source_sha256: ...' and
    'dram_bytes_per_launch: ...'), or None if absent or stale."""
    import hashlib
    src = KERNEL_SOURCE.get(kernel)
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not src or not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(os.path.join(ROOT, "paper_2204_04898_b300", "csrc", src), "rb").read()).hexdigest()
    fields = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            fields[k.strip().lstrip("-* `").rstrip("`")] = v.strip().strip("`")
    if fields.get("source_sha256") != sha:
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="engine", choices=["engine", "reference"])
    p.add_argument("--workload", default="very_large_log", choices=sorted(synth.WORKLOADS))
    p.add_argument("--cases", type=int, default=0, help="override the number of cases (0 = workload default)")
    p.add_argument("--top-k", type=int, default=1000)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-cases", type=int, default=1_000_000)
    p.add_argument("--mode", default="single", choices=["single", "drilldown", "serve", "filters", "efg"])
    p.add_argument("--rates", default="100,300,1000,3000,10000", help="serve: Poisson request rates (req/s)")
    p.add_argument("--seconds", type=float, default=3.0, help="serve: seconds of arrivals per rate")
    p.add_argument("--views", type=int, default=4096)
    p.add_argument("--plain-views", type=int, default=4096, help="views timed through plain calls")
    p.add_argument("--no-tune", action="store_true", help="single mode: keep the default launch choices")
    p.add_argument("--no-drilldown", action="store_true", help="single mode: leave out the drill-down object")
    p.add_argument("--no-serving", action="store_true", help="single mode: leave out the serving object")
    p.add_argument("--dd-steps", type=int, default=10, help="single mode: timed drill-down batches")
    p.add_argument("--serve-rates", default="300,1000,3000", help="single mode: serving rates (req/s)")
    p.add_argument("--serve-seconds", type=float, default=10.0, help="single mode: seconds of arrivals per rate")
    return p.parse_args()


def workload_spec(args):
    spec = synth.WORKLOADS[args.workload]()
    if args.cases:
        spec = spec.scaled(args.cases, spec.name)
    return spec


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples over the timed region.

    Every nvidia-smi sample stalls the GPU's work for a few milliseconds on
    this driver (measured: about 2.5 ms per sample, whatever fields are
    queried), so it samples once a second, and a timed region shorter than
    that is started so that one sample falls in its middle: the sampler's
    phase and period are read from the arrivals of its second and third
    samples, and the region's length from one untimed step on a warm GPU
    (the warm-up steps' time when no such step is given)."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_S = 1.0

    def __init__(self, gpu_index: int, warm=None, steps: int = 0, warm_steps: int = 3, pad=None,
                 period_s: float = 1.0):
        self.PERIOD_S = period_s
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.warm = warm  # untimed steps run after the sampler starts, so the idle wait does not reach the timed steps
        self.steps = steps  # timed steps that follow (0: no alignment)
        self.warm_steps = warm_steps
        self.pad = pad  # one untimed step, run instead of idling until the aligned start

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="pm4g_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms",
                                          str(int(self.PERIOD_S * 1000))],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # the arrivals of the second and third samples give the sampler's
        # phase and period (its start-up is over by then)
        t0 = time.time()
        t_sample, period, seen = None, self.PERIOD_S, {}
        while self.proc is not None and time.time() - t0 < 10.0 + 2 * self.PERIOD_S:
            n_lines = self._lines()
            for m in (2, 3):
                if n_lines >= m and m not in seen:
                    seen[m] = time.time()
            if 3 in seen:
                t_sample = seen[3]
                if 2 in seen and 0.5 * self.PERIOD_S < seen[3] - seen[2] < 1.5 * self.PERIOD_S:
                    period = seen[3] - seen[2]
                break
            time.sleep(0.002)
        if self.warm is not None:
            tw = time.time()
            self.warm()
            t_warm = time.time() - tw
            per_step = t_warm / max(1, self.warm_steps)
            if self.pad is not None:  # one more step, timed on a warm GPU
                tp = time.time()
                self.pad()
                per_step = time.time() - tp
            region = per_step * self.steps
            w2 = per_step * self.warm_steps  # the warm-up that runs last
            if t_sample is not None and 0 < region < period:
                # start so that the next sample lands in the middle of the
                # region; the GPU keeps working until then (an idle GPU is
                # slower for its first steps): untimed steps, an idle gap
                # shorter than one step, then the warm-up again (it also
                # resets the counters of the timed region)
                now = time.time()
                k = max(1, int((now + per_step + w2 - t_sample + region / 2) / period) + 1)
                start = t_sample + k * period - region / 2
                if self.pad is not None:
                    while time.time() + per_step + w2 <= start:
                        self.pad()
                gap = start - w2 - time.time()
                if gap > 0:
                    time.sleep(gap)
                self.warm()
        self.t_begin = time.time()
        return self

    def __exit__(self, *exc):
        self.t_end = time.time()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        """Median SM clock, maximum clock and throttle reasons of the samples
        taken in the timed region (all samples if none fell in it)."""
        import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 10:
                    continue
                try:
                    t = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((t, float(f[2]), float(f[3]),
                                 [nm for nm, v in zip(names, f[6:10]) if v.lower().startswith("active")]))
                except ValueError:
                    continue
        except Exception:
            pass
        t0, t1 = getattr(self, "t_begin", None), getattr(self, "t_end", None)
        inside = [r for r in rows if t0 is not None and t1 is not None and t0 <= r[0] <= t1]
        use = inside or rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "samples_in_region": 0}
        near = [round(r[0] - t0, 3) for r in rows if t0 is not None and t1 is not None and -2 <= r[0] - t0 <= t1 - t0 + 2]
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "reasons": sorted({nm for r in use for nm in r[3]}), "samples": len(use),
                "samples_in_region": len(inside), "period_s": self.PERIOD_S,
                "region_s": round(t1 - t0, 3) if t0 is not None and t1 is not None else None,
                "sample_offsets_s": near}


def run_reference(args):
    """The CPU oracle on the machine's host cores, on a bounded sample per step."""
    import oracle
    rank, world, _ = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    spec = workload_spec(args)
    sample_cases = max(1000, min(spec.n_cases, args.cpu_sample_cases // 4))
    L = synth.generate(spec.scaled(sample_cases))
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        oracle.summarize(L.case_id, L.activity, L.ts_ns, L.n_activities)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    total = sum(times)
    value = L.n_events * len(times) / total
    sample = f"{spec.name} law with {sample_cases} cases ({L.n_events} events) per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": spec.name, "n_cases": sample_cases, "n_events": L.n_events,
                       "n_activities": spec.n_activities},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


DD_METRIC = "sub-log events/s for filter+DFG+perf-DFG+start/end+variants over drill-down views (batched)"


def drilldown_workload(args):
    spec = synth.drilldown_log(args.cases) if args.cases else synth.drilldown_log()
    return spec


def oracle_views(oracle, L, views):
    """Filter then summarise every view with the oracle; returns the sub-log events."""
    n = 0
    for v in views:
        rows = oracle.filter_rows(L.case_id, L.activity, L.ts_ns, L.case_attr, L.n_activities, v.attr_set,
                                  v.t_lo, v.t_hi, 1)
        oracle.summarize(L.case_id[rows], L.activity[rows], L.ts_ns[rows], L.n_activities)
        n += rows.shape[0]
    return n


def run_reference_drilldown(args):
    """The CPU oracle (filter, then summarise) on a bounded sample of views."""
    import oracle
    rank, world, _ = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    spec = drilldown_workload(args)
    small = spec.scaled(max(2000, min(spec.n_cases, args.cpu_sample_cases // 4)))
    L = synth.generate(small)
    views = synth.drilldown_specs(L, n_views=8, lo_events=1e3, hi_events=max(2e3, L.n_events / 4))
    times, ev = [], 0
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        n = oracle_views(oracle, L, views)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
            ev += n
    total = sum(times)
    value = ev / total
    sample = f"{len(views)} views of a {small.name} law log with {small.n_cases} cases ({L.n_events} events) per step"
    line = {"impl": "reference", "metric": DD_METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": "drilldown_views", "n_cases": small.n_cases,
                                            "n_events": L.n_events, "n_activities": small.n_activities,
                                            "n_views": len(views)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def drilldown_core(args, local: int, steps: int, warmup: int, plain_views: int, tune: bool = True,
                   cpu_baseline: bool = True) -> dict:
    """Batched drill-down on one GPU: the resident drilldown_log, its 4,096
    views, `steps` timed pm4g_batch_dfg calls (CUDA events on the context
    stream; inputs resident, results into reused page-locked buffers), then
    the first `plain_views` views through plain calls."""
    import torch
    from paper_2204_04898_b300 import pm4g
    spec = drilldown_workload(args)
    t_gen = time.perf_counter()
    L = synth.generate(spec, pinned=True)
    t_gen = time.perf_counter() - t_gen
    A = L.n_activities
    views = synth.drilldown_specs(L, n_views=args.views)
    sets = [v.attr_set for v in views]
    lo = [v.t_lo for v in views]
    hi = [v.t_hi for v in views]
    modes = [pm4g.TW_EVENTS] * len(views)
    dev = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns, L.case_attr)]
    stream = torch.cuda.Stream()
    ctx = pm4g.pm4g_ctx_create(local, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    log = pm4g.pm4g_load_log(ctx, *dev[:3], case_attr=dev[3], n_activities=A)
    torch.cuda.synchronize()
    load_ms = 1e3 * (time.perf_counter() - t)
    del dev
    buf = pm4g.BatchBuffers(len(views), A, 0)  # page-locked result buffers, reused every step
    bspec = pm4g.BatchSpec(sets, lo, hi, modes)  # the views as flat arrays, built once
    t = time.perf_counter()
    vk = args.top_k
    B = pm4g.pm4g_batch_dfg(log, out=buf, var_top_k=vk, spec=bspec)  # first call builds the index
    first_ms = 1e3 * (time.perf_counter() - t)
    sub_events = int(B.n_events.sum())
    out_edges = int(B.edge_off[-1])
    out_vars = int(B.var_off[-1])
    # launch choices (cases per warp chunk, items per SM, pipeline groups) by
    # the autotuner, timed on this batch before the timed region
    tuned, tune_s = None, 0.0
    if tune:
        from paper_2204_04898_b300 import autotune
        t = time.perf_counter()
        tuned = autotune.Tuner().tune_batch(ctx, log, bspec, var_top_k=vk, out=buf, reps=2,
                                            device=torch.cuda.get_device_name(local))
        tune_s = time.perf_counter() - t
    for _ in range(max(0, warmup - 1)):
        pm4g.pm4g_batch_dfg(log, out=buf, var_top_k=vk, spec=bspec)
    # CUDA events around the batch kernel's launches only (level 2), so the
    # events add no host work to the other launches of the step
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 2)
    pm4g.pm4g_ctx_timing_reset(ctx)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = [0]

    def rewarm():
        for _ in range(3):
            pm4g.pm4g_batch_dfg(log, out=buf, var_top_k=vk, spec=bspec)
        pm4g.pm4g_ctx_timing_reset(ctx)  # the timed steps alone are counted
        launches0[0] = pm4g.pm4g_ctx_timing(ctx, "launches")[0]

    with ClockSampler(local, rewarm, steps=steps,
                      pad=lambda: pm4g.pm4g_batch_dfg(log, out=buf, var_top_k=vk, spec=bspec)) as clk:
        torch.cuda.synchronize()
        t = time.perf_counter()
        ev0.record(stream)
        for _ in range(steps):
            pm4g.pm4g_batch_dfg(log, out=buf, var_top_k=vk, spec=bspec)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t
    dev_ms = ev0.elapsed_time(ev1) / steps
    wall_ms = 1e3 * wall / steps
    n_b, batch_ms = pm4g.pm4g_ctx_timing(ctx, "batch_dfg")
    launches = pm4g.pm4g_ctx_timing(ctx, "launches")[0] - launches0[0]
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 0)
    # plain calls over the first plain_views views
    P = min(plain_views, len(views))
    plain = None
    if P > 0:
        torch.cuda.synchronize()
        t = time.perf_counter()
        pev = 0
        for i in range(P):
            f = pm4g.pm4g_filter(log, sets[i], lo[i], hi[i], pm4g.TW_EVENTS)
            try:
                pm4g.pm4g_perf_dfg(f)
                pm4g.pm4g_start_end(f, A)
                pm4g.pm4g_variants(f, top_k=vk)
                pev += pm4g.pm4g_log_info(f)[0]
            finally:
                pm4g.pm4g_log_free(f)
        torch.cuda.synchronize()
        pt = time.perf_counter() - t
        plain = {"value": pev / pt, "unit": UNIT, "views": P, "sub_log_events": pev, "ms_per_view": 1e3 * pt / P,
                 "timing": "host wall clock over the plain calls, results on the host",
                 "calls": "pm4g_filter + pm4g_perf_dfg + pm4g_start_end + pm4g_variants + pm4g_log_free per view"}
    cpu = None
    if cpu_baseline:
        import oracle
        small = spec.scaled(max(2000, min(spec.n_cases, args.cpu_sample_cases // 4)))
        S = synth.generate(small)
        sv = synth.drilldown_specs(S, n_views=8, lo_events=1e3, hi_events=max(2e3, S.n_events / 4))
        t = time.perf_counter()
        n = oracle_views(oracle, S, sv)
        dt = time.perf_counter() - t
        cpu = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{len(sv)} views of a {small.name} law log with {small.n_cases} cases "
                         f"({S.n_events} events), one run, {dt:.1f} s on 1 of {os.cpu_count()} host cores"}
    res_bytes = out_edges * (4 + 4 + 5 * 8 + 8) + len(views) * (3 * A * 8 + 24)
    spec_bytes = sum(x.size for x in sets) * 4 + len(views) * (8 + 8 + 8 + 4)
    pm4g.pm4g_log_free(log)
    pm4g.pm4g_ctx_destroy(ctx)
    del buf, B
    peak, peak_kind = peaks()
    # the method's bytes: activity + timestamp of every sub-log event, read
    # once from the resident formatted log; a step's views run as a few
    # launches (pipelined groups), so per launch is the step's bytes / launches
    per_launch = 12.0 * sub_events * steps / max(1, n_b)
    kernel_ms = batch_ms / max(1, n_b)
    achieved = per_launch / (kernel_ms * 1e-3) / 1e9 if kernel_ms > 0 else 0.0
    value = sub_events * 1e3 / dev_ms
    return {
        "value": value, "ms_per_step": dev_ms, "wall_ms_per_step": wall_ms, "steps": steps, "warmup": warmup,
        "spec": spec, "n_events": L.n_events, "n_activities": A, "n_views": len(views),
        "sub_log_events": sub_events, "out_edges": out_edges, "out_variants": out_vars, "var_top_k": vk,
        "launches_per_step": n_b / max(1, steps), "tuned": tuned, "tune_s": tune_s, "load_ms": load_ms,
        "first_ms": first_ms, "t_gen": t_gen, "plain": plain,
        "ratio_vs_plain": (value / plain["value"]) if plain else None,
        "roofline": {"bound": "hbm", "kernel": "batch_dfg", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "alg_bytes_per_launch": per_launch, "launch_ms": kernel_ms,
                     "note": "12 B (activity + timestamp) per sub-log event; overlapping views re-read the "
                             "resident log mostly from L2"},
        "gpu_launches": int(launches), "clocks": clk.summary(),
        "e2e": {"value": sub_events * 1e3 / wall_ms, "unit": UNIT, "h2d_bytes_per_step": int(spec_bytes),
                "d2h_bytes_per_step": int(res_bytes)},
        "cpu_baseline": cpu,
    }


def run_drilldown(args):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
    r = drilldown_core(args, local, args.steps, args.warmup, args.plain_views,
                       cpu_baseline=rank == 0 and not args.no_cpu_baseline)
    ms, wall_ms = r["ms_per_step"], r["wall_ms_per_step"]
    if dist is not None:
        t_ = torch.tensor([ms, wall_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t_, op=dist.ReduceOp.MAX)
        ms, wall_ms = float(t_[0]), float(t_[1])
    if rank != 0:
        return
    spec = r["spec"]
    line = {
        "metric": DD_METRIC, "value": r["sub_log_events"] * world * 1e3 / ms, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "drilldown_views", "log": spec.name, "n_events": r["n_events"],
                   "n_cases": spec.n_cases, "n_activities": r["n_activities"], "n_views": r["n_views"],
                   "mode": "EVENTS", "sub_log_events": r["sub_log_events"], "out_edges": r["out_edges"],
                   "var_top_k": r["var_top_k"], "out_variants": r["out_variants"],
                   "batch_dfg_launches_per_step": r["launches_per_step"],
                   "autotuned": r["tuned"], "autotune_s": round(r["tune_s"], 2),
                   "l2": "resident log %.1f GB of activity+timestamp, larger than L2; no flush"
                         % (12 * r["n_events"] / 1e9),
                   "load_ms": round(r["load_ms"], 1), "first_call_ms_with_index": round(r["first_ms"], 1),
                   "parallelism": f"replicas x{world}", "generate_s": round(r["t_gen"], 1)},
        "wall_ms_per_step": wall_ms,
        "plain": r["plain"],
        "ratio_vs_plain": r["ratio_vs_plain"],
        "roofline": r["roofline"],
        "gpu_launches": r["gpu_launches"],
        "clocks": r["clocks"],
        "e2e": {**r["e2e"], "value": r["sub_log_events"] * world * 1e3 / wall_ms},
        "cpu_baseline": r["cpu_baseline"],
    }
    print(json.dumps(line), flush=True)


SERVE_METRIC = "served events/s (filter+DFG views and uploads) under a Poisson request mix; p50/p99 request ms"


def small_log_latency(pm4g, device: int, n_cases: int = 500, reps: int = 50) -> dict:
    """Latency of the DFG, performance DFG and start/end counts of a small log
    (workload-3 law, about 10k events, host columns) through the regular calls,
    the allocation-free call, and the allocation-free call captured once in a
    CUDA graph and replayed (median ms over `reps` calls, results on the device
    for the last two, copied to the host for the first)."""
    import torch
    L = synth.generate(synth.very_large_log(n_cases).scaled(n_cases, "small_upload"), pinned=True)
    A = L.n_activities
    ctx = pm4g.pm4g_ctx_create(device)
    dev = [torch.from_numpy(x).cuda(device) for x in (L.case_id, L.activity, L.ts_ns)]
    g = pm4g.NoallocGraph(A, device)

    def regular():
        log = pm4g.pm4g_load_log(ctx, L.case_id, L.activity, L.ts_ns, n_activities=A)
        try:
            pm4g.pm4g_perf_dfg(log)
            pm4g.pm4g_start_end(log, A)
        finally:
            pm4g.pm4g_log_free(log)

    def noalloc():
        pm4g.pm4g_dfg_noalloc(*dev, n_activities=A)
        torch.cuda.synchronize(device)

    def graph():
        g.run(L.case_id, L.activity, L.ts_ns)

    out = {"events": int(L.n_events), "n_activities": A}
    for name, fn in (("regular_ms", regular), ("noalloc_ms", noalloc), ("graph_replay_ms", graph)):
        fn()
        ts = []
        for _ in range(reps):
            t = time.perf_counter()
            fn()
            ts.append(1e3 * (time.perf_counter() - t))
        out[name] = round(float(np.median(ts)), 3)
    pm4g.pm4g_ctx_destroy(ctx)
    return out


def serve_core(args, local: int, rates: list, seconds: float, small_log: bool = True) -> dict:
    """Serving on one GPU: a resident serving_log and, at each rate, Poisson
    arrivals for `seconds` of 70 % filter+DFG, 20 % variants top-10, 10 %
    uploads of LogUniform(10k, 50M)-event logs of the workload-3 law; latency
    from arrival to result on the host."""
    import torch
    from paper_2204_04898_b300 import pm4g
    from paper_2204_04898_b300.serve import GpuEngine, Request, Server, latency_summary
    spec = synth.serving_log(args.cases) if args.cases else synth.serving_log()
    t_gen = time.perf_counter()
    L = synth.generate(spec, pinned=True)
    A = L.n_activities
    rng = np.random.default_rng(20220416)
    # upload pool: sizes LogUniform(10k, 50M), workload-3 law, page-locked host columns
    pool = []
    for k, n in enumerate(np.exp(rng.uniform(np.log(1e4), np.log(5e7), 6))):
        cases = max(500, int(n / 20.66))
        u = synth.generate(synth.very_large_log(cases).scaled(cases, f"upload{k}"), pinned=True)
        pool.append(u)
    views = synth.drilldown_specs(L, n_views=2048, seed=20220417)
    t_gen = time.perf_counter() - t_gen
    # the queries' context runs on a high-priority stream: their blocks are
    # scheduled ahead of the uploads' whenever both wait for an SM
    qstream = torch.cuda.Stream(device=local, priority=-1)
    ctx = pm4g.pm4g_ctx_create(local, stream=qstream.cuda_stream)
    cols = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns, L.case_attr)]
    t = time.perf_counter()
    log = pm4g.pm4g_load_log(ctx, *cols[:3], case_attr=cols[3], n_activities=A)
    load_ms = 1e3 * (time.perf_counter() - t)
    del cols
    torch.cuda.empty_cache()
    eng = GpuEngine(pm4g, local, log, ctx, upload_slots=2)
    # warm: drill-down index, variant table, a large batch's result buffers,
    # upload contexts
    eng.batch_dfg([Request("dfg", attr_set=v.attr_set, t_lo=v.t_lo, t_hi=v.t_hi, mode=pm4g.TW_EVENTS)
                   for v in views[:1024]])
    eng.variants(10)
    for slot in range(2):  # every upload slot's context, pools and staging buffers
        eng.upload(Request("upload", columns=(pool[0].case_id, pool[0].activity, pool[0].ts_ns), n_activities=A),
                   slot)
    srv = Server(eng, upload_slots=2)
    per_rate = []
    # a sample every 5 s: each one stalls the GPU's work for milliseconds,
    # which shows in the latency tail of the requests queued behind it
    with ClockSampler(local, period_s=5.0) as clk:
        for rate in rates:
            n = max(1, int(rng.poisson(rate * seconds)))
            arrivals = np.sort(rng.uniform(0, seconds, n))
            kinds = rng.choice(3, n, p=[0.7, 0.2, 0.1])
            reqs = []
            for kd in kinds:
                if kd == 0:
                    v = views[int(rng.integers(len(views)))]
                    reqs.append(Request("dfg", attr_set=v.attr_set, t_lo=v.t_lo, t_hi=v.t_hi, mode=pm4g.TW_EVENTS))
                elif kd == 1:
                    reqs.append(Request("variants", top_k=10))
                else:
                    u = pool[int(rng.integers(len(pool)))]
                    reqs.append(Request("upload", columns=(u.case_id, u.activity, u.ts_ns), n_activities=A))
            torch.cuda.synchronize()
            # the Python garbage collector is off while a rate runs: its full
            # collections stop every thread of the process (the server's
            # workers included) for 50-130 ms at this request volume
            gc.collect()
            gc.disable()
            try:
                t0 = time.perf_counter()
                for r, at in zip(reqs, arrivals):
                    d = t0 + at - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    r.t_arrival = t0 + at
                    srv.submit(r)
                for r in reqs:
                    r.done.wait(600)
            finally:
                gc.enable()
            t_end = max(r.t_done for r in reqs)
            ok = [r for r in reqs if r.done.is_set() and r.error is None]
            ev = sum(r.result["n_events"] for r in ok if r.kind in ("dfg", "upload"))
            h2d = sum(16 * r.columns[0].shape[0] for r in ok if r.kind == "upload")
            d2h = sum(sum(v.nbytes for v in r.result.values() if isinstance(v, np.ndarray)) for r in ok)
            entry = {"rate": rate, "requests": n, "completed": len(ok),
                     "errors": sum(1 for r in reqs if r.error is not None),
                     "events_per_s": ev / (t_end - t0), "wall_s": t_end - t0,
                     "all": latency_summary(reqs),
                     "dfg": latency_summary([r for r in reqs if r.kind == "dfg"]),
                     "variants": latency_summary([r for r in reqs if r.kind == "variants"]),
                     "upload": latency_summary([r for r in reqs if r.kind == "upload"]),
                     "dfg_batches": len(srv.batches), "upload_h2d_bytes": h2d, "d2h_bytes": d2h,
                     "error_samples": sorted({f"{r.kind}: {r.error!r}"[:200] for r in reqs if r.error is not None})[:3]}
            srv.batches.clear()
            per_rate.append(entry)
    srv.close()
    launches = pm4g.pm4g_ctx_timing(ctx, "launches")[0]
    eng.close()
    pm4g.pm4g_log_free(log)
    pm4g.pm4g_ctx_destroy(ctx)
    return {"spec": spec, "n_events": L.n_events, "n_activities": A, "per_rate": per_rate,
            "upload_events": [int(u.n_events) for u in pool], "seconds_per_rate": seconds, "load_ms": load_ms,
            "t_gen": t_gen, "gpu_launches": int(launches), "clocks": clk.summary(),
            "small_log": small_log_latency(pm4g, local) if small_log else None}


def run_serve(args):
    import torch
    _, _, local = dist_info()
    torch.cuda.set_device(local)
    r = serve_core(args, local, [float(x) for x in args.rates.split(",") if x], args.seconds)
    per_rate = r["per_rate"]
    spec = r["spec"]
    top = per_rate[-1]
    line = {
        "metric": SERVE_METRIC, "value": top["events_per_s"], "unit": UNIT, "n_gpus": 1, "steps": len(per_rate),
        "warmup": 1, "ms_per_step": 1e3 * top["wall_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "serving_mix", "log": spec.name, "n_events": r["n_events"], "n_cases": spec.n_cases,
                   "n_activities": r["n_activities"], "mix": "70% filter+DFG (EVENTS), 20% variants top-10, 10% upload",
                   "upload_events": r["upload_events"], "seconds_per_rate": r["seconds_per_rate"],
                   "load_ms": round(r["load_ms"], 1), "generate_s": round(r["t_gen"], 1),
                   "l2": "resident log larger than L2; no flush", "python_gc": "off while a rate runs"},
        "rates": per_rate,
        "small_log": r["small_log"],
        "p50_ms": top["all"].get("p50_ms"), "p99_ms": top["all"].get("p99_ms"),
        "gpu_launches": r["gpu_launches"],
        "clocks": r["clocks"],
        # every latency above is end to end (arrival to result on the host)
        "e2e": {"value": top["events_per_s"], "unit": UNIT, "h2d_bytes_per_step": int(top["upload_h2d_bytes"]),
                "d2h_bytes_per_step": int(top["d2h_bytes"])},
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


FILTERS_METRIC = "input events/s for filter + performance DFG of the sub-log (six-filter mix)"


def filter_mix(oracle_summary, L):
    """The benchmark's six filters, from the log's own summaries: (name, kind,
    arguments) with kind 'paths' or 'cases'."""
    R = oracle_summary
    order = np.argsort(-R["count"].astype(np.int64), kind="stable")[:20]
    pairs = [(int(R["src"][i]), int(R["dst"][i])) for i in order]
    lens, dur = R["case_len"], R["duration"]
    return [
        ("paths_top20", "paths", {"pairs": pairs}),
        ("size_ge_median", "cases", {"min_events": int(np.median(lens))}),
        ("duration_iqr", "cases", {"min_duration": int(np.percentile(dur, 25)),
                                   "max_duration": int(np.percentile(dur, 75))}),
        ("end_top3", "cases", {"end_set": [int(a) for a in np.argsort(-R["end"].astype(np.int64))[:3]]}),
        ("contains_rare5", "cases", {"act_set": [int(a) for a in np.argsort(R["freq"].astype(np.int64))[:5]]}),
        ("variant_top10", "cases", {"variant_set": list(range(10))}),
    ]


def run_filters(args):
    """Filters on derived results over the resident single log."""
    if args.impl == "reference":
        return run_reference_filters(args)
    import torch
    from paper_2204_04898_b300 import pm4g
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    spec = workload_spec(args)
    t_gen = time.perf_counter()
    L = synth.generate(spec, pinned=True)
    t_gen = time.perf_counter() - t_gen
    N, A = L.n_events, L.n_activities
    dev = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns)]
    stream = torch.cuda.Stream()
    ctx = pm4g.pm4g_ctx_create(local, stream=stream.cuda_stream)
    log = pm4g.pm4g_load_log(ctx, *dev, n_activities=A)
    # the filters' arguments from the log's own summaries (through the engine)
    p = pm4g.pm4g_perf_dfg(log)
    st, en, fr = pm4g.pm4g_start_end(log, A)
    e = pm4g.pm4g_log_export(log)
    starts = np.flatnonzero(np.r_[True, e["case_id"][1:] != e["case_id"][:-1]])
    ends = np.r_[starts[1:], e["case_id"].size] - 1
    summ = {"count": p.count, "src": p.src, "dst": p.dst, "end": en, "freq": fr,
            "case_len": ends - starts + 1,
            "duration": (e["ts_ns"][ends].astype(np.uint64) - e["ts_ns"][starts].astype(np.uint64)).astype(np.int64)}
    summ_cases = summ["case_len"].size
    del e
    mix = filter_mix(summ, L)

    def run_one(kind, kw):
        f = pm4g.pm4g_filter_paths(log, **kw) if kind == "paths" else pm4g.pm4g_filter_cases(log, **kw)
        try:
            d = pm4g.pm4g_perf_dfg(f)
            return pm4g.pm4g_log_info(f)[0], d
        finally:
            pm4g.pm4g_log_free(f)

    kept = {}
    for name, kind, kw in mix:
        kept[name] = run_one(kind, kw)[0]
    for _ in range(args.warmup):
        for name, kind, kw in mix:
            run_one(kind, kw)
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 2)  # the filter and segment kernels
    pm4g.pm4g_ctx_timing_reset(ctx)
    launches0 = pm4g.pm4g_ctx_timing(ctx, "launches")[0]
    per = {name: 0.0 for name, _, _ in mix}
    d2h = 0
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    def rewarm():
        for name, kind, kw in mix:
            run_one(kind, kw)
        pm4g.pm4g_ctx_timing_reset(ctx)  # the timed steps alone are counted

    with ClockSampler(local, rewarm, steps=args.steps, warm_steps=1,
                      pad=lambda: [run_one(kind, kw) for _, kind, kw in mix]) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            for name, kind, kw in mix:
                t = time.perf_counter()
                _, d = run_one(kind, kw)
                per[name] += time.perf_counter() - t
                d2h += sum(x.nbytes for x in (d.src, d.dst, d.count, d.sum_lo, d.sum_hi, d.min, d.max, d.mean))
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    kt = {k: pm4g.pm4g_ctx_timing(ctx, k) for k in ("filter", "segment", "segment_sort", "partition", "export",
                                                   "scan", "dfg",
                                                   "variants", "radix_sort", "bucket_hist", "stats")}
    launches = pm4g.pm4g_ctx_timing(ctx, "launches")[0] - launches0
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 0)
    if dist is not None:
        t_ = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t_, op=dist.ReduceOp.MAX)
        ms = float(t_[0])
    value = len(mix) * N * world * 1e3 / ms
    kt = {k: v for k, v in kt.items() if v[0] > 0}
    dom = max(kt, key=lambda k: kt[k][1])
    peak, peak_kind = peaks()
    # the method's bytes of a filter: read every event's activity and
    # timestamp once (12 B) and write the kept ones (12 B each); the sub-log's
    # own formatting (its segment pass) is not charged to the filter kernels
    alg = sum(12.0 * N + 12.0 * kept[name] for name, _, _ in mix)
    filt_ms = kt.get("filter", (0, 0.0))[1] / args.steps
    achieved = alg / (filt_ms * 1e-3) / 1e9 if filt_ms > 0 else 0.0
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = reference_filters_sample(args, spec)
    pm4g.pm4g_log_free(log)
    pm4g.pm4g_ctx_destroy(ctx)
    if rank != 0:
        return
    line = {
        "metric": FILTERS_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "filters_mix", "log": spec.name, "n_events": N, "n_cases": int(summ_cases),
                   "n_activities": A, "filters": [name for name, _, _ in mix],
                   "kept_events": kept, "ms_per_filter": {k: round(1e3 * v / args.steps, 3) for k, v in per.items()},
                   "l2": "resident log larger than L2; no flush", "parallelism": f"replicas x{world}",
                   "generate_s": round(t_gen, 1)},
        "roofline": {"bound": "hbm", "kernel": "filter", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "alg_bytes_per_step": alg, "filter_kernels_ms_per_step": filt_ms},
        "kernels_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in sorted(kt.items(), key=lambda x: -x[1][1])},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        # each filter's result (the sub-log's performance DFG) is read on the host
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(d2h / args.steps)},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def reference_filters_sample(args, spec):
    """The oracle's six filters on a bounded sample of the same log law."""
    import oracle
    small = spec.scaled(max(2000, min(spec.n_cases, args.cpu_sample_cases // 4)))
    S = synth.generate(small)
    R = oracle.summarize(S.case_id, S.activity, S.ts_ns, S.n_activities)
    rows = R.sorted_rows
    off = np.r_[0, np.cumsum(R.case_len)]
    summ = {"count": R.count, "src": R.src, "dst": R.dst, "end": R.end, "freq": R.freq, "case_len": R.case_len,
            "duration": (S.ts_ns[rows[off[1:] - 1]].astype(np.uint64) - S.ts_ns[rows[off[:-1]]].astype(np.uint64)).astype(np.int64)}
    mix = filter_mix(summ, S)
    t = time.perf_counter()
    for _, kind, kw in mix:
        if kind == "paths":
            k = oracle.filter_paths(S.case_id, S.activity, S.ts_ns, S.n_activities, kw["pairs"])
        else:
            k = oracle.filter_cases(S.case_id, S.activity, S.ts_ns, S.n_activities, **kw)
        sub = S.take(k)
        oracle.summarize(sub.case_id, sub.activity, sub.ts_ns, S.n_activities)
    dt = time.perf_counter() - t
    return {"value": len(mix) * S.n_events / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the six filters (each followed by its sub-log's summary) on a {small.name} law log with "
                      f"{small.n_cases} cases ({S.n_events} events), one run, {dt:.1f} s on 1 of "
                      f"{os.cpu_count()} host cores"}


def run_reference_filters(args):
    rank, world, _ = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    spec = workload_spec(args)
    vals = []
    cpu = None
    for i in range(args.warmup + args.steps):
        cpu = reference_filters_sample(args, spec)
        if i >= args.warmup:
            vals.append(cpu["value"])
    value = statistics.median(vals)
    cpu["value"] = value
    line = {"impl": "reference", "metric": FILTERS_METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "filters_mix", "log": spec.name}, "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


EFG_METRIC = "eventually-follows pairs/s for the EFG + temporal profile (exact moments)"


def efg_sample(args, spec):
    """The oracle's eventually-follows graph on a bounded sample of the law."""
    import oracle
    small = spec.scaled(max(500, min(spec.n_cases, args.cpu_sample_cases // 50)))
    S = synth.generate(small)
    t = time.perf_counter()
    E = oracle.efg(S.case_id, S.activity, S.ts_ns, S.n_activities)
    dt = time.perf_counter() - t
    pairs = int(E.count.astype(np.int64).sum())
    return {"value": pairs / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"{small.name} law with {small.n_cases} cases ({S.n_events} events, {pairs} pairs), one run, "
                      f"{dt:.1f} s on 1 of {os.cpu_count()} host cores"}


def run_efg(args):
    rank, world, local = dist_info()
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
            if rank != 0:
                dist.barrier()
                return
        spec = workload_spec(args)
        vals = []
        cpu = None
        for i in range(args.warmup + args.steps):
            cpu = efg_sample(args, spec)
            if i >= args.warmup:
                vals.append(cpu["value"])
        cpu["value"] = statistics.median(vals)
        print(json.dumps({"impl": "reference", "metric": EFG_METRIC, "value": cpu["value"], "unit": "pairs/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
                          "data": "synthetic", "config": {"workload": "efg", "log": spec.name}, "cpu_baseline": cpu,
                          "e2e": {"value": cpu["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        return
    import torch
    from paper_2204_04898_b300 import pm4g
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    spec = workload_spec(args)
    t_gen = time.perf_counter()
    L = synth.generate(spec, pinned=True)
    t_gen = time.perf_counter() - t_gen
    N, A = L.n_events, L.n_activities
    dev = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns)]
    stream = torch.cuda.Stream()
    ctx = pm4g.pm4g_ctx_create(local, stream=stream.cuda_stream)
    log = pm4g.pm4g_load_log(ctx, *dev, n_activities=A)
    E = pm4g.pm4g_efg(log)  # also forms the timestamps in case order, once
    pairs = int(E.count.astype(np.int64).sum())
    n_cells = int(E.count.size)
    d2h = sum(x.nbytes for x in (E.src, E.dst, E.count, E.sum_lo, E.sum_hi, E.sq0, E.sq1, E.sq2, E.mean, E.stdev))
    for _ in range(args.warmup):
        pm4g.pm4g_efg(log)
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 1)
    pm4g.pm4g_ctx_timing_reset(ctx)
    launches0 = pm4g.pm4g_ctx_timing(ctx, "launches")[0]
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    def rewarm():
        pm4g.pm4g_efg(log)
        pm4g.pm4g_ctx_timing_reset(ctx)  # the timed steps alone are counted

    with ClockSampler(local, rewarm, steps=args.steps, warm_steps=1, pad=lambda: pm4g.pm4g_efg(log)) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            pm4g.pm4g_efg(log)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    n_k, efg_ms = pm4g.pm4g_ctx_timing(ctx, "efg")
    scan_ms = pm4g.pm4g_ctx_timing(ctx, "scan")[1]
    launches = pm4g.pm4g_ctx_timing(ctx, "launches")[0] - launches0
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 0)
    if dist is not None:
        t_ = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t_, op=dist.ReduceOp.MAX)
        ms = float(t_[0])
    cpu = efg_sample(args, spec) if rank == 0 and not args.no_cpu_baseline else None
    pm4g.pm4g_log_free(log)
    pm4g.pm4g_ctx_destroy(ctx)
    if rank != 0:
        return
    value = pairs * world * 1e3 / ms
    peak, peak_kind = peaks()
    # the method's bytes: the resident formatted log's activity and timestamp
    # (12 B/event), read once; every pair then lives in registers and is added
    # to an L2-resident A x A table by 64-bit atomics (implementation traffic,
    # reported beside it and never held against the HBM peak)
    alg = 12.0 * N
    atomic_bytes = 96.0 * pairs
    kern_ms = efg_ms / args.steps
    line = {
        "metric": EFG_METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": "efg", "log": spec.name, "n_events": N, "n_activities": A, "pairs": pairs,
                   "activity_pairs": n_cells, "events_per_s": N * world * 1e3 / ms,
                   "l2": "resident log larger than L2; the A x A table (48 B a cell) stays in L2",
                   "parallelism": f"replicas x{world}", "generate_s": round(t_gen, 1)},
        "roofline": {"bound": "hbm", "kernel": "efg", "achieved": alg / (kern_ms * 1e-3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": alg / (kern_ms * 1e-3) / 1e9 / peak, "traffic": None,
                     "peak_kind": peak_kind, "alg_bytes_per_step": alg, "efg_kernels_ms_per_step": kern_ms,
                     "l2_atomic_bytes_per_step": atomic_bytes,
                     "note": "algorithmic bytes: 12 B/event of the formatted log read once; the pair updates "
                             "(64-bit atomics, 96 B a pair, on an L2-resident table) are implementation "
                             "traffic and have no fraction"},
        "kernels_ms_per_step": {"efg": round(kern_ms, 4), "scan": round(scan_ms / args.steps, 4)},
        "gpu_launches": int(launches), "clocks": clk.summary(),
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(d2h)},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.mode == "efg":
        return run_efg(args)
    if args.mode == "filters":
        return run_filters(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "drilldown":
        return run_reference_drilldown(args) if args.impl == "reference" else run_drilldown(args)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2204_04898_b300 import pm4g

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    spec = workload_spec(args)
    t_gen = time.perf_counter()
    L = synth.generate(spec, pinned=True)
    t_gen = time.perf_counter() - t_gen
    N = L.n_events
    A = L.n_activities
    dev = [torch.from_numpy(x).cuda() for x in (L.case_id, L.activity, L.ts_ns)]
    stream = torch.cuda.Stream()
    ctx = pm4g.pm4g_ctx_create(local, stream=stream.cuda_stream)
    info = {}

    def step(cols, k=args.top_k):
        log = pm4g.pm4g_load_log(ctx, *cols, n_activities=A)
        try:
            d = pm4g.pm4g_dfg(log)
            p = pm4g.pm4g_perf_dfg(log)
            s, e, f = pm4g.pm4g_start_end(log, A)
            v = pm4g.pm4g_variants(log, top_k=k)
            info["C"] = pm4g.pm4g_log_info(log)[1]
            info["E"] = int(d["src"].shape[0])
            info["V"] = int(v.n_variants)
            info["d2h"] = (d["src"].nbytes + d["dst"].nbytes + d["count"].nbytes + 5 * 8 * p.n_edges
                           + 8 * 3 * A + v.count.nbytes + v.min_case.nbytes + 4 * v.off.nbytes // 2
                           + v.acts.nbytes)
        finally:
            pm4g.pm4g_log_free(log)

    # launch choices of the single-log pass (bucket width, partition units,
    # streaming-pass warps, streaming pass on/off, edge table) by the
    # autotuner, timed on this log before the timed region
    from paper_2204_04898_b300 import autotune
    t_tune = time.perf_counter()
    tuned = autotune.Tuner().tune_load(ctx, dev, A, top_k=args.top_k, reps=2,
                                       device=torch.cuda.get_device_name(local)) if not args.no_tune else None
    t_tune = time.perf_counter() - t_tune
    for _ in range(args.warmup):
        step(dev)
    # timed region: device-resident inputs (3 columns, larger than L2)
    torch.cuda.synchronize()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    def rewarm():
        for _ in range(3):
            step(dev)
        # inside the timed region, CUDA events around the dominant kernels only
        pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 2)
        pm4g.pm4g_ctx_timing_reset(ctx)  # the timed steps alone are counted

    with ClockSampler(local, rewarm, steps=args.steps, pad=lambda: step(dev)) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step(dev)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = max_over_ranks(ms)
    value = N * world * 1e3 / ms_max
    live = {name: pm4g.pm4g_ctx_timing(ctx, name) for name in ("segment", "segment_sort", "partition")}
    launches = pm4g.pm4g_ctx_timing(ctx, "launches")[0]

    # the breakdown of every kernel (CUDA events around each launch), same
    # number of steps after the timed region
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 1)
    pm4g.pm4g_ctx_timing_reset(ctx)
    for _ in range(args.steps):
        step(dev)
    kt = {}
    for name in pm4g.pm4g_kernel_names():
        n_l, t_ms = pm4g.pm4g_ctx_timing(ctx, name)
        if n_l:
            kt[name] = (n_l, t_ms)
    sorted_windows = pm4g.pm4g_ctx_timing(ctx, "sorted_windows")[0] // max(1, args.steps)
    regrouped = pm4g.pm4g_ctx_timing(ctx, "variant_regrouped")[0] // max(1, args.steps)
    pm4g.pm4g_ctx_set_option(ctx, pm4g.OPT_TIMING, 0)
    total_kt = sum(v[1] for v in kt.values()) or 1.0
    dom = max(kt, key=lambda k: kt[k][1])
    peak, peak_kind = peaks()
    C = info["C"]
    per_ev, per_case = ALG_BYTES.get(dom, (0.0, 0.0))
    alg = per_ev * N + per_case * C
    # the dominant kernel's launches timed live in the timed region
    n_dom, t_dom = live[dom] if dom in live and live[dom][0] else kt[dom]
    launch_ms = t_dom / n_dom
    # bytes per launch: the kernel runs once per step for the modelled kernels
    per_launch = alg * args.steps / n_dom
    achieved = per_launch / (launch_ms * 1e-3) / 1e9
    b_alg = 40.0 * N + 4.0 * C

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        host = [L.case_id, L.activity, L.ts_ns]
        step(host)
        torch.cuda.synchronize()
        barrier()
        t = time.perf_counter()
        for _ in range(args.steps):
            step(host)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t)
        e2e = {"value": N * world * args.steps / el, "unit": UNIT, "h2d_bytes_per_step": 16 * N,
               "d2h_bytes_per_step": int(info["d2h"])}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        sample_cases = max(1000, min(spec.n_cases, args.cpu_sample_cases))
        S = synth.generate(spec.scaled(sample_cases))
        t = time.perf_counter()
        oracle.summarize(S.case_id, S.activity, S.ts_ns, S.n_activities)
        dt = time.perf_counter() - t
        cpu = {"value": S.n_events / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{spec.name} law with {sample_cases} cases ({S.n_events} events), one run, "
                         f"{dt:.1f} s on 1 of {os.cpu_count()} host cores"}

    pm4g.pm4g_ctx_destroy(ctx)
    del dev, L
    torch.cuda.empty_cache()
    # The batched and served forms (drill-down views and the serving mix) on
    # one GPU, after the single-log pass: at N = 1 only (replicas add nothing)
    drill = serving = None
    if world == 1 and not args.no_drilldown:
        r = drilldown_core(args, local, max(1, args.dd_steps), max(3, args.warmup), args.plain_views, tune=True,
                           cpu_baseline=False)
        drill = {"metric": DD_METRIC, "workload": "drilldown_views", "log": r["spec"].name,
                 "n_events": r["n_events"], "n_activities": r["n_activities"], "n_views": r["n_views"],
                 "sub_log_events": r["sub_log_events"], "var_top_k": r["var_top_k"],
                 "batched": {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"],
                             "steps": r["steps"], "warmup": r["warmup"],
                             "timing": "CUDA events on the context stream around each pm4g_batch_dfg call",
                             "launches_per_step": r["launches_per_step"], "autotuned": r["tuned"]},
                 "plain": r["plain"], "ratio_vs_plain": r["ratio_vs_plain"],
                 "e2e": r["e2e"], "roofline": r["roofline"], "gpu_launches": r["gpu_launches"],
                 "first_call_ms_with_index": round(r["first_ms"], 1), "clocks": r["clocks"]}
        torch.cuda.empty_cache()
    if world == 1 and not args.no_serving:
        r = serve_core(args, local, [float(x) for x in args.serve_rates.split(",") if x], args.serve_seconds,
                       small_log=False)
        serving = {"metric": SERVE_METRIC, "workload": "serving_mix", "log": r["spec"].name,
                   "n_events": r["n_events"], "seconds_per_rate": r["seconds_per_rate"],
                   "mix": "70% filter+DFG (EVENTS), 20% variants top-10, 10% upload",
                   "upload_events": r["upload_events"],
                   "rates": [{"rate": e["rate"], "requests": e["requests"], "completed": e["completed"],
                              "errors": e["errors"], "events_per_s": e["events_per_s"],
                              "p50_ms": e["all"].get("p50_ms"), "p99_ms": e["all"].get("p99_ms"),
                              "dfg_p50_ms": e["dfg"].get("p50_ms"), "dfg_p99_ms": e["dfg"].get("p99_ms"),
                              "variants_p99_ms": e["variants"].get("p99_ms"),
                              "upload_p99_ms": e["upload"].get("p99_ms"), "dfg_batches": e["dfg_batches"]}
                             for e in r["per_rate"]],
                   "latency": "arrival to result on the host", "python_gc": "off while a rate runs",
                   "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
        torch.cuda.empty_cache()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": spec.name, "n_events": N, "n_cases": C, "n_activities": A, "n_edges": info["E"],
                   "n_variants": info["V"], "top_k": args.top_k,
                   "l2": "inputs (16 B/event, %.1f GB) larger than L2; no flush" % (16 * N / 1e9),
                   "parallelism": f"replicas x{world}", "generate_s": round(t_gen, 1),
                   "autotuned": tuned, "autotune_s": round(t_tune, 2)},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(dom, spec.name), "peak_kind": peak_kind,
                     "alg_bytes_per_launch": per_launch, "launch_ms": launch_ms,
                     "launch_timing": "CUDA events around the kernel's launches inside the timed region",
                     "path_alg_bytes": b_alg, "path_frac": b_alg / (ms_max * 1e-3) / 1e9 / peak},
        "kernels_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in sorted(kt.items(), key=lambda x: -x[1][1])},
        "kernel_share": {k: round(v[1] / total_kt, 4) for k, v in kt.items()},
        "gpu_launches": int(launches),
        "sorted_windows_per_step": int(sorted_windows),
        "variant_regrouped_per_step": int(regrouped),
        "clocks": clk.summary(),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "drilldown": drill if world == 1 else "measured at N = 1 only",
        "serving": serving if world == 1 else "measured at N = 1 only",
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
