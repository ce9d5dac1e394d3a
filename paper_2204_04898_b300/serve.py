"""Serving over a device-resident log with continuous batching (host runtime).

A Server keeps one formatted log resident on the GPU and answers three kinds of
requests (Section 1: interactive drill-down is the use the library is built
for):

* ``dfg``      - filter(attribute set, window, mode) + frequency/performance DFG
                 and start/end/frequency counts of the filtered view;
* ``variants`` - the resident log's top-k variants;
* ``upload``   - a new log is loaded, summarised (DFG, start/end, top-k
                 variants) and released.

Continuous batching: requests arriving while the GPU works are queued; when the
query worker becomes free it takes every pending ``dfg`` request (up to
``max_batch``) and answers them with one pm4g_batch_dfg launch, then every
pending ``variants`` request with one call per distinct k. Uploads run on their
own contexts (own CUDA streams) in ``upload_slots`` workers, so they overlap
with query batches on the device. Admission is by free HBM: the server starts
with a byte budget (the device's free memory when it starts, less the query
side's share), every admitted upload reserves its estimate until it is done,
and an upload waits until the budget minus the reservations covers it (one
that could never fit is refused at once). Stream-ordered pools reuse freed
blocks, so reservations track what the uploads actually hold.

Every result is a plain host object computed by the engine's kernels; a
request's result does not depend on what it was batched with (the batch gives
each view exactly what it gives alone).

The engine is the C ABI through the binding (GpuEngine); the scheduler only
needs the four methods of that class, so its logic is testable with a fake.
"""

from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    kind: str                                  # "dfg" | "variants" | "upload"
    attr_set: np.ndarray | None = None         # dfg: attribute values (None/empty: all cases)
    t_lo: int = -(2 ** 63)
    t_hi: int = 2 ** 63 - 1
    mode: int = 1                              # PM4G_TW_* of the window
    top_k: int = 10                            # variants / upload
    columns: tuple | None = None               # upload: (case_id, activity, ts_ns) host arrays
    n_activities: int = 0                      # upload
    t_arrival: float = 0.0
    t_done: float = 0.0
    result: object = None
    error: BaseException | None = None
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class GpuEngine:
    """The engine behind the server: one context for the resident log and its
    query batches, one context per upload slot."""

    def __init__(self, pm4g, device: int, log: int, query_ctx: int, upload_slots: int):
        self.pm4g = pm4g
        self.log = log
        self.ctx = query_ctx
        self.upload_ctx = [pm4g.pm4g_ctx_create(device) for _ in range(upload_slots)]
        self.buf = pm4g.BatchBuffers(0, 0, 0)
        import torch
        self._torch = torch
        self.device = device

    def close(self):
        for c in self.upload_ctx:
            self.pm4g.pm4g_ctx_destroy(c)
        self.upload_ctx = []

    def free_bytes(self) -> int:
        return int(self._torch.cuda.mem_get_info(self.device)[0])

    @staticmethod
    def upload_bytes(n_events: int, n_activities: int) -> int:
        # input columns, two record buffers, activity sequence and per-case
        # arrays, and the global edge table: dense (40 B a pair) up to 4096
        # activities, else hashed (48 B a slot, twice the possible pairs)
        n, A = int(n_events), int(n_activities)
        if A <= 4096:
            table = A * A * 40
        else:
            slots = 4096
            while slots < 2 * max(1, min(A * A, n)):
                slots <<= 1
            table = slots * 48
        return n * 80 + table + (64 << 20)

    def batch_dfg(self, reqs: list[Request]) -> list[dict]:
        pm4g = self.pm4g
        B = pm4g.pm4g_batch_dfg(self.log, [r.attr_set for r in reqs], [r.t_lo for r in reqs],
                                [r.t_hi for r in reqs], [r.mode for r in reqs], out=self.buf)
        out = []
        for i in range(len(reqs)):
            d = {k: v.copy() for k, v in B.sub(i).items()}
            d.update(n_events=int(B.n_events[i]), n_cases=int(B.n_cases[i]), start=B.start[i].copy(),
                     end=B.end[i].copy(), freq=B.freq[i].copy())
            out.append(d)
        return out

    def variants(self, top_k: int):
        v = self.pm4g.pm4g_variants(self.log, top_k=top_k)
        return {"n_variants": v.n_variants, "count": v.count, "min_case": v.min_case, "off": v.off, "acts": v.acts}

    def upload(self, req: Request, slot: int) -> dict:
        pm4g = self.pm4g
        ctx = self.upload_ctx[slot]
        log = pm4g.pm4g_load_log(ctx, *req.columns, n_activities=req.n_activities)
        try:
            p = pm4g.pm4g_perf_dfg(log)
            st, en, fr = pm4g.pm4g_start_end(log, req.n_activities)
            v = pm4g.pm4g_variants(log, top_k=req.top_k)
            n, c = pm4g.pm4g_log_info(log)
            return {"n_events": n, "n_cases": c, "src": p.src, "dst": p.dst, "count": p.count, "sum_lo": p.sum_lo,
                    "sum_hi": p.sum_hi, "min": p.min, "max": p.max, "mean": p.mean, "start": st, "end": en,
                    "freq": fr, "n_variants": v.n_variants, "var_count": v.count, "var_min_case": v.min_case,
                    "var_off": v.off, "var_acts": v.acts}
        finally:
            pm4g.pm4g_log_free(log)


class Server:
    """Continuous-batching request loop over an engine (see the module text)."""

    def __init__(self, engine, max_batch: int = 4096, upload_slots: int = 2, admit_timeout: float = 60.0,
                 mem_budget: int | None = None, query_share: int = 8 << 30):
        self.engine = engine
        self.max_batch = max_batch
        self.admit_timeout = admit_timeout
        if mem_budget is None:
            mem_budget = int(engine.free_bytes() * 0.9) - query_share
        self.mem_budget = max(0, int(mem_budget))
        self._lock = threading.Condition()
        self._dfg: collections.deque[Request] = collections.deque()
        self._var: collections.deque[Request] = collections.deque()
        self._up: collections.deque[Request] = collections.deque()
        self._mem = threading.Condition()
        self._reserved = 0
        self._stop = False
        self.batches: list[int] = []   # size of every dfg batch, for reporting
        self._threads = [threading.Thread(target=self._query_loop, daemon=True)]
        self._threads += [threading.Thread(target=self._upload_loop, args=(s,), daemon=True)
                          for s in range(upload_slots)]
        for t in self._threads:
            t.start()

    # ---- client side ----
    def submit(self, req: Request) -> Request:
        if not req.t_arrival:
            req.t_arrival = time.perf_counter()
        with self._lock:
            {"dfg": self._dfg, "variants": self._var, "upload": self._up}[req.kind].append(req)
            self._lock.notify_all()
        return req

    def close(self, timeout: float = 60.0) -> None:
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        with self._mem:
            self._mem.notify_all()
        for t in self._threads:
            t.join(timeout)

    # ---- workers ----
    @staticmethod
    def _finish(req: Request, result=None, error: BaseException | None = None) -> None:
        req.result, req.error = result, error
        req.t_done = time.perf_counter()
        req.done.set()

    def _query_loop(self) -> None:
        while True:
            with self._lock:
                while not self._dfg and not self._var and not self._stop:
                    self._lock.wait()
                if self._stop and not self._dfg and not self._var:
                    return
                take = min(len(self._dfg), self.max_batch)
                dfg = [self._dfg.popleft() for _ in range(take)]
                var = list(self._var)
                self._var.clear()
            if dfg:
                self.batches.append(len(dfg))
                try:
                    res = self.engine.batch_dfg(dfg)
                    for r, x in zip(dfg, res):
                        self._finish(r, x)
                except BaseException as e:  # every request of the batch reports the failure
                    for r in dfg:
                        self._finish(r, error=e)
            by_k: dict[int, list[Request]] = {}
            for r in var:
                by_k.setdefault(int(r.top_k), []).append(r)
            for k, rs in by_k.items():
                try:
                    x = self.engine.variants(k)
                    for r in rs:
                        self._finish(r, x)
                except BaseException as e:
                    for r in rs:
                        self._finish(r, error=e)

    def set_mem_budget(self, nbytes: int) -> None:
        """Replace the upload budget while serving (for example when another
        tenant of the device grows or shrinks). The budget is not sampled
        again by itself: the engine's contexts keep freed blocks for reuse, so
        the device's free memory under-counts what the server can still use.
        Uploads waiting for memory are judged again against the new budget;
        those that can no longer fit at all are refused."""
        with self._mem:
            self.mem_budget = max(0, int(nbytes))
            self._mem.notify_all()

    def _admit(self, need: int) -> bool:
        """Reserve `need` bytes of the budget for an upload, waiting while
        admitted uploads hold what it needs; False if it can never fit (or
        the wait times out)."""
        deadline = time.perf_counter() + self.admit_timeout
        with self._mem:
            while self._reserved + need > self.mem_budget:
                if need > self.mem_budget or self._stop or time.perf_counter() > deadline:
                    return False
                self._mem.wait(0.05)
            self._reserved += need
            return True

    def _release(self, need: int) -> None:
        with self._mem:
            self._reserved -= need
            self._mem.notify_all()

    def _upload_loop(self, slot: int) -> None:
        while True:
            with self._lock:
                while not self._up and not self._stop:
                    self._lock.wait()
                if not self._up:
                    return
                req = self._up.popleft()
            n = int(req.columns[0].shape[0]) if req.columns else 0
            need = self.engine.upload_bytes(n, req.n_activities)
            if not self._admit(need):
                self._finish(req, error=MemoryError(f"upload of {n} events not admitted: "
                                                    f"{need} bytes of device memory never became free"))
                continue
            try:
                self._finish(req, self.engine.upload(req, slot))
            except BaseException as e:
                self._finish(req, error=e)
            finally:
                self._release(need)


def latency_summary(reqs: list[Request]) -> dict:
    lat = np.array([r.latency for r in reqs if r.done.is_set() and r.error is None]) * 1e3
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max())}
