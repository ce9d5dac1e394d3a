"""The serving loop's scheduling on CPU, with a fake engine: continuous batching
of pending filter+DFG requests, variants answered per distinct k, uploads
overlapping on their own slots, admission by a byte budget (never above it,
refusal of what can never fit), and failure reporting."""

import threading
import time

import numpy as np
import pytest

from paper_2204_04898_b300.serve import Request, Server, latency_summary


class FakeEngine:
    def __init__(self, batch_s=0.02, upload_s=0.05, free=1000):
        self.batch_s, self.upload_s, self.free = batch_s, upload_s, free
        self.batch_sizes = []
        self.active_uploads = 0
        self.max_active = 0
        self.active_bytes = 0
        self.max_bytes = 0
        self.lock = threading.Lock()
        self.fail_batch = False

    def free_bytes(self):
        return self.free

    @staticmethod
    def upload_bytes(n_events, n_activities):
        return n_events

    def batch_dfg(self, reqs):
        self.batch_sizes.append(len(reqs))
        time.sleep(self.batch_s)
        if self.fail_batch:
            raise RuntimeError("device failure")
        return [{"key": (tuple(r.attr_set.tolist()), r.t_lo, r.t_hi)} for r in reqs]

    def variants(self, k):
        return {"k": k}

    def upload(self, req, slot):
        n = req.columns[0].shape[0]
        with self.lock:
            self.active_uploads += 1
            self.active_bytes += n
            self.max_active = max(self.max_active, self.active_uploads)
            self.max_bytes = max(self.max_bytes, self.active_bytes)
        time.sleep(self.upload_s)
        with self.lock:
            self.active_uploads -= 1
            self.active_bytes -= n
        return {"n": n, "slot": slot}


def _dfg(i):
    return Request("dfg", attr_set=np.array([i], np.int32), t_lo=i, t_hi=i + 10)


def _upload(n):
    return Request("upload", columns=(np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int64)),
                   n_activities=1)


def test_pending_requests_are_batched():
    eng = FakeEngine(batch_s=0.03)
    srv = Server(eng, mem_budget=10_000)
    try:
        reqs = [srv.submit(_dfg(i)) for i in range(200)]
        for r in reqs:
            assert r.done.wait(10)
        # each request got its own answer, whatever batch it rode in
        for i, r in enumerate(reqs):
            assert r.error is None and r.result["key"] == ((i,), i, i + 10)
        assert sum(eng.batch_sizes) == 200
        assert max(eng.batch_sizes) > 1, "requests pending during a batch must form the next batch"
        assert len(eng.batch_sizes) < 200
    finally:
        srv.close()


def test_batch_size_is_capped():
    eng = FakeEngine(batch_s=0.05)
    srv = Server(eng, max_batch=16, mem_budget=10_000)
    try:
        reqs = [srv.submit(_dfg(i)) for i in range(100)]
        for r in reqs:
            assert r.done.wait(10)
        assert max(eng.batch_sizes) <= 16
    finally:
        srv.close()


def test_variants_grouped_by_k():
    eng = FakeEngine()
    srv = Server(eng, mem_budget=10_000)
    try:
        reqs = [srv.submit(Request("variants", top_k=k)) for k in (10, 10, 3, 10, 3)]
        for r in reqs:
            assert r.done.wait(10)
        assert [r.result["k"] for r in reqs] == [10, 10, 3, 10, 3]
    finally:
        srv.close()


def test_uploads_overlap_within_the_budget():
    eng = FakeEngine(upload_s=0.1)
    srv = Server(eng, upload_slots=3, mem_budget=1000)
    try:
        reqs = [srv.submit(_upload(300)) for _ in range(9)]
        for r in reqs:
            assert r.done.wait(20)
            assert r.error is None
        assert eng.max_active == 3           # three slots, 900 bytes fit
        assert eng.max_bytes <= 1000
    finally:
        srv.close()


def test_admission_waits_for_memory():
    eng = FakeEngine(upload_s=0.1)
    srv = Server(eng, upload_slots=3, mem_budget=1000)
    try:
        reqs = [srv.submit(_upload(600)) for _ in range(4)]
        for r in reqs:
            assert r.done.wait(20)
            assert r.error is None
        assert eng.max_active == 1           # two of 600 never fit together
        assert eng.max_bytes <= 1000
    finally:
        srv.close()


def test_upload_that_never_fits_is_refused():
    eng = FakeEngine()
    srv = Server(eng, mem_budget=1000)
    try:
        big, ok = srv.submit(_upload(5000)), srv.submit(_upload(10))
        assert big.done.wait(10) and ok.done.wait(10)
        assert isinstance(big.error, MemoryError)
        assert ok.error is None and ok.result["n"] == 10
    finally:
        srv.close()


def test_budget_set_while_serving():
    """A waiting upload is admitted as soon as a larger budget covers it, and
    refused once a smaller one can never hold it; uploads never exceed the
    budget in force when they were admitted."""
    eng = FakeEngine(upload_s=0.3)
    srv = Server(eng, upload_slots=2, mem_budget=1000)
    try:
        first = srv.submit(_upload(800))
        time.sleep(0.05)
        second = srv.submit(_upload(700))      # waits: 800 + 700 > 1000
        time.sleep(0.05)
        assert not second.done.is_set()
        srv.set_mem_budget(1500)               # now both fit
        assert second.done.wait(5) and second.error is None
        assert first.done.wait(5) and first.error is None
        assert eng.max_active == 2 and eng.max_bytes == 1500
        third = srv.submit(_upload(900))
        time.sleep(0.05)
        fourth = srv.submit(_upload(900))      # waits behind the third
        time.sleep(0.05)
        srv.set_mem_budget(500)                # neither can ever fit now
        assert third.done.wait(5) and fourth.done.wait(5)
        assert third.error is None             # admitted before the change
        assert isinstance(fourth.error, MemoryError)
        ok = srv.submit(_upload(400))
        assert ok.done.wait(5) and ok.error is None
    finally:
        srv.close()


def test_engine_failure_reaches_every_request_of_the_batch():
    eng = FakeEngine(batch_s=0.01)
    eng.fail_batch = True
    srv = Server(eng, mem_budget=1000)
    try:
        reqs = [srv.submit(_dfg(i)) for i in range(5)]
        for r in reqs:
            assert r.done.wait(10)
            assert isinstance(r.error, RuntimeError)
        eng.fail_batch = False
        r = srv.submit(_dfg(7))
        assert r.done.wait(10) and r.error is None   # the server keeps serving
    finally:
        srv.close()


def test_latency_summary():
    reqs = []
    for i, lat in enumerate([1, 2, 3, 4, 100]):
        r = Request("dfg")
        r.t_arrival, r.t_done = 10.0, 10.0 + lat / 1e3
        r.done.set()
        reqs.append(r)
    s = latency_summary(reqs)
    assert s["n"] == 5 and s["p50_ms"] == pytest.approx(3.0) and s["max_ms"] == pytest.approx(100.0)
