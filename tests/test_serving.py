"""Scheduling logic of the continuous-batching server, on the host with a fake
executor (no GPU): routing of rows back to requests, batching only requests
with the same index and budget, FIFO order, the max-batch cap and admission
by the device-memory budget."""
import threading
import time

import numpy as np

from paper_2305_19435_gb300.serving import Budget, Server, poisson_stream


class FakeExecutor:
    """Result row i of a batch = (sum of query row i, 2 * sum): checkable."""

    def __init__(self, delay=0.004, bytes_per_row=1000):
        self.delay = delay
        self.bytes_per_row = bytes_per_row
        self.launched = []
        self.lock = threading.Lock()
        self.concurrent = 0
        self.max_concurrent = 0

    def scratch_bytes(self, key, budget, n):
        return n * self.bytes_per_row

    def launch(self, slot, key, budget, reqs):
        q = np.concatenate([r.queries for r in reqs])
        with self.lock:
            self.launched.append((slot, key, budget, [r.rid for r in reqs]))
            self.concurrent += 1
            self.max_concurrent = max(self.max_concurrent, self.concurrent)
        return {"t": time.perf_counter(), "q": q}

    def ready(self, h):
        ok = time.perf_counter() - h["t"] >= self.delay
        if ok and not h.get("counted"):
            h["counted"] = True
            with self.lock:
                self.concurrent -= 1
        return ok

    def results(self, h):
        s = h["q"].sum(1, keepdims=True)
        return s.astype(np.int64), (2 * s).astype(np.float32)


def make_q(rng, n):
    return rng.integers(0, 100, size=(n, 4)).astype(np.float32)


def test_rows_return_to_their_requests_and_batches_share_keys():
    rng = np.random.default_rng(0)
    ex = FakeExecutor()
    srv = Server({}, streams=3, max_batch=64, mem_budget=1 << 40, executor=ex).start()
    b1, b2 = Budget(16, 64, 4, 10), Budget(16, 128, 4, 10, 2, 40)
    reqs = []
    for i in range(60):
        reqs.append(srv.submit(make_q(rng, int(rng.integers(1, 20))), b1 if i % 3 else b2,
                               index_key=i % 2))
        if i % 7 == 0:
            time.sleep(0.002)
    for r in reqs:
        assert r.wait(10)
    srv.stop()
    for r in reqs:
        assert r.error is None
        want = r.queries.sum(1, keepdims=True)
        assert np.array_equal(r.ids, want.astype(np.int64))
        assert np.array_equal(r.dist, (2 * want).astype(np.float32))
    byid = {r.rid: r for r in reqs}
    for slot, key, budget, rids in ex.launched:
        assert all(byid[i].index_key == key and byid[i].budget == budget for i in rids)
        assert sum(byid[i].n for i in rids) <= 64 or len(rids) == 1
        assert rids == sorted(rids)                      # FIFO inside a batch
    assert ex.max_concurrent > 1                         # batches overlapped
    st = srv.stats()
    assert st["requests"] == 60 and st["p99_ms"] >= st["p50_ms"] > 0
    assert st["mean_requests_per_batch"] > 1             # continuous batching merged requests


def test_admission_respects_memory_budget():
    rng = np.random.default_rng(1)
    ex = FakeExecutor(delay=0.01, bytes_per_row=100)
    srv = Server({}, streams=4, max_batch=10, mem_budget=1500, executor=ex).start()
    b = Budget(16, 64, 4, 10)
    reqs = [srv.submit(make_q(rng, 10), b) for _ in range(12)]
    for r in reqs:
        assert r.wait(10)
    srv.stop()
    # each batch is 10 rows = 1000 bytes; a second one would exceed 1500
    assert srv.max_inflight_bytes <= 1500
    assert ex.max_concurrent == 1


def test_oversized_request_runs_alone():
    rng = np.random.default_rng(2)
    ex = FakeExecutor()
    srv = Server({}, streams=2, max_batch=8, mem_budget=1 << 40, executor=ex).start()
    b = Budget(16, 64, 4, 10)
    big = srv.submit(make_q(rng, 50), b)
    small = srv.submit(make_q(rng, 3), b)
    assert big.wait(10) and small.wait(10)
    srv.stop()
    assert big.ids.shape == (50, 1) and small.ids.shape == (3, 1)


def test_poisson_stream_rate_and_sizes():
    arr = poisson_stream(20000.0, 200.0, seed=3, max_rows=4096)
    rows = np.array([a[1] for a in arr])
    assert rows.min() >= 1 and rows.max() <= 4096
    rate = rows.sum() / 200.0
    assert 0.8 * 20000 < rate < 1.2 * 20000
    gaps = np.diff([0.0] + [a[0] for a in arr])
    assert np.all(gaps > 0)
