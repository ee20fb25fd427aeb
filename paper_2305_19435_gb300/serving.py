"""Continuous-batching search server over resident AdANNS indices.

Requests (a batch of query rows plus a per-request compute budget: d_c, d_s,
nprobe, k, storage tier, shortlist size) arrive at any time.  A scheduler
thread keeps a FIFO of pending requests and, whenever a stream slot is free,
packs the oldest request together with later pending requests of the same
index and budget into one batch of at most `max_batch` query rows, admits it
only if its scratch estimate fits the device-memory budget next to the work
already in flight, and launches it on that slot's CUDA stream (host-to-device
copy, search, device-to-host copy of the results, completion event).  Work
of different slots overlaps on the device; requests that arrive while others
run join the next batch as soon as a slot and memory free up.  Completions
are detected by polling the events; each request's rows are returned to it
and its latency (arrival to results on the host) is recorded.

The execution backend is pluggable (`executor`): the default runs the
library's CUDA search; tests substitute a host-only fake to exercise the
scheduling logic without a GPU.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Budget:
    """Per-request compute budget (all fields as in search_ivf; method 1 is the
    IVF-OPQ search, whose d_s and storage are those of the index's OPQ data)."""
    d_c: int
    d_s: int
    nprobe: int
    k: int
    storage: int = 1
    rerank_k: int = 0
    method: int = 0


@dataclass
class Request:
    rid: int
    queries: object            # [n, d] float32 (host or device tensor / array)
    budget: Budget
    index_key: object
    t_arrive: float
    t_done: float = 0.0
    ids: object = None
    dist: object = None
    error: Exception | None = None
    _done: threading.Event = field(default_factory=threading.Event, repr=False)

    @property
    def n(self) -> int:
        return int(self.queries.shape[0])

    def wait(self, timeout: float | None = None) -> bool:
        return self._done.wait(timeout)

    @property
    def latency_ms(self) -> float:
        return 1000.0 * (self.t_done - self.t_arrive)


class GpuExecutor:
    """Runs a batch with the CUDA library on a slot's stream."""

    def __init__(self, indexes: dict, streams: int):
        import torch
        import paper_2305_19435_gb300 as P
        self.torch, self.P = torch, P
        self.indexes = indexes
        self.streams = [torch.cuda.Stream() for _ in range(streams)]

    def scratch_bytes(self, index_key, budget: Budget, n: int) -> int:
        idx = self.indexes[index_key]
        if budget.method == 1:   # IVF-OPQ: per-member scores of the probed lists dominate
            return n * (budget.nprobe * 64 + budget.k * 12 + idx.d * 4) + (64 << 20)
        return self.P.scratch_bytes(idx, n, budget.d_c, budget.d_s, budget.nprobe, budget.k,
                                    budget.storage, budget.rerank_k)

    def launch(self, slot: int, index_key, budget: Budget, reqs: list):
        torch = self.torch
        st = self.streams[slot]
        with torch.cuda.stream(st):
            parts = []
            for r in reqs:
                q = r.queries
                if not isinstance(q, torch.Tensor):
                    q = torch.from_numpy(np.ascontiguousarray(q))
                parts.append(q.cuda(non_blocking=True) if not q.is_cuda else q)
            q = parts[0] if len(parts) == 1 else torch.cat(parts)
            if budget.method == 1:
                ids, dist = self.P.search_ivfopq(self.indexes[index_key], q, budget.d_c,
                                                 budget.nprobe, budget.k, rerank_k=budget.rerank_k)
            else:
                ids, dist = self.P.search_ivf(self.indexes[index_key], q, budget.d_c, budget.d_s,
                                              budget.nprobe, budget.k, storage=budget.storage,
                                              rerank_k=budget.rerank_k)
            ids_h = torch.empty(ids.shape, dtype=ids.dtype, pin_memory=True)
            dist_h = torch.empty(dist.shape, dtype=dist.dtype, pin_memory=True)
            ids_h.copy_(ids, non_blocking=True)
            dist_h.copy_(dist, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"event": ev, "ids": ids_h, "dist": dist_h, "keep": (q, ids, dist)}

    def ready(self, handle) -> bool:
        return handle["event"].query()

    def results(self, handle):
        return handle["ids"].numpy(), handle["dist"].numpy()


class Server:
    def __init__(self, indexes: dict, streams: int = 2, max_batch: int = 8192,
                 mem_budget: int = 16 << 30, executor=None, idle_sleep: float = 5e-5):
        self.executor = executor if executor is not None else GpuExecutor(indexes, streams)
        self.nslots = streams
        self.max_batch = max_batch
        self.mem_budget = mem_budget
        self.idle_sleep = idle_sleep
        self._pending: collections.deque[Request] = collections.deque()
        self._lock = threading.Lock()
        self._wake = threading.Event()
        self._slots = [None] * streams           # (handle, reqs, bytes) per busy slot
        self._inflight_bytes = 0
        self._next_id = 0
        self._running = False
        self._thread = None
        self.completed: list[Request] = []
        self.batches: list[tuple[int, int]] = []  # (requests, rows) of each launched batch
        self.max_inflight_bytes = 0

    # ------------------------------------------------------------ client side
    def submit(self, queries, budget: Budget, index_key=None) -> Request:
        with self._lock:
            r = Request(self._next_id, queries, budget, index_key, time.perf_counter())
            self._next_id += 1
            self._pending.append(r)
        self._wake.set()
        return r

    def start(self):
        self._running = True
        self._thread = threading.Thread(target=self._loop, daemon=True)
        self._thread.start()
        return self

    def stop(self, drain: bool = True, timeout: float = 60.0):
        if drain:
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < timeout:
                with self._lock:
                    busy = bool(self._pending) or any(s is not None for s in self._slots)
                if not busy:
                    break
                time.sleep(1e-3)
        self._running = False
        self._wake.set()
        if self._thread is not None:
            self._thread.join(timeout)

    def stats(self) -> dict:
        lat = np.array([r.latency_ms for r in self.completed if r.error is None])
        rows = sum(r.n for r in self.completed if r.error is None)
        if len(lat) == 0:
            return {"requests": 0}
        t0 = min(r.t_arrive for r in self.completed)
        t1 = max(r.t_done for r in self.completed)
        return {"requests": len(lat), "queries": rows,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "qps": rows / max(t1 - t0, 1e-9),
                "batches": len(self.batches),
                "mean_requests_per_batch": float(np.mean([b[0] for b in self.batches])),
                "max_inflight_bytes": self.max_inflight_bytes}

    # ------------------------------------------------------------ scheduler
    def _finish(self, slot: int):
        handle, reqs, nbytes = self._slots[slot]
        now = time.perf_counter()
        try:
            ids, dist = self.executor.results(handle)
            off = 0
            for r in reqs:
                r.ids, r.dist = ids[off:off + r.n], dist[off:off + r.n]
                off += r.n
        except Exception as e:  # the batch failed: every request in it reports it
            for r in reqs:
                r.error = e
        for r in reqs:
            r.t_done = now
            r._done.set()
        self.completed.extend(reqs)
        self._slots[slot] = None
        self._inflight_bytes -= nbytes

    def _take_batch(self):
        """Oldest pending request plus later ones with the same key, within
        max_batch rows; returns (reqs, key) or None."""
        with self._lock:
            if not self._pending:
                return None
            head = self._pending[0]
            key = (head.index_key, head.budget)
            reqs, rows = [], 0
            keep = collections.deque()
            while self._pending:
                r = self._pending.popleft()
                if (r.index_key, r.budget) == key and (not reqs or rows + r.n <= self.max_batch):
                    reqs.append(r)
                    rows += r.n
                else:
                    keep.append(r)
            self._pending = keep if not self._pending else keep + self._pending
            return reqs, key

    def _requeue_front(self, reqs):
        with self._lock:
            for r in reversed(reqs):
                self._pending.appendleft(r)

    def _loop(self):
        while self._running:
            progressed = False
            for s in range(self.nslots):
                if self._slots[s] is not None and self.executor.ready(self._slots[s][0]):
                    self._finish(s)
                    progressed = True
            free = [s for s in range(self.nslots) if self._slots[s] is None]
            if free:
                got = self._take_batch()
                if got is not None:
                    reqs, (ikey, budget) = got
                    rows = sum(r.n for r in reqs)
                    nbytes = self.executor.scratch_bytes(ikey, budget, rows)
                    busy = any(x is not None for x in self._slots)
                    if busy and self._inflight_bytes + nbytes > self.mem_budget:
                        # wait for memory: keep arrival order
                        self._requeue_front(reqs)
                    else:
                        slot = free[0]
                        try:
                            h = self.executor.launch(slot, ikey, budget, reqs)
                            self._slots[slot] = (h, reqs, nbytes)
                            self._inflight_bytes += nbytes
                            self.max_inflight_bytes = max(self.max_inflight_bytes,
                                                          self._inflight_bytes)
                            self.batches.append((len(reqs), rows))
                        except Exception as e:
                            for r in reqs:
                                r.error = e
                                r.t_done = time.perf_counter()
                                r._done.set()
                            self.completed.extend(reqs)
                        progressed = True
            if not progressed:
                self._wake.wait(self.idle_sleep)
                self._wake.clear()


def poisson_stream(rate_qps: float, duration_s: float, seed: int, max_rows: int = 4096,
                   budgets=None):
    """Seeded open-loop arrivals: (time offset, rows, budget index) with
    request sizes uniform in [1, max_rows] and exponential gaps chosen so the
    mean query rate is rate_qps."""
    rng = np.random.default_rng(seed)
    mean_rows = (1 + max_rows) / 2.0
    lam = rate_qps / mean_rows
    t, out = 0.0, []
    nb = 1 if budgets is None else len(budgets)
    while True:
        t += rng.exponential(1.0 / lam)
        if t > duration_s:
            return out
        out.append((t, int(rng.integers(1, max_rows + 1)), int(rng.integers(0, nb))))


# ---------------------------------------------------------------- native server
class NativeRequest:
    """A request of the library's server; results are collected on wait()."""

    def __init__(self, server, ticket: int, n: int, k: int):
        self._srv, self.ticket, self._n, self._k = server, ticket, n, k
        self.ids = self.dist = None
        self.error: Exception | None = None
        self.latency_ms = None
        self._lock = threading.Lock()
        self._done = False

    @property
    def n(self) -> int:
        return self._n

    def wait(self, timeout: float | None = None) -> bool:
        """Block until the results are on the host (True) or timeout seconds pass."""
        import ctypes
        with self._lock:
            if self._done:
                return True
            P = self._srv.P
            ids = np.empty((self._n, self._k), dtype=np.int64)
            dist = np.empty((self._n, self._k), dtype=np.float32)
            lat = ctypes.c_double()
            ms = -1 if timeout is None else max(0, int(timeout * 1000))
            rc = P.lib().adanns_server_poll(self._srv.handle, self.ticket, ms,
                                            ids.ctypes.data_as(ctypes.c_void_p),
                                            dist.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.byref(lat))
            if rc == P.PENDING:
                return False
            if rc != 0:
                self.error = P.AdannsError(rc, P.lib().adanns_last_error().decode())
            else:
                self.ids, self.dist, self.latency_ms = ids, dist, lat.value
            self._done = True
            return True


class NativeServer:
    """Continuous batching done by the library (adanns_server_*): the same
    scheduling as Server (arrival order, memory admission, one batch per CUDA
    stream in flight) in a native worker thread, and it also packs requests
    whose budgets differ but can share one pass (adanns_search_ivf_budgets:
    FP32 requests of one index and d_c; low-precision ones of one d_c, d_s and
    shortlist) up to max_batch rows.  Queries are host arrays or CPU tensors."""

    def __init__(self, indexes: dict, streams: int = 2, max_batch: int = 8192,
                 mem_budget: int = 16 << 30):
        import ctypes
        import paper_2305_19435_gb300 as P
        self.P = P
        self._keys = list(indexes)
        self._d = {key: indexes[key].d for key in self._keys}
        arr = (ctypes.c_void_p * len(self._keys))(*[indexes[key].handle.value for key in self._keys])
        self._arr = arr
        h = ctypes.c_void_p()
        P._check(P.lib().adanns_server_create(arr, len(self._keys), streams, max_batch, mem_budget,
                                              ctypes.byref(h)))
        self.handle = h
        self.requests: list[NativeRequest] = []

    def start(self):
        return self

    def submit(self, queries, budget: Budget, index_key=None) -> NativeRequest:
        import ctypes
        P = self.P
        if index_key is None:
            index_key = self._keys[0]
        q = queries.numpy() if hasattr(queries, "numpy") else queries
        q = np.ascontiguousarray(q, dtype=np.float32)
        b = P.BudgetC(budget.method, budget.d_c, budget.d_s, budget.nprobe, budget.k,
                      budget.storage, budget.rerank_k)
        t = ctypes.c_int64()
        P._check(P.lib().adanns_server_submit(self.handle, self._keys.index(index_key),
                                              q.ctypes.data_as(ctypes.c_void_p), q.shape[0],
                                              ctypes.byref(b), ctypes.byref(t)))
        r = NativeRequest(self, t.value, q.shape[0], budget.k)
        self.requests.append(r)
        return r

    def stop(self, drain: bool = True, timeout: float = 600.0):
        for r in self.requests:
            r.wait(timeout if drain else 0)
        self._stats = self.stats()
        self.P.lib().adanns_server_destroy(self.handle)
        self.handle = None

    def stats(self) -> dict:
        import ctypes
        if self.handle is None:
            return self._stats
        p50, p99, qps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        req, bat, rows, mx = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self.P._check(self.P.lib().adanns_server_stats(self.handle, ctypes.byref(p50),
                                                       ctypes.byref(p99), ctypes.byref(req),
                                                       ctypes.byref(bat), ctypes.byref(rows),
                                                       ctypes.byref(qps), ctypes.byref(mx)))
        return {"requests": req.value, "queries": rows.value, "p50_ms": p50.value,
                "p99_ms": p99.value, "qps": qps.value, "batches": bat.value,
                "mean_requests_per_batch": req.value / max(bat.value, 1),
                "max_inflight_bytes": mx.value, "scheduler": "native (adanns_server)"}
