"""The continuous-batching server on the GPU: requests with different budgets
arrive while others run, are batched and overlapped, and every request's
result equals the same request searched alone (identical ids; distances
within the FP32 tolerance, in practice bit-identical since each query's
arithmetic does not depend on its batch)."""
import time

import numpy as np
import pytest

import oracle
import synthdata
from parity import tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2305_19435_gb300 as P
    P.build()
    data = synthdata.small(40_000, 3000, 256, 64, 601)
    idx = {}
    for d_c in (16, 64):
        o = oracle.build_ivf(data["db"], d_c, 48, 6, 20_000, seed=31)
        idx[d_c] = P.index_create(torch.from_numpy(data["db"]).cuda(),
                                  torch.from_numpy(o["centroids"]).cuda(),
                                  torch.from_numpy(o["assign"].astype(np.int32)).cuda(),
                                  storage=3)
    yield P, data, idx
    for g in idx.values():
        g.free()


def test_results_same_alone_and_in_the_mix(setup):
    P, data, idx = setup
    from paper_2305_19435_gb300.serving import Budget, Server
    budgets = [Budget(16, 128, 4, 10), Budget(64, 256, 8, 100, P.STORE_BF16, 400),
               Budget(16, 64, 1, 10, P.STORE_BF16, 40), Budget(64, 192, 16, 10)]
    rng = np.random.default_rng(7)
    srv = Server(idx, streams=3, max_batch=1024, mem_budget=8 << 30)
    reqs, q = [], data["queries"]
    # a burst queued before the scheduler starts: it must be served as shared batches
    for i in range(8):
        b = budgets[i % 2]
        reqs.append(srv.submit(q[100 * i:100 * i + 37], b, index_key=b.d_c))
    srv.start()
    for i in range(32):
        n = int(rng.integers(1, 200))
        lo = int(rng.integers(0, len(q) - n))
        b = budgets[int(rng.integers(0, len(budgets)))]
        reqs.append(srv.submit(q[lo:lo + n], b, index_key=b.d_c))
        time.sleep(float(rng.exponential(0.002)))
    for r in reqs:
        assert r.wait(60)
    srv.stop()
    st = srv.stats()
    assert st["requests"] == 40 and st["batches"] < 40          # some requests shared a batch
    for r in reqs:
        assert r.error is None, r.error
        b = r.budget
        ids, dist = P.search_ivf(idx[b.d_c], torch.from_numpy(np.ascontiguousarray(r.queries)).cuda(),
                                 b.d_c, b.d_s, b.nprobe, b.k, storage=b.storage,
                                 rerank_k=b.rerank_k)
        ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
        assert np.array_equal(r.ids, ids), r.rid
        fin = np.isfinite(dist)
        assert np.all(np.abs(r.dist[fin] - dist[fin]) <= tol(dist[fin]))
    for g in idx.values():
        g.status()


def test_native_server_same_alone_and_in_the_mix(setup):
    """The library's own server (adanns_server_*): FP32, BF16 + rerank and IVF-OPQ
    requests over two resident indices, a burst submitted at once (shared
    batches) and a paced stream; every request equals the same rows searched
    alone through the search calls, bit for bit."""
    P, data, idx = setup
    from paper_2305_19435_gb300.serving import Budget, NativeServer
    if idx[16].opq is None:
        P.build_opq(idx[16], torch.from_numpy(data["db"]).cuda(), 64, 16, 2, 2, 4, 8_000, 3)
    budgets = [Budget(16, 128, 4, 10), Budget(64, 256, 8, 100, P.STORE_BF16, 400),
               Budget(16, 64, 1, 10, P.STORE_BF16, 40), Budget(16, 0, 6, 20, method=1),
               Budget(16, 0, 4, 10, rerank_k=80, method=1)]
    rng = np.random.default_rng(11)
    srv = NativeServer(idx, streams=3, max_batch=1024, mem_budget=8 << 30)
    q = data["queries"]
    reqs = []
    for i in range(10):
        b = budgets[i % 2]
        reqs.append((srv.submit(q[50 * i:50 * i + 31], b, index_key=b.d_c), b, 50 * i, 31))
    for i in range(40):
        n = int(rng.integers(1, 300))
        lo = int(rng.integers(0, len(q) - n))
        b = budgets[int(rng.integers(0, len(budgets)))]
        reqs.append((srv.submit(q[lo:lo + n], b, index_key=b.d_c), b, lo, n))
        time.sleep(float(rng.exponential(0.001)))
    for r, _, _, _ in reqs:
        assert r.wait(120)
    st = srv.stats()
    srv.stop()
    assert st["requests"] == 50 and st["queries"] == sum(n for _, _, _, n in reqs)
    assert st["batches"] < 50 and st["p99_ms"] >= st["p50_ms"] > 0
    for r, b, lo, n in reqs:
        assert r.error is None, r.error
        qq = torch.from_numpy(np.ascontiguousarray(q[lo:lo + n])).cuda()
        if b.method == 1:
            ids, dist = P.search_ivfopq(idx[b.d_c], qq, b.d_c, b.nprobe, b.k, rerank_k=b.rerank_k)
        else:
            ids, dist = P.search_ivf(idx[b.d_c], qq, b.d_c, b.d_s, b.nprobe, b.k,
                                     storage=b.storage, rerank_k=b.rerank_k)
        assert np.array_equal(r.ids, ids.cpu().numpy())
        assert np.array_equal(r.dist.view(np.int32), dist.cpu().numpy().view(np.int32))
        assert r.latency_ms > 0
    for g in idx.values():
        g.status()


def test_native_server_packs_mixed_budgets(setup):
    """Requests of one index with different d_s / nprobe / k (FP32 tier), with
    different nprobe / k at one d_s (BF16 tier) and with different nprobe / k
    (IVF-OPQ) share batches: a burst queued behind a long request is served in
    a few launches of the per-query-budget searches, and every request equals
    the same rows searched alone, bit for bit."""
    P, data, idx = setup
    from paper_2305_19435_gb300.serving import Budget, NativeServer
    if idx[16].opq is None:
        P.build_opq(idx[16], torch.from_numpy(data["db"]).cuda(), 64, 16, 2, 2, 4, 8_000, 3)
    rng = np.random.default_rng(13)
    q = data["queries"]
    srv = NativeServer(idx, streams=1, max_batch=2048, mem_budget=8 << 30)
    reqs = [(srv.submit(q[:1500], Budget(64, 256, 48, 100), index_key=64),
             Budget(64, 256, 48, 100), 0, 1500)]
    for i in range(36):
        n = int(rng.integers(1, 60))
        lo = int(rng.integers(0, len(q) - n))
        if i % 3 == 1:
            b = Budget(64, int(rng.choice([64, 128, 192, 256])), int(rng.integers(1, 30)),
                       int(rng.choice([1, 10, 100])))
        elif i % 3 == 2:
            b = Budget(16, 0, int(rng.integers(1, 30)), int(rng.choice([5, 20])), method=1)
        else:
            b = Budget(16, 128, int(rng.integers(1, 30)), int(rng.choice([5, 10])),
                       P.STORE_BF16, 40)
        reqs.append((srv.submit(q[lo:lo + n], b, index_key=b.d_c), b, lo, n))
    for r, _, _, _ in reqs:
        assert r.wait(120)
    st = srv.stats()
    srv.stop()
    assert st["requests"] == 37
    assert st["batches"] <= 8, st      # the burst shares launches across budgets
    for r, b, lo, n in reqs:
        assert r.error is None, r.error
        qq = torch.from_numpy(np.ascontiguousarray(q[lo:lo + n])).cuda()
        # BF16: the batch's shortlist is pruned against its largest k, which keeps
        # a superset of what the request's own k keeps (certified pruning)
        if b.method == 1:
            ids, dist = P.search_ivfopq(idx[b.d_c], qq, b.d_c, b.nprobe, b.k)
        else:
            ids, dist = P.search_ivf(idx[b.d_c], qq, b.d_c, b.d_s, b.nprobe, b.k,
                                     storage=b.storage, rerank_k=b.rerank_k)
        assert np.array_equal(r.ids, ids.cpu().numpy())
        assert np.array_equal(r.dist.view(np.int32),
                              np.ascontiguousarray(dist.cpu().numpy()).view(np.int32))
    for g in idx.values():
        g.status()


def test_native_server_rejects_bad_requests(setup):
    P, data, idx = setup
    from paper_2305_19435_gb300.serving import Budget, NativeServer
    srv = NativeServer({64: idx[64]}, streams=1, max_batch=64)
    q = data["queries"][:8]
    for b, code in ((Budget(16, 100, 4, 10), -2),               # d_s not a granularity
                    (Budget(16, 128, 4, 0), -1),                # k = 0
                    (Budget(16, 128, 4, 10, P.STORE_BF16, 4), -1),   # shortlist below k
                    (Budget(16, 0, 4, 10, method=1), -6)):      # no OPQ data on this index
        with pytest.raises(P.AdannsError) as e:
            srv.submit(q, b, index_key=64)
        assert e.value.code == code
    with pytest.raises(P.AdannsError):
        srv.submit(data["queries"][:65], Budget(16, 128, 4, 10), index_key=64)  # > max_batch
    r = srv.submit(q, Budget(64, 128, 4, 10), index_key=64)
    assert r.wait(60) and r.error is None
    srv.stop()
