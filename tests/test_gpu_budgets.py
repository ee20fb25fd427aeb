"""Per-query budgets in one search pass (adanns_search_ivf_budgets): every query
of a batch carries its own d_s, nprobe and k (Sec. 5, compute-aware elastic
search).  Each row is checked against the FP64 oracle searched with that
query's own budget, and against the single-budget search call on the same rows
(bit for bit).
"""
import numpy as np
import pytest

import oracle
import synthdata
from parity import ambiguous_probe_rows, check_topk, full_groups, recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PN = oracle.METRIC_L2_PREFIXNORM


@pytest.fixture(scope="module")
def A():
    import paper_2305_19435_gb300 as P
    P.build()
    return P


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def setup(A):
    # d = 512: d_s from 8 (half a 16-coordinate block) to 512; 40 lists
    data = synthdata.small(9000, 260, 512, 48, 811)
    o = oracle.build_ivf(data["db"], 32, 40, 5, 9000, seed=5)
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                       storage=1 | A.STORE_BF16)
    yield data, o, g
    g.free()


def groups(*cols):
    """rows of each distinct tuple of per-query values"""
    keys = list(zip(*[c.tolist() for c in cols]))
    out = {}
    for i, key in enumerate(keys):
        out.setdefault(key, []).append(i)
    return {k: np.array(v) for k, v in out.items()}


# FP32 routes: about 10 queries per probed list take the streaming scan with a
# d_s per query; about 80 take the tiled scan, one pass per d_s group
F32_PROBES = {"stream": [1, 2, 3], "tiled": [1, 2, 5, 13, 40]}


@pytest.mark.parametrize("route", ["stream", "tiled"])
def test_budgets_f32_match_oracle_per_query(A, setup, route):
    data, o, g = setup
    db, q = data["db"], data["queries"]
    rng = np.random.default_rng(3)
    B = len(q)
    ds = rng.choice([8, 16, 48, 64, 96, 192, 256, 512], B).astype(np.int32)
    npb = rng.choice(F32_PROBES[route], B).astype(np.int32)
    kq = rng.choice([1, 7, 10, 33], B).astype(np.int32)
    gi, gd = A.search_ivf_budgets(g, cu(q), 32, ds, npb, kq, k_max=40)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    checked = 0
    for (d_s, nprobe, k), rows in groups(ds, npb, kq).items():
        # padding past each query's own k
        assert np.all(gi[rows, k:] == -1) and np.all(np.isinf(gd[rows, k:]))
        ores = full_groups(oracle.search_ivf(db, o, q[rows], 32, d_s, nprobe, k + 16),
                           lambda r, kk: oracle.search_ivf(db, o, q[rows][r], 32, d_s, nprobe, kk),
                           k)
        amb = ambiguous_probe_rows(ores["probe_dist"], nprobe)
        n, fails = check_topk(gi[rows, :k], gd[rows, :k], ores["ids"], ores["dist"], k,
                              skip_rows=amb)
        assert not fails, (d_s, nprobe, k, fails[:2])
        checked += n
    assert checked > 0.9 * B


@pytest.mark.parametrize("route", ["stream", "tiled"])
def test_budgets_f32_equal_single_budget_calls(A, setup, route):
    data, o, g = setup
    q = data["queries"]
    rng = np.random.default_rng(4)
    B = len(q)
    ds = rng.choice([16, 64, 128, 384, 512], B).astype(np.int32)
    npb = rng.choice(F32_PROBES[route], B).astype(np.int32)
    kq = rng.choice([5, 50, 100], B).astype(np.int32)
    gi, gd = A.search_ivf_budgets(g, cu(q), 16, ds, npb, kq)   # IVF-D: d_c below the built 32
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert gi.shape == (B, 100)
    for (d_s, nprobe, k), rows in groups(ds, npb, kq).items():
        si, sd = A.search_ivf(g, cu(q[rows]), 16, d_s, nprobe, k)
        assert np.array_equal(gi[rows, :k], si.cpu().numpy())
        assert np.array_equal(gd[rows, :k].view(np.int32), sd.cpu().numpy().view(np.int32))


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_budgets_lowp_equal_single_budget_calls(A, setup, storage):
    data, o, g = setup
    db, q = data["db"], data["queries"]
    st = A.STORE_BF16 if storage == "bf16" else A.STORE_FP8
    if storage == "fp8":
        g = A.index_create(cu(db), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                           storage=1 | A.STORE_FP8)
    rng = np.random.default_rng(5)
    B = len(q)
    npb = rng.choice([1, 4, 9, 40], B).astype(np.int32)
    kq = rng.choice([1, 10, 25], B).astype(np.int32)
    gi, gd = A.search_ivf_budgets(g, cu(q), 32, 256, npb, kq, k_max=25, storage=st, rerank_k=100)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    for (nprobe, k), rows in groups(npb, kq).items():
        si, sd = A.search_ivf(g, cu(q[rows]), 32, 256, nprobe, 25, storage=st, rerank_k=100)
        assert np.array_equal(gi[rows, :k], si.cpu().numpy()[:, :k])
        assert np.array_equal(gd[rows, :k].view(np.int32),
                              sd.cpu().numpy()[:, :k].view(np.int32))
        assert np.all(gi[rows, k:] == -1)
        # certified pruning against k_max keeps a superset of what the query's
        # own k keeps: the same k best as a call with k itself
        si, sd = A.search_ivf(g, cu(q[rows]), 32, 256, nprobe, k, storage=st, rerank_k=100)
        assert np.array_equal(gi[rows, :k], si.cpu().numpy())
        # the shortlist holds the exact top-k: recall against the oracle
        ores = oracle.search_ivf(db, o, q[rows], 32, 256, nprobe, k)
        assert recall(gi[rows, :k], ores["ids"], k) >= 0.97
    if storage == "fp8":
        g.free()


def test_budgets_argument_errors(A, setup):
    data, o, g = setup
    q = cu(data["queries"][:4])
    bad = [
        (dict(d_s=[64, 64, 100, 64], nprobe=2, k=5), -2),             # 100 not a granularity
        (dict(d_s=64, nprobe=[1, 0, 1, 1], k=5), -1),                 # nprobe 0
        (dict(d_s=64, nprobe=[1, 41, 1, 1], k=5), -1),                # above nlist
        (dict(d_s=64, nprobe=2, k=[5, 5, 9, 5], k_max=8), -1),        # k above k_max
        (dict(d_s=[64, 128, 64, 64], nprobe=2, k=5, storage=A.STORE_BF16, rerank_k=20), -1),
        (dict(d_s=64, nprobe=2, k=5, storage=A.STORE_BF16, rerank_k=4), -1),
        (dict(d_s=64, nprobe=2, k=5, rerank_k=20), -1),                # FP32 takes no shortlist
    ]
    for kw, code in bad:
        with pytest.raises(A.AdannsError) as e:
            A.search_ivf_budgets(g, q, 32, **kw)
        assert e.value.code == code, kw
    # an empty batch is a no-op
    ids, dist = A.search_ivf_budgets(g, q[:0], 32, [], [], [], k_max=5)
    assert ids.shape == (0, 5)


@pytest.fixture(scope="module")
def opq_case(A):
    """an IVF-OPQ index (d = 96, d_s = 64, M = 16) built by the oracle"""
    data = synthdata.small(12_000, 240, 96, 48, 821)
    db = data["db"]
    o = oracle.build_ivf(db, 32, 24, 6, 12_000, seed=9)
    opq = oracle.train_opq(db, 64, 16, 3, 3, 5, 4000, seed=13)
    codes = oracle.pq_encode(db, 64, 16, opq["R"], opq["codebooks"])
    g = A.index_create(cu(db), cu(o["centroids"]), cu(o["assign"].astype(np.int32)))
    A.set_opq(g, 64, 16, cu(opq["R"]), cu(opq["codebooks"]), cu(codes))
    yield data, o, opq, codes, g
    g.free()


def test_budgets_ivfopq_match_oracle_and_single_calls(A, opq_case):
    data, o, opq, codes, g = opq_case
    db, q = data["db"], data["queries"]
    rng = np.random.default_rng(6)
    B = len(q)
    npb = rng.choice([1, 3, 8, 24], B).astype(np.int32)
    kq = rng.choice([1, 10, 30], B).astype(np.int32)
    gi, gd = A.search_ivfopq_budgets(g, cu(q), 32, npb, kq, k_max=30)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    for (nprobe, k), rows in groups(npb, kq).items():
        assert np.all(gi[rows, k:] == -1) and np.all(np.isinf(gd[rows, k:]))
        si, sd = A.search_ivfopq(g, cu(q[rows]), 32, nprobe, k)
        assert np.array_equal(gi[rows, :k], si.cpu().numpy())
        assert np.array_equal(gd[rows, :k].view(np.int32), sd.cpu().numpy().view(np.int32))
        orr = oracle.search_ivfopq(db, o, opq, codes, q[rows], 32, nprobe, k + 20)
        amb = ambiguous_probe_rows(orr["probe_dist"], nprobe)
        n, fails = check_topk(gi[rows, :k], gd[rows, :k], orr["ids"], orr["dist"], k,
                              skip_rows=amb)
        assert not fails, (nprobe, k, fails[:2])


def test_budgets_ivfopq_rerank_equal_single_calls(A, opq_case):
    data, o, opq, codes, g = opq_case
    q = data["queries"]
    rng = np.random.default_rng(7)
    B = len(q)
    npb = rng.choice([2, 6, 24], B).astype(np.int32)
    kq = rng.choice([5, 10], B).astype(np.int32)
    gi, gd = A.search_ivfopq_budgets(g, cu(q), 32, npb, kq, k_max=10, rerank_k=40)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    for (nprobe, k), rows in groups(npb, kq).items():
        # the shortlist is the rerank_k best by ADC for every k: the k best of
        # the re-scored shortlist are a prefix of the k_max best
        si, sd = A.search_ivfopq(g, cu(q[rows]), 32, nprobe, 10, rerank_k=40)
        assert np.array_equal(gi[rows, :k], si.cpu().numpy()[:, :k])
        assert np.array_equal(gd[rows, :k].view(np.int32),
                              np.ascontiguousarray(sd.cpu().numpy()[:, :k]).view(np.int32))
    with pytest.raises(A.AdannsError) as e:
        A.search_ivfopq_budgets(g, cu(q[:3]), 32, [1, 300, 2], 5)     # nprobe above 256
    assert e.value.code == -1
    with pytest.raises(A.AdannsError) as e:
        A.search_ivfopq_budgets(g, cu(q[:3]), 32, 2, [5, 5, 5], k_max=5, rerank_k=4)
    assert e.value.code == -1
