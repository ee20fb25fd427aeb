"""Low-d graph shortlist + high-d rerank (AdANNS-DiskANN, Sec. 4.3) against the
FP64 oracle.

* Search parity on the oracle's own graph (imported): for every query whose
  traversal made no decision within the FP32 tolerance (the oracle flags the
  others), the GPU's shortlist holds the oracle's rows and the re-ranked ids
  and distances match under the parity rule.
* The GPU build against the oracle's build of the same rows: the same entry
  point and the same neighbour set for nearly every row (decisions within the
  tolerance can differ and propagate through offered edges).
* The GPU-built graph searches with high recall of exact search.
"""
import numpy as np
import pytest

import oracle
import synthdata
from parity import check_topk, recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import paper_2305_19435_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    return P


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def case():
    data = synthdata.small(20_000, 300, 128, 64, 801)
    gr = oracle.build_graph(data["db"], 16, 48, 24, 1.2)
    return data, gr


def exact(data, d_s, k):
    N = data["db"].shape[0]
    one = {"centroids": np.zeros((1, 8), np.float32), "list_off": np.array([0, N], np.int64),
           "list_ids": np.arange(N, dtype=np.int32), "metric": oracle.METRIC_L2_PREFIXNORM}
    return oracle.search_ivf(data["db"], one, data["queries"], 8, d_s, 1, k)


@pytest.mark.parametrize("L,d_s,k,kr", [(64, 128, 10, 40), (32, 64, 5, 32), (128, 96, 20, 80),
                                        (200, 128, 100, 200)])
def test_graph_search_parity_on_oracle_graph(A, case, L, d_s, k, kr):
    data, gr = case
    g = A.graph_create(cu(data["db"]), 16, cu(gr["graph"]), gr["entry"])
    gi, gd, gs = A.graph_search(g, cu(data["queries"]), L, d_s, k, kr, return_shortlist=True)
    ref = oracle.search_graph(data["db"], gr, data["queries"], L, d_s, k, kr)
    # a query is flagged when one of its many traversal comparisons fell within
    # the FP32 error bound of the distances (about 1e-5 relative at d_g = 16);
    # longer lists make more comparisons and flag more queries
    amb = ref["amb"]
    assert amb.mean() < 0.6, amb.mean()
    gs = gs.cpu().numpy()
    for i in np.nonzero(~amb)[0]:
        assert set(gs[i].tolist()) == set(ref["short_ids"][i].tolist()), i
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    n, fails = check_topk(gi, gd, ref["ids"], ref["dist"], k, skip_rows=amb)
    assert n > 0.4 * len(amb) and not fails, fails[:2]
    # the flagged queries still agree with the oracle almost everywhere
    assert recall(gi, ref["ids"], k) >= 0.98
    g.free()


def test_graph_build_matches_oracle(A, case):
    data, gr = case
    g = A.graph_build(cu(data["db"]), 16, 48, 24, 1.2)
    assert g.entry == gr["entry"]
    nb = g.neighbours().cpu().numpy()
    same = np.array([set(nb[p][nb[p] >= 0].tolist()) == set(gr["graph"][p][gr["graph"][p] >= 0].tolist())
                     for p in range(len(nb))])
    clean = ~gr["amb"]
    assert same[clean].mean() >= 0.99, same[clean].mean()
    # rows are sorted by distance, hold no self edge and no duplicate
    X = oracle.prefix(data["db"], 16)
    for p in range(0, len(nb), 97):
        row = nb[p][nb[p] >= 0]
        assert p not in row and len(row) == len(set(row.tolist())) and len(row) <= 24
        d = ((X[row] - X[p]) ** 2).sum(1)
        assert np.all(np.diff(d) >= -1e-6)
    g.free()


def test_gpu_built_graph_recall(A, case):
    data, _ = case
    g = A.graph_build(cu(data["db"]), 16, 48, 24, 1.2)
    gi, gd = A.graph_search(g, cu(data["queries"]), 64, 128, 10, 40)
    ex = exact(data, 128, 10)
    r = recall(gi.cpu().numpy(), ex["ids"], 10)
    assert r >= 0.95, r
    # the returned distances are the exact d_s distances of the returned ids
    P = oracle.prefix(data["queries"], 128)
    ids = gi.cpu().numpy()
    X = oracle.prefix(data["db"][ids[:50].ravel()], 128).reshape(50, 10, 128)
    dd = ((X - P[:50, None, :]) ** 2).sum(-1)
    assert np.allclose(gd.cpu().numpy()[:50], dd, rtol=1e-5, atol=2.4e-7)
    g.free()


def test_graph_errors(A, case):
    data, gr = case
    db = cu(data["db"][:1000])
    with pytest.raises(A.AdannsError) as e:
        A.graph_build(db, 12, 16, 8, 1.2)          # d_g not a granularity
    assert e.value.code == -2
    with pytest.raises(A.AdannsError) as e:
        A.graph_build(db, 16, 16, 80, 1.2)         # R above 64
    assert e.value.code == -1
    with pytest.raises(A.AdannsError) as e:
        A.graph_build(db, 16, 16, 8, 0.5)          # alpha below 1
    assert e.value.code == -1
    g = A.graph_build(db, 16, 16, 8, 1.2)
    with pytest.raises(A.AdannsError) as e:
        A.graph_search(g, cu(data["queries"][:4]), 16, 64, 10, 20)   # rerank_k above L
    assert e.value.code == -1
    g.free()
