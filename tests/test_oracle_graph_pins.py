"""Pins for the graph shortlist oracle (AdANNS-DiskANN, Sec. 4.3: graph formed
with a low-d MR, shortlist re-ranked with a high-d MR).  Checked against a
hand-worked example, brute force by another route, and the special cases that
reduce to exact search; never against itself."""
import numpy as np

import oracle
import synthdata
from conftest import read_golden
from parity import check_topk

L2, PN = oracle.METRIC_L2, oracle.METRIC_L2_PREFIXNORM


def line_case():
    g = read_golden("graph_line.txt")
    pos = np.array([float(v) for v in g["positions"][0]], dtype=np.float32)
    return g, pos[:, None]


def test_graph_build_hand_example():
    g, db = line_case()
    gr = oracle.build_graph(db, 1, 4, 2, 1.0, metric=L2)
    for r in range(5):
        want = [int(v) for v in g[f"row{r}"][0]]
        got = [int(v) for v in gr["graph"][r] if v >= 0]
        assert got == want, (r, got, want)
    assert gr["entry"] == int(g["entry"][0][0])
    assert not gr["amb"].any()


def test_graph_search_hand_example():
    g, db = line_case()
    gr = oracle.build_graph(db, 1, 4, 2, 1.0, metric=L2)
    q = np.array([[7.0]], dtype=np.float32)
    r = oracle.search_graph(db, gr, q, 2, 1, 2, 2)
    assert r["short_ids"][0].tolist() == [int(v) for v in g["search_ids"][0]]
    assert r["short_dist"][0].tolist() == [float(v) for v in g["search_dist"][0]]
    assert int(r["expanded"][0]) == int(g["search_expanded"][0][0])
    # the rerank at the same single coordinate keeps the same order
    assert r["ids"][0].tolist() == [3, 4] and r["dist"][0].tolist() == [1.0, 9.0]


def brute_knn(db, m, K, metric):
    """K nearest other rows by the Gram expansion with an FP64 matrix product."""
    X = db[:, :m].astype(np.float64)
    if metric == PN:
        n = np.linalg.norm(X, axis=1, keepdims=True)
        X = np.divide(X, n, out=np.zeros_like(X), where=n > 0)
    D = (X * X).sum(1)[:, None] + (X * X).sum(1)[None, :] - 2.0 * X @ X.T
    np.fill_diagonal(D, np.inf)
    order = np.lexsort((np.broadcast_to(np.arange(len(X)), D.shape), D), axis=1)[:, :K]
    return order, np.take_along_axis(np.maximum(D, 0), order, 1)


def test_knn_graph_is_brute_force():
    data = synthdata.small(700, 1, 32, 8, 51)
    nbr, dist, amb = oracle.knn_graph(data["db"], 16, 12)
    ref, rd = brute_knn(data["db"], 16, 12, PN)
    assert np.allclose(dist, rd, rtol=1e-9, atol=1e-12)
    n, fails = check_topk(nbr.astype(np.int64), dist, ref, rd, 12)
    assert not fails


def test_huge_alpha_keeps_the_nearest_candidates():
    """alpha so large that no candidate is ever pruned (distinct points): every
    forward list is the R nearest neighbours, and the final rows contain them."""
    data = synthdata.small(400, 1, 16, 6, 52)
    gr = oracle.build_graph(data["db"], 16, 20, 6, 1e30)
    nbr, _, _ = oracle.knn_graph(data["db"], 16, 6)
    for p in range(400):
        assert set(nbr[p].tolist()) <= set(gr["graph"][p][gr["graph"][p] >= 0].tolist())


def test_complete_graph_search_is_exact():
    """A graph where every row links to every other row: the search expands
    the entry and then sees every row, so its shortlist is the exact kk
    nearest at d_g, and with every row re-ranked the result is the exact
    search at d_s."""
    data = synthdata.small(60, 8, 32, 4, 53)
    db, q = data["db"], data["queries"]
    N = len(db)
    full = np.array([[j for j in range(N) if j != i] for i in range(N)], dtype=np.int32)
    gr = {"graph": full, "entry": 0, "d_g": 8, "R": N - 1, "metric": PN}
    r = oracle.search_graph(db, gr, q, N, 32, 5, 20)
    ref, rd = [], []
    X8 = oracle.prefix(db, 8)
    for i in range(len(q)):
        d = ((X8 - oracle.prefix(q[i:i + 1], 8)) ** 2).sum(1)
        o = np.lexsort((np.arange(N), d))[:20]
        assert np.array_equal(r["short_ids"][i], o)
        assert np.allclose(r["short_dist"][i], d[o], rtol=1e-12, atol=1e-14)
    r2 = oracle.search_graph(db, gr, q, N, 32, 5, N)
    one = {"centroids": np.zeros((1, 8), np.float32), "list_off": np.array([0, N], np.int64),
           "list_ids": np.arange(N, dtype=np.int32), "metric": PN}
    ex = oracle.search_ivf(db, one, q, 8, 32, 1, 5)
    n, fails = check_topk(r2["ids"], r2["dist"], ex["ids"], ex["dist"], 5)
    assert not fails


def test_graph_degree_and_symmetry_properties():
    """Rows hold at most R distinct ids, never themselves, sorted by distance;
    on a clustered sample the search reaches recall@10 >= 0.9 of exact search."""
    data = synthdata.small(3000, 40, 64, 24, 54)
    db, q = data["db"], data["queries"]
    gr = oracle.build_graph(db, 16, 32, 16, 1.2)
    X = oracle.prefix(db, 16)
    for p in range(0, 3000, 37):
        row = gr["graph"][p][gr["graph"][p] >= 0]
        assert len(row) == len(set(row.tolist())) and p not in row and 0 < len(row) <= 16
        d = ((X[row] - X[p]) ** 2).sum(1)
        assert np.all(np.diff(d) >= 0)
    r = oracle.search_graph(db, gr, q, 64, 64, 10, 40)
    one = {"centroids": np.zeros((1, 16), np.float32), "list_off": np.array([0, 3000], np.int64),
           "list_ids": np.arange(3000, dtype=np.int32), "metric": PN}
    ex = oracle.search_ivf(db, one, q, 16, 64, 1, 10)
    rec = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(r["ids"], ex["ids"])])
    assert rec >= 0.9, rec


def test_graph_pin_catches_a_reversed_prune_test():
    """Planted slip: keeping instead of dropping the candidates that the chosen
    neighbour covers changes the hand example's rows."""
    g, db = line_case()
    X = db.astype(np.float64)
    # prune of row 0 written with the comparison reversed
    cand = [1, 2, 3, 4]
    out, alive = [], list(cand)
    while alive and len(out) < 2:
        c = alive.pop(0)
        out.append(c)
        alive = [v for v in alive if ((X[c] - X[v]) ** 2).sum() <= ((X[0] - X[v]) ** 2).sum()]
    assert out != [int(v) for v in g["row0"][0]]
