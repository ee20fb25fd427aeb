"""Pins for the FP64 oracle: it is checked against closed forms, hand-worked
examples, published generator outputs, invariants and brute force, never
against itself.  Each test names the passage it pins."""
import numpy as np
import pytest

import oracle
import synthdata
from conftest import read_golden
from parity import check_topk

L2, PN = oracle.METRIC_L2, oracle.METRIC_L2_PREFIXNORM


def brute_force(db, queries, m, k, metric):
    """Exact kNN by the Gram expansion ||a||^2 + ||b||^2 - 2 a.b with an FP64
    matrix product: a different route from the oracle's difference-form loop."""
    def P(x):
        x = x[:, :m].astype(np.float64)
        if metric == PN:
            n = np.linalg.norm(x, axis=1, keepdims=True)
            x = np.divide(x, n, out=np.zeros_like(x), where=n > 0)
        return x
    X, Q = P(db), P(queries)
    D = (Q * Q).sum(1)[:, None] + (X * X).sum(1)[None, :] - 2.0 * Q @ X.T
    D = np.maximum(D, 0.0)
    order = np.lexsort((np.broadcast_to(np.arange(X.shape[0]), D.shape), D), axis=1)[:, :k]
    return order.astype(np.int64), np.take_along_axis(D, order, 1)


# ---------------------------------------------------------------- generator
def test_splitmix64_published_vectors():
    g = read_golden("splitmix64.txt")
    for seed_key in ("0", "1234567"):
        want = [int(v) for v in g[seed_key][0]]
        assert oracle.splitmix64(int(seed_key), len(want)) == want


def test_sample_is_prefix_of_permutation():
    p = oracle.sample(7, 1000, 1000)
    assert sorted(p.tolist()) == list(range(1000))
    # the first draw is j = next() mod n, from the pinned generator
    first = oracle.splitmix64(7, 1)[0]
    assert oracle.sample(7, 1000, 1)[0] == first % 1000
    assert np.array_equal(oracle.sample(7, 1000, 10), p[:10])


# ---------------------------------------------------------------- prefixes
def test_prefix_normalisation_hand_example():
    g = read_golden("prefix_norm.txt")
    v = np.array([[float(x) for x in g["v"][0]]], dtype=np.float32)
    assert np.allclose(oracle.prefix(v, 2)[0], [float(x) for x in g["P2"][0]], rtol=0, atol=1e-15)
    assert np.allclose(oracle.prefix(v, 3)[0], [float(x) for x in g["P3"][0]], rtol=0, atol=1e-15)
    z = np.zeros((1, 3), dtype=np.float32)
    assert np.all(oracle.prefix(z, 3) == 0.0)          # P_m(0) = 0
    assert np.allclose(oracle.prefix(v, 2, L2)[0], [3.0, 4.0])   # raw prefix


def test_prefix_unit_norm_and_scale_invariance():
    x = synthdata.small(50, 1, 48, 4, 3)["db"]
    for m in (8, 16, 48):
        P = oracle.prefix(x, m)
        assert np.allclose(np.linalg.norm(P, axis=1), 1.0, atol=1e-14)
        assert np.allclose(oracle.prefix(4.0 * x, m), P, atol=1e-15)


# ---------------------------------------------------------------- k-means
def test_lloyd_hand_example():
    g = read_golden("lloyd_1d.txt")
    T = np.array([[float(v)] for v in g["points"][0]])
    C0 = np.array([[float(v)] for v in g["init"][0]])
    C, objs = oracle.lloyd(T, C0, 3)
    assert np.allclose(objs, [float(v) for v in g["objective"][0]], rtol=1e-15, atol=0)
    assert np.allclose(C[:, 0], [float(v) for v in g["final"][0]], rtol=0, atol=1e-15)
    a, _, _ = oracle.assign(T, C)
    assert a.tolist() == [int(v) for v in g["assign_final"][0]]


def test_assign_tie_goes_to_smallest_index_and_runner_up():
    T = np.array([[5.0]])
    a, b, s = oracle.assign(T, np.array([[6.0], [4.0], [9.0]]))
    assert a[0] == 0 and b[0] == 1.0 and s[0] == 1.0
    a, b, s = oracle.assign(T, np.array([[9.0], [4.5], [4.0]]))
    assert a[0] == 1 and b[0] == 0.25 and s[0] == 1.0


def test_empty_cluster_keeps_centroid():
    T = np.array([[0.0], [1.0]])
    C = oracle.update(T, np.array([0, 0], dtype=np.int32), np.array([[5.0], [7.0]]))
    assert C[0, 0] == 0.5 and C[1, 0] == 7.0


def test_kmeans_each_point_its_own_centroid():
    x = synthdata.small(3, 1, 16, 3, 5)["db"]
    idx = oracle.build_ivf(x, 16, 3, 4, 3, seed=9)
    assert idx["objectives"][-1] == 0.0
    assert sorted(idx["assign"].tolist()) == [0, 1, 2]


def test_kmeans_objective_never_increases():
    data = synthdata.small(3000, 1, 32, 16, 11)
    idx = oracle.build_ivf(data["db"], 16, 24, 15, 3000, seed=5)
    J = np.array(idx["objectives"])
    assert np.all(J[1:] <= J[:-1] * (1 + 1e-12))
    assert J[-1] < J[0]


def test_final_assignment_is_nearest_fp32_centroid():
    data = synthdata.small(2000, 1, 32, 8, 12)
    idx = oracle.build_ivf(data["db"], 16, 8, 5, 1000, seed=1)
    X = oracle.prefix(data["db"], 16)
    C = idx["centroids"].astype(np.float64)
    D = ((X[:, None, :] - C[None]) ** 2).sum(-1)
    assert np.array_equal(idx["assign"], np.argmin(D, axis=1))
    off, ids = idx["list_off"], idx["list_ids"]
    assert off[-1] == 2000 and sorted(ids.tolist()) == list(range(2000))
    for l in range(8):
        mem = ids[off[l]:off[l + 1]]
        assert np.all(np.diff(mem) > 0) and np.all(idx["assign"][mem] == l)


# ---------------------------------------------------------------- IVF search
@pytest.mark.parametrize("metric", [PN, L2])
def test_full_probe_full_dim_equals_exact_search(metric):
    """n_p = nlist and d_s = d scans every point at full dimension: IVF then is
    exact search (Sec. 3 "IVF"; Table "formula")."""
    data = synthdata.small(1500, 40, 32, 12, 21)
    db, q = data["db"].copy(), data["queries"].copy()
    db[7] = db[3]          # duplicate vectors (a tie)
    q[5] = db[11]          # a query equal to a database vector (distance 0)
    db[13] = 0.0           # zero vector (P_m(0) = 0)
    idx = oracle.build_ivf(db, 8, 10, 6, 1500, seed=3, metric=metric)
    k = 25
    res = oracle.search_ivf(db, idx, q, 8, 32, 10, k + 10)
    bi, bd = brute_force(db, q, 32, k + 10, metric)
    assert np.allclose(res["dist"], bd, rtol=1e-9, atol=1e-9)
    scale = None if metric == PN else (q.astype(np.float64) ** 2).sum(1)
    n, fails = check_topk(res["ids"], res["dist"], bi, bd, k, scale=scale)
    assert not fails, fails[:3]
    assert res["ids"][5, 0] == 11 and res["dist"][5, 0] == 0.0


def test_prefix_scan_equals_exact_search_on_prefix():
    """With all lists probed, the scan at d_s < d is exact search on P_ds."""
    data = synthdata.small(800, 20, 64, 6, 22)
    idx = oracle.build_ivf(data["db"], 16, 6, 4, 800, seed=4)
    res = oracle.search_ivf(data["db"], idx, data["queries"], 16, 24, 6, 12)
    bi, bd = brute_force(data["db"], data["queries"], 24, 12, PN)
    assert np.allclose(res["dist"], bd, rtol=1e-9, atol=1e-9)
    n, fails = check_topk(res["ids"], res["dist"], bi, bd, 12)
    assert not fails


def test_cluster_mapping_and_single_probe():
    """n_p = 1: results come from the list of the nearest centroid at d_c."""
    data = synthdata.small(1000, 30, 32, 8, 23)
    idx = oracle.build_ivf(data["db"], 8, 12, 5, 1000, seed=6)
    res = oracle.search_ivf(data["db"], idx, data["queries"], 8, 32, 1, 10)
    Q = oracle.prefix(data["queries"], 8)
    C = idx["centroids"].astype(np.float64)
    D = (Q * Q).sum(1)[:, None] + (C * C).sum(1)[None] - 2 * Q @ C.T
    near = np.argmin(D, axis=1)
    assert np.array_equal(res["probes"][:, 0], near)
    for i in range(30):
        got = res["ids"][i][res["ids"][i] >= 0]
        assert np.all(idx["assign"][got] == near[i])


def test_ivf_d_uses_the_stored_centroid_prefix():
    """IVF-D (Table "formula" IVF-D row) probes with P_dhat(q) against the first
    d_hat coordinates of the centroids as stored.  Hand case, d_hat = 8 of a
    16-dim index: P_8(q) = e0; centroid A's prefix is 0.3 e0 (distance 0.49),
    B's is 0.8 e0 + 0.6 e1 (distance 0.40), so the single probe is B; had the
    centroid prefix been renormalised, A (distance 0) would win."""
    C = np.zeros((2, 16), dtype=np.float32)
    C[0, 0], C[0, 8] = 0.3, 0.95
    C[1, 0], C[1, 1] = 0.8, 0.6
    db = np.zeros((2, 32), dtype=np.float32)
    db[0, 0], db[0, 9] = 1.0, 1.0
    db[1, 0], db[1, 1] = 1.0, 1.0
    off, ids = oracle.lists_from_assignment(np.array([0, 1]), 2)
    idx = {"centroids": C, "list_off": off, "list_ids": ids, "metric": PN}
    q = np.zeros((1, 32), dtype=np.float32)
    q[0, 0], q[0, 20] = 2.0, 5.0
    res = oracle.search_ivf(db, idx, q, 8, 32, 1, 1)
    assert res["probes"][0, 0] == 1 and res["ids"][0, 0] == 1
    assert res["probe_dist"][0, 0] == pytest.approx(0.04 + 0.36, abs=1e-6)
    assert res["probe_dist"][0, 1] == pytest.approx(0.49, abs=1e-6)
    # d_hat = the built d_c is plain AdANNS-IVF: P_16(q) = e0 as well
    res16 = oracle.search_ivf(db, idx, q, 16, 32, 2, 2)
    assert res16["probe_dist"][0, 0] == pytest.approx(0.40, abs=1e-6)
    assert res16["probe_dist"][0, 1] == pytest.approx(0.49 + 0.95 ** 2, abs=1e-6)


def test_probes_sorted_and_padding():
    data = synthdata.small(300, 10, 16, 4, 24)
    idx = oracle.build_ivf(data["db"], 16, 30, 3, 300, seed=7)
    res = oracle.search_ivf(data["db"], idx, data["queries"], 16, 16, 4, 200)
    pd = res["probe_dist"]
    assert np.all(np.diff(pd, axis=1) >= 0)
    for i in range(10):
        nc = res["ncand"][i]
        assert nc < 200
        assert np.all(res["ids"][i, nc:] == -1) and np.all(np.isinf(res["dist"][i, nc:]))
        assert np.all(res["ids"][i, :nc] >= 0)


def test_prefix_norm_distance_is_two_minus_two_cosine():
    data = synthdata.small(400, 8, 32, 4, 25)
    idx = oracle.build_ivf(data["db"], 8, 4, 3, 400, seed=8)
    res = oracle.search_ivf(data["db"], idx, data["queries"], 8, 32, 4, 5)
    for i in range(8):
        q = data["queries"][i].astype(np.float64)
        for j, dd in zip(res["ids"][i], res["dist"][i]):
            x = data["db"][j].astype(np.float64)
            cos = q @ x / np.linalg.norm(q) / np.linalg.norm(x)
            assert abs(dd - (2 - 2 * cos)) < 1e-12


# ---------------------------------------------------------------- PQ / OPQ
def test_opq_rotation_is_orthonormal_and_distortion_never_increases():
    data = synthdata.small(3000, 1, 64, 16, 31)
    opq = oracle.train_opq(data["db"], 32, 8, opq_iters=4, pq_iters=3, final_iters=4,
                           train_n=2000, seed=2)
    R = opq["R64"]
    assert np.allclose(R.T @ R, np.eye(32), atol=1e-10)
    Rf = opq["R"].astype(np.float64)
    assert np.allclose(Rf.T @ Rf, np.eye(32), atol=1e-6)
    tr = np.array(opq["trace"])
    assert np.all(tr[1:] <= tr[:-1] * (1 + 1e-12)), tr


def test_procrustes_is_optimal_and_identity_for_spd():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((200, 12))
    Zh = Y @ np.linalg.qr(rng.standard_normal((12, 12)))[0] + 0.1 * rng.standard_normal((200, 12))
    R = oracle.procrustes(Y, Zh)
    best = ((Y @ R - Zh) ** 2).sum()
    for _ in range(20):
        A = rng.standard_normal((12, 12)) * 1e-2
        Rp = R @ np.linalg.qr(np.eye(12) + A - A.T)[0]
        assert ((Y @ Rp - Zh) ** 2).sum() >= best - 1e-9
    # Y^T Y is symmetric positive definite, so its polar factor is I
    assert np.allclose(oracle.procrustes(Y, Y), np.eye(12), atol=1e-10)


def test_codes_are_nearest_codewords():
    data = synthdata.small(1500, 1, 32, 8, 32)
    opq = oracle.train_opq(data["db"], 32, 4, 2, 2, 3, 1500, seed=3)
    codes = oracle.pq_encode(data["db"][:64], 32, 4, opq["R"], opq["codebooks"])
    Z = oracle.prefix(data["db"][:64], 32) @ opq["R"].astype(np.float64)
    C = opq["codebooks"].astype(np.float64)
    for m in range(4):
        D = ((Z[:, None, m * 8:(m + 1) * 8] - C[m][None]) ** 2).sum(-1)
        assert np.array_equal(codes[:, m], np.argmin(D, axis=1))


def test_adc_is_distance_to_reconstruction():
    """ADC by M lookups equals ||z_q - decode(code_x)||^2 (Sec. 3 "OPQ")."""
    data = synthdata.small(1200, 12, 48, 8, 33)
    db, q = data["db"], data["queries"]
    idx = oracle.build_ivf(db, 16, 4, 4, 1200, seed=2)
    opq = oracle.train_opq(db, 48, 6, 2, 2, 3, 1200, seed=4)
    codes = oracle.pq_encode(db, 48, 6, opq["R"], opq["codebooks"])
    res = oracle.search_ivfopq(db, idx, opq, codes, q, 16, 4, 30)
    Zq = oracle.prefix(q, 48) @ opq["R"].astype(np.float64)
    rec = oracle.pq_decode(codes, opq["codebooks"].astype(np.float64))
    for i in range(12):
        dd = ((Zq[i][None] - rec[res["ids"][i]]) ** 2).sum(1)
        assert np.allclose(dd, res["dist"][i], rtol=1e-12, atol=1e-14)
        assert np.all(np.diff(res["dist"][i]) >= 0)


@pytest.mark.parametrize("opq_iters", [2, 0])
def test_one_list_ivfopq_is_exhaustive_adc(opq_iters):
    """Exhaustive AdANNS-OPQ (Sec. 4.2: ADC over every quantized vector) read as
    IVF-OPQ over an index with one list: the oracle's result is the full ADC
    ranking of every row by (||z_q - decode(code_x)||^2, id), computed here from
    the reconstructions.  opq_iters = 0 is plain PQ: the rotation stays I."""
    data = synthdata.small(900, 10, 32, 6, 35)
    db, q = data["db"], data["queries"]
    N = db.shape[0]
    opq = oracle.train_opq(db, 24, 6, opq_iters, 2, 3, 900, seed=8)
    if opq_iters == 0:
        assert np.array_equal(opq["R64"], np.eye(24))
    codes = oracle.pq_encode(db, 24, 6, opq["R"], opq["codebooks"])
    one = {"centroids": np.zeros((1, 8), np.float32), "list_off": np.array([0, N], np.int64),
           "list_ids": np.arange(N, dtype=np.int32), "assign": np.zeros(N, np.int32),
           "metric": PN}
    res = oracle.search_ivfopq(db, one, opq, codes, q, 8, 1, 25)
    Zq = oracle.prefix(q, 24) @ opq["R"].astype(np.float64)
    rec = oracle.pq_decode(codes, opq["codebooks"].astype(np.float64))
    for i in range(len(q)):
        dd = ((Zq[i][None] - rec) ** 2).sum(1)
        order = np.lexsort((np.arange(N), dd))[:25]
        assert np.array_equal(res["ids"][i], order)
        assert np.allclose(res["dist"][i], dd[order], rtol=1e-12, atol=1e-14)


def test_small_training_set_makes_adc_exact():
    """With at most 256 training points each point is its own codeword and
    the Procrustes factor of the SPD matrix Y^T Y is I, so ADC on the training
    points equals the exact distance and IVF-OPQ equals IVF."""
    data = synthdata.small(200, 15, 32, 4, 34)
    db, q = data["db"], data["queries"]
    opq = oracle.train_opq(db, 16, 4, 3, 2, 2, 200, seed=5)
    assert np.allclose(opq["R64"], np.eye(16), atol=1e-9)
    codes = oracle.pq_encode(db, 16, 4, opq["R"], opq["codebooks"])
    idx = oracle.build_ivf(db, 8, 5, 3, 200, seed=6)
    a = oracle.search_ivfopq(db, idx, opq, codes, q, 8, 5, 20)
    b = oracle.search_ivf(db, idx, q, 8, 16, 5, 20)
    assert np.allclose(a["dist"], b["dist"], rtol=1e-6, atol=1e-7)
    n, fails = check_topk(a["ids"], a["dist"], b["ids"], b["dist"], 15)
    assert not fails


def test_list_centroids_are_member_means():
    """Residual centres: the mean of each list's normalised d_s prefixes,
    computed here list by list with np.mean; an empty list gets zeros."""
    data = synthdata.small(600, 5, 32, 4, 40)
    db = data["db"]
    idx = oracle.build_ivf(db, 8, 7, 3, 600, seed=9)
    idx = dict(idx)
    a = idx["assign"].copy()
    a[a == 6] = 5                          # list 6 becomes empty
    idx["assign"] = a
    lc = oracle.list_centroids(db, idx, 24)
    for l in range(7):
        rows = db[a == l, :24].astype(np.float64)
        if len(rows) == 0:
            assert np.all(lc[l] == 0)
            continue
        rows /= np.linalg.norm(rows, axis=1, keepdims=True)
        assert np.allclose(lc[l], rows.mean(0), rtol=1e-6, atol=1e-7)


def _residual_case(seed, N=1500, d=48, d_s=48, M=6, nlist=6, train_n=1500):
    data = synthdata.small(N, 12, d, 8, seed)
    db, q = data["db"], data["queries"]
    idx = oracle.build_ivf(db, 16, nlist, 4, N, seed=seed + 1)
    lc = oracle.list_centroids(db, idx, d_s)
    res = {"lcent": lc, "assign": idx["assign"]}
    opq = oracle.train_opq(db, d_s, M, 2, 2, 3, train_n, seed=seed + 2, residual=res)
    codes = oracle.pq_encode(db, d_s, M, opq["R"], opq["codebooks"], lcent=lc,
                             assign=idx["assign"])
    return db, q, idx, lc, opq, codes


def test_residual_adc_is_distance_to_reconstruction():
    """Residual IVF-OPQ: a member x of list l is reconstructed as
    lcent[l] + decode(code_x) R^T, and its ADC score equals the squared
    distance from P_ds(q) to that reconstruction (R orthogonal up to FP32
    rounding), computed here directly in the unrotated space."""
    db, q, idx, lc, opq, codes = _residual_case(41)
    res = oracle.search_ivfopq(db, idx, opq, codes, q, 16, 3, 40)
    Pq = oracle.prefix(q, 48)
    R = opq["R"].astype(np.float64)
    rec = oracle.pq_decode(codes, opq["codebooks"].astype(np.float64)) @ R.T + \
        lc[idx["assign"]].astype(np.float64)
    for i in range(len(q)):
        dd = ((Pq[i][None] - rec[res["ids"][i]]) ** 2).sum(1)
        assert np.allclose(dd, res["dist"][i], rtol=1e-5, atol=1e-7)
        assert np.all(np.diff(res["dist"][i]) >= 0)
        # every returned id lies in a probed list
        assert set(idx["assign"][res["ids"][i]]) <= set(res["probes"][i])


def test_residual_with_zero_centres_is_plain_ivfopq():
    """With all list centres zero the residual codes and tables are the plain
    ones: identical codes and results."""
    data = synthdata.small(1000, 10, 32, 6, 42)
    db, q = data["db"], data["queries"]
    idx = oracle.build_ivf(db, 8, 5, 3, 1000, seed=3)
    zero = np.zeros((5, 32), np.float32)
    res = {"lcent": zero, "assign": idx["assign"]}
    o1 = oracle.train_opq(db, 32, 4, 2, 2, 2, 1000, seed=4, residual=res)
    o0 = oracle.train_opq(db, 32, 4, 2, 2, 2, 1000, seed=4)
    assert np.array_equal(o1["R"], o0["R"]) and np.array_equal(o1["codebooks"], o0["codebooks"])
    c1 = oracle.pq_encode(db, 32, 4, o1["R"], o1["codebooks"], lcent=zero, assign=idx["assign"])
    c0 = oracle.pq_encode(db, 32, 4, o0["R"], o0["codebooks"])
    assert np.array_equal(c1, c0)
    a = oracle.search_ivfopq(db, idx, o1, c1, q, 8, 3, 10)
    b = oracle.search_ivfopq(db, idx, o0, c0, q, 8, 3, 10)
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["dist"], b["dist"])


def test_residual_small_training_set_is_exact():
    """At most 256 rows: every residual is its own codeword, so residual ADC is
    the exact distance up to the rotation's FP32 orthogonality, and IVF-OPQ
    ranks like IVF."""
    data = synthdata.small(220, 10, 32, 4, 43)
    db, q = data["db"], data["queries"]
    idx = oracle.build_ivf(db, 8, 4, 3, 220, seed=5)
    lc = oracle.list_centroids(db, idx, 16)
    res = {"lcent": lc, "assign": idx["assign"]}
    opq = oracle.train_opq(db, 16, 4, 2, 2, 2, 220, seed=6, residual=res)
    codes = oracle.pq_encode(db, 16, 4, opq["R"], opq["codebooks"], lcent=lc, assign=idx["assign"])
    a = oracle.search_ivfopq(db, idx, opq, codes, q, 8, 4, 15)
    b = oracle.search_ivf(db, idx, q, 8, 16, 4, 15)
    assert np.allclose(a["dist"], b["dist"], rtol=1e-5, atol=1e-6)
    n, fails = check_topk(a["ids"], a["dist"], b["ids"], b["dist"], 15)
    assert not fails


def test_residual_pin_catches_a_wrong_sign():
    """Planted slip: adding the list centre instead of subtracting it breaks
    the reconstruction pin."""
    db, q, idx, lc, opq, codes = _residual_case(44)
    res = oracle.search_ivfopq(db, idx, opq, codes, q, 16, 3, 40)
    Pq = oracle.prefix(q, 48)
    R = opq["R"].astype(np.float64)
    wrong = oracle.pq_decode(codes, opq["codebooks"].astype(np.float64)) @ R.T - \
        lc[idx["assign"]].astype(np.float64)
    dd = ((Pq[0][None] - wrong[res["ids"][0]]) ** 2).sum(1)
    assert not np.allclose(dd, res["dist"][0], rtol=1e-5, atol=1e-7)


def test_full_rerank_equals_exact_ivf():
    """Reranking every ADC candidate with the exact d_s distance gives the
    plain IVF result (Sec. 4.3 shortlist-rerank)."""
    data = synthdata.small(1000, 10, 32, 8, 35)
    db, q = data["db"], data["queries"]
    idx = oracle.build_ivf(db, 8, 6, 3, 1000, seed=7)
    opq = oracle.train_opq(db, 32, 4, 2, 2, 2, 1000, seed=8)
    codes = oracle.pq_encode(db, 32, 4, opq["R"], opq["codebooks"])
    a = oracle.search_ivfopq(db, idx, opq, codes, q, 8, 3, 10, rerank_k=1000)
    b = oracle.search_ivf(db, idx, q, 8, 32, 3, 10)
    assert np.array_equal(a["ids"], b["ids"]) and np.allclose(a["dist"], b["dist"], atol=1e-14)


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_a_dropped_term():
    """A plausible slip (dropping the last coordinate of the scan) must fail the
    brute-force pin: the pin is sensitive to the scan's index range."""
    data = synthdata.small(600, 10, 16, 4, 36)
    idx = oracle.build_ivf(data["db"], 8, 4, 3, 600, seed=2)
    bi, bd = brute_force(data["db"], data["queries"], 16, 10, PN)
    bad = oracle.search_ivf(data["db"], idx, data["queries"], 8, 15, 4, 10)   # d_s - 1
    assert not np.allclose(bad["dist"], bd, rtol=1e-9, atol=1e-9)


def test_cost_model_reading():
    c = oracle.mflops_per_query(64, 2048, 1024, 1, 1_281_167)
    assert abs(c["mflops"] - (64 * 1024 + 2048 * 1_281_167 / 1024) / 1e6) < 1e-12
