"""GPU-vs-oracle parity for AdANNS-IVF: index layout, k-means steps, search.

Every expected value comes from the FP64 oracle on the same seeded inputs.
Search parity runs on the oracle's own index (its FP32 centroids and list
assignment imported through adanns_index_create), so the scan and the
cluster mapping are compared on identical lists.
"""
import numpy as np
import pytest

import oracle
import synthdata
from parity import ambiguous_probe_rows, check_topk, full_groups, recall, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PN, L2 = oracle.METRIC_L2_PREFIXNORM, oracle.METRIC_L2


@pytest.fixture(scope="module")
def A():
    import paper_2305_19435_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    return P


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def import_index(A, db, oidx, metric):
    return A.index_create(cu(db), cu(oidx["centroids"]), cu(oidx["assign"].astype(np.int32)),
                          metric=metric)


def search_parity(A, db, q, oidx, d_c, d_s, nprobe, k, metric, extra=24):
    gidx = import_index(A, db, oidx, metric)
    gi, gd, gp = A.search_ivf(gidx, cu(q), d_c, d_s, nprobe, k, return_probes=True)
    torch.cuda.synchronize()
    gi, gd, gp = gi.cpu().numpy(), gd.cpu().numpy(), gp.cpu().numpy()
    o = full_groups(oracle.search_ivf(db, oidx, q, d_c, d_s, nprobe, k + extra, metric=metric),
                    lambda rows, kk: oracle.search_ivf(db, oidx, q[rows], d_c, d_s, nprobe, kk,
                                                       metric=metric), k)
    scale, scale_c = None, 1.0
    if metric == L2:
        scale = (q[:, :d_s].astype(np.float64) ** 2).sum(1)
        scale_c = (q[:, :d_c].astype(np.float64) ** 2).sum(1)
    amb = ambiguous_probe_rows(o["probe_dist"], nprobe, scale_c)
    # probe lists of unambiguous queries match exactly (as sets; order by distance)
    for i in np.nonzero(~amb)[0]:
        assert set(gp[i]) == set(o["probes"][i]), i
    n, fails = check_topk(gi, gd, o["ids"], o["dist"], k, skip_rows=amb, scale=scale)
    assert n > 0
    assert not fails, f"{len(fails)}/{n} queries differ, e.g. {fails[:2]}"
    gidx.free()
    return gi, gd, o, amb


# ---------------------------------------------------------------- index layout
def test_index_lists_match_oracle_csr(A):
    data = synthdata.small(5000, 1, 64, 32, 101)
    o = oracle.build_ivf(data["db"], 16, 40, 5, 5000, seed=3)
    g = import_index(A, data["db"], o, PN)
    off, ids = g.lists()
    assert np.array_equal(off.cpu().numpy(), o["list_off"])
    assert np.array_equal(ids.cpu().numpy(), o["list_ids"])
    assert np.array_equal(g.centroids().cpu().numpy(), o["centroids"])


def test_empty_lists_and_tiny_lists(A):
    data = synthdata.small(700, 30, 32, 8, 102)
    db, q = data["db"], data["queries"]
    o = oracle.build_ivf(db, 16, 12, 4, 700, seed=4)
    # force two empty lists and one single-member list
    a = o["assign"].copy()
    a[a == 3] = 4
    a[a == 7] = 8
    a[5] = 7
    o = dict(o)
    o["assign"] = a
    o["list_off"], o["list_ids"] = oracle.lists_from_assignment(a, 12)
    search_parity(A, db, q, o, 16, 32, 12, 20, PN)
    search_parity(A, db, q, o, 16, 32, 3, 7, PN)


# ---------------------------------------------------------------- search parity
def tiny_workload():
    w = synthdata.WORKLOADS["tiny"]
    return synthdata.make(w)


@pytest.fixture(scope="module")
def tiny():
    data = tiny_workload()
    o = oracle.build_ivf(data["db"], 16, 64, 20, 10_000, seed=42)
    return data, o


def test_tiny_config_full_parity(A, tiny):
    """Tiny AdANNS-IVF: 10k x 64, nlist 64 at d_c=16, nprobe 4, d_s 64, k 10."""
    data, o = tiny
    gi, gd, orr, amb = search_parity(A, data["db"], data["queries"], o, 16, 64, 4, 10, PN)
    assert recall(gi, orr["ids"], 10) > 0.999
    assert amb.mean() < 0.05


@pytest.mark.parametrize("d_s,nprobe,k", [(8, 1, 1), (16, 2, 5), (32, 4, 10), (48, 8, 33),
                                          (64, 16, 100), (64, 64, 128), (64, 3, 300)])
def test_tiny_sweep(A, tiny, d_s, nprobe, k):
    data, o = tiny
    search_parity(A, data["db"], data["queries"], o, 16, d_s, nprobe, k, PN)


def test_full_probe_full_dim_is_exact_search(A, tiny):
    """n_p = nlist, d_s = d: the GPU result is exact kNN (via the oracle pin)."""
    data, o = tiny
    search_parity(A, data["db"], data["queries"][:50], o, 16, 64, 64, 50, PN)


@pytest.mark.parametrize("B", [60, 200])
def test_largest_k(A, tiny, B):
    """k = 1024, the largest allowed: 60 queries take the streaming scan (15
    queries per probed list), 200 the tiled scan."""
    data, o = tiny
    search_parity(A, data["db"], data["queries"][:B], o, 16, 64, 16, 1024, PN)


def test_raw_l2_metric(A):
    data = synthdata.small(4000, 64, 64, 16, 103)
    o = oracle.build_ivf(data["db"], 32, 30, 6, 4000, seed=5, metric=L2)
    search_parity(A, data["db"], data["queries"], o, 32, 64, 5, 20, L2)


def test_duplicates_zero_vectors_and_exact_matches(A):
    data = synthdata.small(3000, 40, 64, 16, 104)
    db, q = data["db"].copy(), data["queries"].copy()
    db[100:140] = db[7]            # a block of duplicates: an exact tie group
    db[200] = 0.0                  # zero vector
    q[0] = db[7]                   # query equal to a duplicated vector
    q[1] = db[300] * 3.0           # same direction: distance 0 after normalisation
    q[2] = 0.0                     # zero query
    o = oracle.build_ivf(db, 16, 20, 5, 3000, seed=6)
    gi, gd, orr, amb = search_parity(A, db, q, o, 16, 64, 20, 60, PN)
    assert set(gi[0, :41].tolist()) == {7, *range(100, 140)}
    assert gi[1, 0] == 300


@pytest.mark.parametrize("B", [1, 17, 63, 64, 65, 129])
def test_ragged_batches(A, tiny, B):
    data, o = tiny
    search_parity(A, data["db"], data["queries"][:B], o, 16, 32, 4, 10, PN)


def test_many_tiles_wider_vectors(A):
    """Lists long enough for many member chunks and queries for many tiles."""
    data = synthdata.small(60_000, 600, 256, 64, 105)
    o = oracle.build_ivf(data["db"], 32, 48, 8, 20_000, seed=7)
    search_parity(A, data["db"], data["queries"], o, 32, 256, 6, 100, PN)
    search_parity(A, data["db"], data["queries"][:200], o, 32, 96, 12, 10, PN)


def test_argument_errors(A, tiny):
    data, o = tiny
    g = import_index(A, data["db"], o, PN)
    qq = cu(data["queries"][:4])
    with pytest.raises(A.AdannsError) as e:
        A.search_ivf(g, qq, 16, 40, 4, 10)          # d_s not in G
    assert e.value.code == -2
    with pytest.raises(A.AdannsError) as e:
        A.search_ivf(g, qq, 16, 128, 4, 10)         # d_s beyond d
    assert e.value.code == -2
    with pytest.raises(A.AdannsError) as e:
        A.search_ivf(g, qq, 16, 64, 65, 10)         # nprobe > nlist
    assert e.value.code == -1
    with pytest.raises(A.AdannsError) as e:
        A.search_ivf(g, qq, 16, 64, 4, 1025)        # k too large
    assert e.value.code == -1
    with pytest.raises(A.AdannsError) as e:
        A.search_ivf(g, qq, 32, 64, 4, 10)          # d_c above the built prefix
    assert e.value.code == -2
    with pytest.raises(A.AdannsError) as e:
        A.search_ivf(g, qq, 12, 64, 4, 10)          # d_c not in G
    assert e.value.code == -2
    ids, dist = A.search_ivf(g, cu(data["queries"][:0]), 16, 64, 4, 10)
    assert ids.shape == (0, 10)
    g.free()


# ---------------------------------------------------------------- IVF-D
@pytest.mark.parametrize("d_hat,d_s,nprobe,metric", [(8, 64, 5, PN), (16, 128, 3, PN),
                                                     (32, 32, 8, PN), (64, 96, 4, PN),
                                                     (16, 96, 5, L2)])
def test_ivf_d_probes_with_a_prefix_of_the_built_centroids(A, d_hat, d_s, nprobe, metric):
    """AdANNS-IVF-D (Table "formula" IVF-D row): lists built at d_c = 64,
    probed at d_hat <= 64 with the stored centroids' first d_hat coordinates."""
    data = synthdata.small(12_000, 250, 128, 40, 131)
    o = oracle.build_ivf(data["db"], 64, 48, 5, 12_000, seed=13, metric=metric)
    search_parity(A, data["db"], data["queries"], o, d_hat, d_s, nprobe, 20, metric)


# ---------------------------------------------------------------- k-means steps
def teacher_forced_case(seed=106, n=6000, d=64, d_c=32, nc=50):
    data = synthdata.small(n, 1, d, 24, seed)
    x = data["db"]
    T = oracle.prefix(x, d_c)
    init = oracle.sample(seed, n, nc)
    C0 = T[init].astype(np.float32)
    return x, T, C0


@pytest.mark.parametrize("nc,d_c", [(50, 32), (300, 32), (1024, 64), (256, 16)])
def test_kmeans_assign_step_matches_oracle(A, nc, d_c):
    """From 256 centroids up (d_c <= 64) the assignment runs on the tensor cores
    (BF16 products, exact FP32 re-score within the error bound)."""
    x, T, C0 = teacher_forced_case(d_c=d_c, nc=nc)
    a, dist = A.kmeans_assign(cu(x), cu(C0), d_c)
    a, dist = a.cpu().numpy(), dist.cpu().numpy()
    oa, ob, os2 = oracle.assign(T, C0.astype(np.float64))
    tied = os2 - ob <= tol(os2)
    assert tied.mean() < 0.01
    assert np.array_equal(a[~tied], oa[~tied])
    assert np.all(np.abs(dist - ob) <= tol(ob))


def test_kmeans_update_step_matches_oracle(A):
    x, T, C0 = teacher_forced_case(seed=107)
    oa, _, _ = oracle.assign(T, C0.astype(np.float64))
    want = oracle.update(T, oa, C0.astype(np.float64))
    got = A.kmeans_update(cu(x), cu(oa.astype(np.int32)), cu(C0.copy()), 32).cpu().numpy()
    # FP32 normalised inputs summed in FP64: within FP32 rounding of the mean,
    # plus the normalisation rounding (2^-24 relative per coordinate)
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 1e-7)
    # empty clusters keep their centroid
    nc = C0.shape[0]
    a2 = np.zeros(len(x), dtype=np.int32)
    got2 = A.kmeans_update(cu(x), cu(a2), cu(C0.copy()), 32).cpu().numpy()
    assert np.array_equal(got2[1:], C0[1:])


def test_build_ivf_free_running_objective(A, tiny):
    data, o = tiny
    g = A.build_ivf(cu(data["db"]), 16, 64, 20, 10_000, 42)
    Jg, Jo = np.array(g.objective), np.array(o["objectives"])
    assert abs(Jg[0] - Jo[0]) <= 1e-5 * Jo[0]       # same sample, same init
    assert abs(Jg[-1] - Jo[-1]) <= 1e-4 * Jo[-1]
    assert np.all(Jg[1:] <= Jg[:-1] * (1 + 1e-6))
    off, ids = g.lists()
    off, ids = off.cpu().numpy(), ids.cpu().numpy()
    assert off[-1] == 10_000 and sorted(ids.tolist()) == list(range(10_000))
    # the GPU's final assignment is the nearest of its own centroids (a
    # property, checked with a plain FP64 distance table, not the oracle)
    C = g.centroids().cpu().numpy().astype(np.float64)
    X = oracle.prefix(data["db"], 16)
    D = ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    srt = np.sort(D, axis=1)
    oa, ob, os2 = np.argmin(D, axis=1), srt[:, 0], srt[:, 1]
    lab = np.empty(10_000, dtype=np.int64)
    for l in range(64):
        lab[ids[off[l]:off[l + 1]]] = l
    tied = os2 - ob <= tol(os2)
    assert np.array_equal(lab[~tied], oa[~tied])
    g.free()


def test_build_ivf_tensor_core_assignment_objective(A):
    """A build with 256 lists (assignment on the tensor cores): the same sample
    and initialisation as the oracle's give the same first objective, the
    free-running trace stays within 1e-4 and never increases."""
    data = synthdata.small(30_000, 1, 64, 300, 117)
    o = oracle.build_ivf(data["db"], 32, 256, 8, 30_000, seed=7)
    g = A.build_ivf(cu(data["db"]), 32, 256, 8, 30_000, 7)
    Jg, Jo = np.array(g.objective), np.array(o["objectives"])
    assert abs(Jg[0] - Jo[0]) <= 1e-5 * Jo[0]
    assert abs(Jg[-1] - Jo[-1]) <= 1e-4 * Jo[-1]
    assert np.all(Jg[1:] <= Jg[:-1] * (1 + 1e-6))
    g.status()
    g.free()


def test_gpu_built_index_search_recall(A, tiny):
    """The GPU-built index, searched on the GPU, agrees with the oracle's index
    searched by the oracle at recall@10 >= 0.95 (builds may diverge only at
    near-ties of the Lloyd trajectory)."""
    data, o = tiny
    g = A.build_ivf(cu(data["db"]), 16, 64, 20, 10_000, 42)
    gi, gd = A.search_ivf(g, cu(data["queries"]), 16, 64, 4, 10)
    orr = oracle.search_ivf(data["db"], o, data["queries"], 16, 64, 4, 10)
    assert recall(gi.cpu().numpy(), orr["ids"], 10) >= 0.95
    g.free()


# ---------------------------------------------------------------- tensor-core cluster mapping
@pytest.fixture(scope="module")
def wide(A):
    """An index with enough lists (320) for the tensor-core cluster mapping."""
    data = synthdata.small(60_000, 500, 128, 96, 151)
    o = oracle.build_ivf(data["db"], 64, 320, 4, 30_000, seed=17)
    return data, o


@pytest.mark.parametrize("d_c,nprobe", [(64, 1), (64, 16), (32, 32), (16, 8), (64, 33),
                                         (64, 100), (32, 300), (16, 64)])
def test_tensor_core_cluster_mapping_is_exact(A, wide, d_c, nprobe):
    """BF16 tensor-core shortlist + exact FP32 re-score of every centroid within
    the quantisation bound: the same probes and results as the FP32 cluster
    mapping (d_c < 64 is IVF-D on the d_c = 64 index), and oracle parity.
    n_p <= 32 picks with one warp per query, larger n_p with one CTA."""
    data, o = wide
    g = import_index(A, data["db"], o, PN)
    q = cu(data["queries"])
    with A.option(A.OPT_COARSE_TC, 0):
        i0, d0, p0 = A.search_ivf(g, q, d_c, 128, nprobe, 20, return_probes=True)
    with A.option(A.OPT_COARSE_TC, 1):
        i1, d1, p1 = A.search_ivf(g, q, d_c, 128, nprobe, 20, return_probes=True)
    assert torch.equal(p0, p1)
    assert torch.equal(i0, i1) and torch.equal(d0, d1)
    g.status()
    g.free()
    search_parity(A, data["db"], data["queries"], o, d_c, 128, nprobe, 20, PN)


@pytest.mark.parametrize("B,d_s,nprobe,k", [(40, 8, 1, 1), (100, 48, 4, 10), (500, 128, 1, 100),
                                            (300, 96, 8, 33), (17, 128, 33, 50), (3, 16, 2, 5)])
def test_fp32_stream_scan_equals_tiled_scan(A, wide, B, d_s, nprobe, k):
    """Few queries per probed list: the streaming scan (register accumulation,
    distances written, then a per-query select) and the shared-memory tiled
    scan compute the same FP32 distances and keep the same (distance, id)
    top-k, bit for bit; d_s = 8 and 48 end in a partial 16-coordinate block."""
    data, o = wide
    g = import_index(A, data["db"], o, PN)
    q = cu(data["queries"][:B])
    i0, d0, p0 = A.search_ivf(g, q, 64, d_s, nprobe, k, return_probes=True)
    with A.option(A.OPT_FP32_STREAM, 0):
        i1, d1, p1 = A.search_ivf(g, q, 64, d_s, nprobe, k, return_probes=True)
    assert torch.equal(p0, p1)
    assert torch.equal(i0, i1)
    assert torch.equal(d0.view(torch.int32), d1.view(torch.int32))
    g.free()
