"""Mixed-precision AdANNS-IVF (BF16 / FP8-E4M3 storage, tensor-core scan,
exact FP32 rerank of the k' shortlist) against the FP64 oracle.

The approximate scan only chooses the shortlist; every returned distance is
the exact FP32 d_s distance, so each (id, distance) pair must match the
oracle's exact distance for that id, and the ids must reach the stated
recall@10 against the oracle's exact IVF search on the same index.
"""
import numpy as np
import pytest

import oracle
import synthdata
from parity import recall, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PN = oracle.METRIC_L2_PREFIXNORM
BF16, FP8 = 2, 4


@pytest.fixture(scope="module")
def A():
    import paper_2305_19435_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    return P


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def case(A):
    data = synthdata.small(40_000, 700, 256, 64, 401)
    o = oracle.build_ivf(data["db"], 32, 48, 8, 20_000, seed=21)
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                       storage=1 | BF16 | FP8)
    yield data, o, g
    g.free()


def exact_dist(db, q, ids, d_s):
    """dist_ds of each returned id (FP64, the definition), +inf for padding."""
    P = oracle.prefix(q[None], d_s)[0]
    out = np.full(ids.shape, np.inf)
    ok = ids >= 0
    X = oracle.prefix(db[ids[ok]], d_s)
    out[ok] = ((X - P) ** 2).sum(1)
    return out


def check(A, case, storage, d_s, nprobe, k, kr, min_recall, B=None, d_c=32):
    data, o, g = case
    q = data["queries"] if B is None else data["queries"][:B]
    gi, gd = A.search_ivf(g, cu(q), d_c, d_s, nprobe, k, storage=storage, rerank_k=kr)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    ref = oracle.search_ivf(data["db"], o, q, d_c, d_s, nprobe, k)
    # every returned distance is the exact distance of the returned id
    for i in range(len(q)):
        ex = exact_dist(data["db"], q[i], gi[i], d_s)
        fin = np.isfinite(ex)
        assert np.all(np.abs(gd[i][fin] - ex[fin]) <= tol(ex[fin])), i
        assert np.all(np.diff(gd[i][fin]) >= 0)
        assert len(set(gi[i][gi[i] >= 0].tolist())) == int((gi[i] >= 0).sum())
    r = recall(gi, ref["ids"], min(10, k))
    assert r >= min_recall, r
    return r


@pytest.mark.parametrize("storage", [BF16, FP8])
def test_mixed_main_point(A, case, storage):
    """d_s = 256, nprobe = 8, k = 100, shortlist 4k = 400."""
    check(A, case, storage, 256, 8, 100, 400, 0.995 if storage == BF16 else 0.99)


@pytest.mark.parametrize("d_s,nprobe,k,kr", [(64, 4, 10, 40), (96, 6, 10, 40), (128, 12, 50, 200),
                                             (192, 2, 1, 4), (256, 48, 20, 80)])
def test_mixed_bf16_sweep(A, case, d_s, nprobe, k, kr):
    check(A, case, BF16, d_s, nprobe, k, kr, 0.98)


@pytest.mark.parametrize("d_s", [128, 256])
def test_mixed_fp8_sweep(A, case, d_s):
    check(A, case, FP8, d_s, 8, 10, 40, 0.97)


@pytest.mark.parametrize("storage", [BF16, FP8])
def test_mixed_largest_k_and_shortlist(A, case, storage):
    """k = 1024 with the largest shortlist, k' = 2048: the selection takes its
    exact path over the whole region (k' above its buffer) and the final sort
    its shared-memory path (more than 256 keys)."""
    check(A, case, storage, 256, 16, 1024, 2048, 0.99, B=100)


@pytest.mark.parametrize("B", [1, 3, 129])
def test_mixed_ragged_batches(A, case, B):
    check(A, case, BF16, 256, 8, 10, 40, 0.95, B=B)


def test_full_shortlist_is_exact(A, case):
    """When the shortlist holds every candidate, the result equals the exact scan."""
    data, o, g = case
    from parity import ambiguous_probe_rows, check_topk
    sizes = np.diff(o["list_off"])
    ref = oracle.search_ivf(data["db"], o, data["queries"], 32, 128, 1, 60)
    fits = sizes[ref["probes"][:, 0]] <= 2048
    q = data["queries"][fits][:64]
    ref = {key: v[fits][:64] for key, v in ref.items()}
    gi, gd = A.search_ivf(g, cu(q), 32, 128, 1, 20, storage=BF16, rerank_k=2048)
    amb = ambiguous_probe_rows(ref["probe_dist"], 1)
    n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), ref["ids"], ref["dist"], 20,
                          skip_rows=amb)
    assert n > 0 and not fails, fails[:2]


def test_mixed_errors(A, case):
    data, o, g = case
    q = cu(data["queries"][:4])
    with pytest.raises(A.AdannsError) as e:
        A.search_ivf(g, q, 32, 256, 8, 10, storage=BF16, rerank_k=5)    # shortlist < k
    assert e.value.code == -1
    h = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)))
    with pytest.raises(A.AdannsError) as e:
        A.search_ivf(h, q, 32, 256, 8, 10, storage=BF16, rerank_k=40)    # tier not built
    assert e.value.code == -6
    h.free()


@pytest.mark.parametrize("storage,d_c", [(BF16, 8), (FP8, 16)])
def test_mixed_ivf_d(A, case, storage, d_c):
    """IVF-D on the tensor-core path: the d_c = 32 lists probed at a smaller prefix."""
    check(A, case, storage, 128, 6, 10, 40, 0.99, d_c=d_c)


@pytest.mark.parametrize("storage", [BF16, FP8])
def test_shortlist_ties_are_deterministic(A, storage):
    """Massive key ties at the shortlist cut (2,000 identical database rows,
    queries equal to them, every other row duplicated): the shortlist takes
    tied candidates in candidate order, so a query's result does not depend on
    the batch it is in or on the run, and matches the oracle under the tie rule."""
    from parity import ambiguous_probe_rows, check_topk
    data = synthdata.small(20_000, 200, 128, 32, 409)
    db = data["db"].copy()
    db[1::2] = db[0::2]
    db[5000:7000] = db[5000]
    q = data["queries"].copy()
    q[:8] = db[5000] * np.float32(1.5)
    o = oracle.build_ivf(db, 32, 24, 5, 20_000, seed=23)
    g = A.index_create(cu(db), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                       storage=1 | storage)
    args = (32, 128, 4, 10)
    full1 = A.search_ivf(g, cu(q), *args, storage=storage, rerank_k=40)[0].cpu().numpy()
    full2 = A.search_ivf(g, cu(q), *args, storage=storage, rerank_k=40)[0].cpu().numpy()
    part = A.search_ivf(g, cu(q[3:90]), *args, storage=storage, rerank_k=40)[0].cpu().numpy()
    assert np.array_equal(full1, full2)
    assert np.array_equal(part, full1[3:90])
    gi, gd = A.search_ivf(g, cu(q[:8]), *args, storage=storage, rerank_k=40)
    ref = oracle.search_ivf(db, o, q[:8], 32, 128, 4, 20_000)   # every candidate: whole tie group
    amb = ambiguous_probe_rows(ref["probe_dist"], 4)
    n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), ref["ids"], ref["dist"], 10,
                          skip_rows=amb)
    assert not fails, fails[:2]
    g.free()


@pytest.mark.parametrize("kr", [40, 200])
def test_shortlist_ties_inside_the_survivor_buffer(A, kr):
    """300 identical rows (one list), queries equal to them: the shortlist cut
    falls inside a group of 300 equal keys that all fit the survivor buffer
    (more than its 128-entry tie sort), so the ties are ranked by a radix select
    on their candidate positions.  The smallest positions are the smallest ids
    of the group, so the result is the exact FP32 search's, run after run."""
    data = synthdata.small(20_000, 64, 128, 32, 411)
    db = data["db"].copy()
    db[8000:8300] = db[8000]
    q = np.repeat(db[8000:8001] * np.float32(1.25), 16, axis=0)
    o = oracle.build_ivf(db, 32, 24, 5, 20_000, seed=29)
    g = A.index_create(cu(db), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                       storage=1 | BF16)
    args = (32, 128, 4, 10)
    i1, d1 = A.search_ivf(g, cu(q), *args, storage=BF16, rerank_k=kr)
    i2, _ = A.search_ivf(g, cu(q), *args, storage=BF16, rerank_k=kr)
    ie, de = A.search_ivf(g, cu(q), *args)                       # exact FP32 scan
    assert torch.equal(i1, i2)
    assert torch.equal(i1, ie)
    assert np.array_equal(i1[0].cpu().numpy(), np.arange(8000, 8010))
    g.free()


@pytest.mark.parametrize("storage,d_s,nprobe,k,kr", [(BF16, 256, 8, 100, 400), (BF16, 128, 12, 10, 40),
                                                    (BF16, 64, 4, 1, 2048), (FP8, 256, 8, 100, 400),
                                                    (FP8, 128, 6, 10, 40)])
def test_certified_pruning_changes_nothing(A, case, storage, d_s, nprobe, k, kr):
    """The shortlist candidates dropped before the exact rerank (quantisation
    residual bound) cannot reach the top-k: results with and without the
    pruning are bit-identical, and the pruning does drop candidates (BF16)."""
    data, o, g = case
    q = cu(data["queries"])
    with A.option(A.OPT_RERANK_PRUNE, 0):
        i0, d0 = A.search_ivf(g, q, 32, d_s, nprobe, k, storage=storage, rerank_k=kr)
    A.profile_enable(True)
    with A.option(A.OPT_RERANK_PRUNE, 1):
        i1, d1 = A.search_ivf(g, q, 32, d_s, nprobe, k, storage=storage, rerank_k=kr)
    cnt = A.profile_read_counters()
    A.profile_enable(False)
    assert torch.equal(i0, i1)
    assert torch.equal(d0, d1)
    assert cnt["shortlist_slots"] == q.shape[0] * kr
    assert k * q.shape[0] <= cnt["rerank_pairs"] <= cnt["shortlist_slots"]
    if storage == BF16 and kr >= 4 * k:
        assert cnt["rerank_pairs"] < cnt["shortlist_slots"]


def test_status_clean_after_mixed_searches(A, case):
    """No device-side consistency check or pipeline wait fired in this module."""
    data, o, g = case
    A.search_ivf(g, cu(data["queries"]), 32, 256, 8, 100, storage=BF16, rerank_k=400)
    g.status()


def _candidates(A, g, q, d_c, nprobe):
    """Total members of every query's probed lists (the unfiltered scan's keys)."""
    _, _, pr = A.search_ivf(g, q, d_c, 64, nprobe, 1, return_probes=True)
    off, _ = g.lists()
    sizes = (off[1:] - off[:-1]).cpu().numpy()
    return int(sizes[pr.cpu().numpy()].sum())


@pytest.mark.parametrize("storage,d_s,nprobe,k,kr", [(BF16, 256, 8, 100, 400), (BF16, 128, 1, 10, 40),
                                                    (BF16, 64, 12, 50, 2048), (FP8, 256, 8, 100, 400),
                                                    (FP8, 96, 3, 1, 4), (BF16, 256, 48, 20, 80),
                                                    (BF16, 192, 2, 7, 1000)])
def test_filtered_scan_equals_unfiltered(A, case, storage, d_s, nprobe, k, kr):
    """The filtered tensor-core scan keeps, outside each query's nearest list,
    only members whose key is at most the kk-th key of that list (a bound on the
    query's kk-th key), and selects the shortlist from them with the same
    (key, candidate position) order: ids and distance bits equal those of the
    scan that writes every key, and for a selective shortlist far fewer
    candidates reach the selection."""
    data, o, g = case
    q = cu(data["queries"])
    with A.option(A.OPT_SCAN_FILTER, 0):
        i0, d0 = A.search_ivf(g, q, 32, d_s, nprobe, k, storage=storage, rerank_k=kr)
    A.profile_enable(True)
    with A.option(A.OPT_SCAN_FILTER, 1):
        i1, d1 = A.search_ivf(g, q, 32, d_s, nprobe, k, storage=storage, rerank_k=kr)
    cnt = A.profile_read_counters()
    A.profile_enable(False)
    g.status()
    assert torch.equal(i0, i1)
    assert torch.equal(d0.view(torch.int32), d1.view(torch.int32))
    total = _candidates(A, g, q, 32, nprobe)
    assert 0 < cnt["scan_survivors"] <= total
    if nprobe >= 8 and kr <= 400:
        assert cnt["scan_survivors"] < 0.6 * total, (cnt, total)


@pytest.mark.parametrize("kr", [40, 400])
def test_filtered_scan_ties_at_the_bound(A, kr):
    """Every other database row duplicated and a block of 2,000 identical rows,
    queries equal to them: many keys equal the bound taken from the nearest
    list; all of them are kept, so the result is the unfiltered scan's."""
    data = synthdata.small(20_000, 200, 128, 32, 413)
    db = data["db"].copy()
    db[1::2] = db[0::2]
    db[5000:7000] = db[5000]
    q = data["queries"].copy()
    q[:8] = db[5000] * np.float32(1.5)
    o = oracle.build_ivf(db, 32, 24, 5, 20_000, seed=31)
    g = A.index_create(cu(db), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                       storage=1 | BF16 | FP8)
    for storage in (BF16, FP8):
        with A.option(A.OPT_SCAN_FILTER, 0):
            i0, d0 = A.search_ivf(g, cu(q), 32, 128, 6, 10, storage=storage, rerank_k=kr)
        with A.option(A.OPT_SCAN_FILTER, 1):
            i1, d1 = A.search_ivf(g, cu(q), 32, 128, 6, 10, storage=storage, rerank_k=kr)
        assert torch.equal(i0, i1)
        assert torch.equal(d0.view(torch.int32), d1.view(torch.int32))
    g.status()
    g.free()
