"""GPU-vs-oracle parity at the ImageNet-shaped prefix lengths (d = 2048).

The benchmark scans d_s = 512 and up to 2048 coordinates; the smaller parity
cases stop at d = 256.  This module runs every search kernel at the long
prefixes on a 60,000 x 2048 database (256 lists built by the oracle at
d_c = 64, one of them empty) with 256 queries:

* the FP32 streaming and tiled scans, element by element under the parity
  rule, at d_s = 512 and 2048 (the tiled scan through ADANNS_OPT_FP32_STREAM);
* the BF16 / FP8 tensor-core scans (8, 16 and 32 K-blocks) with the exact
  rerank at d_s = 512, 1024 and 2048: every returned distance is the exact
  dist_ds of the returned id, and recall@10 against the oracle's exact IVF
  search; with a shortlist that holds every candidate the result must equal
  the oracle's top-k element by element (this is the rerank's own parity);
* the tensor-core cluster mapping at d_c = 64 (and IVF-D at d_c = 32 and 16):
  the probed lists equal the oracle's for every query whose probe set is
  unique.
"""
import numpy as np
import pytest

import oracle
import synthdata
from parity import ambiguous_probe_rows, check_topk, full_groups, recall, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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
def wide(A):
    data = synthdata.small(60_000, 256, 2048, 120, 515)
    o = oracle.build_ivf(data["db"], 64, 256, 8, 60_000, seed=9)
    assert (np.diff(o["list_off"]) == 0).any()   # an empty list is part of the case
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                       storage=1 | BF16 | FP8)
    yield data, o, g
    g.status()
    g.free()


def oracle_topk(data, o, q, d_c, d_s, nprobe, k):
    return full_groups(oracle.search_ivf(data["db"], o, q, d_c, d_s, nprobe, k + 24),
                       lambda rows, kk: oracle.search_ivf(data["db"], o, q[rows], d_c, d_s,
                                                          nprobe, kk), k)


def exact_dist(db, q, ids, d_s):
    """dist_ds of each returned id (FP64, the definition), +inf for padding."""
    out = np.full(ids.shape, np.inf)
    ok = ids >= 0
    P = oracle.prefix(q[None], d_s)[0]
    X = oracle.prefix(db[ids[ok]], d_s)
    out[ok] = ((X - P) ** 2).sum(1)
    return out


@pytest.mark.parametrize("stream", [1, 0])
@pytest.mark.parametrize("d_s", [512, 2048])
def test_fp32_scans_long_prefix(A, wide, d_s, stream):
    data, o, g = wide
    q = data["queries"]
    nprobe, k = 8, 50
    with A.option(A.OPT_FP32_STREAM, stream):
        gi, gd, gp = A.search_ivf(g, cu(q), 64, d_s, nprobe, k, return_probes=True)
    gi, gd, gp = gi.cpu().numpy(), gd.cpu().numpy(), gp.cpu().numpy()
    ref = oracle_topk(data, o, q, 64, d_s, nprobe, k)
    amb = ambiguous_probe_rows(ref["probe_dist"], nprobe)
    for i in np.nonzero(~amb)[0]:
        assert set(gp[i]) == set(ref["probes"][i]), i
    n, fails = check_topk(gi, gd, ref["ids"], ref["dist"], k, skip_rows=amb)
    assert n > 200 and not fails, f"{len(fails)}/{n} queries differ, e.g. {fails[:2]}"


@pytest.mark.parametrize("storage", [BF16, FP8])
@pytest.mark.parametrize("d_s", [512, 1024, 2048])
def test_mixed_rerank_long_prefix(A, wide, storage, d_s):
    """Shortlist of 4k = 400 of ~1,900 candidates per query, then the exact rerank."""
    data, o, g = wide
    q = data["queries"]
    nprobe, k, kr = 8, 100, 400
    gi, gd = A.search_ivf(g, cu(q), 64, d_s, nprobe, k, storage=storage, rerank_k=kr)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    for i in range(len(q)):
        ex = exact_dist(data["db"], q[i], gi[i], d_s)
        fin = np.isfinite(ex)
        assert fin.sum() == k, i
        assert np.all(np.abs(gd[i][fin] - ex[fin]) <= tol(ex[fin])), i
        assert np.all(np.diff(gd[i]) >= 0), i
        assert len(set(gi[i].tolist())) == k, i
    ref = oracle.search_ivf(data["db"], o, q, 64, d_s, nprobe, k)
    r = recall(gi, ref["ids"], 10)
    assert r >= (0.995 if storage == BF16 else 0.99), r


@pytest.mark.parametrize("storage", [BF16, FP8])
@pytest.mark.parametrize("d_s", [512, 1024, 2048])
def test_full_shortlist_equals_oracle_long_prefix(A, wide, storage, d_s):
    """nprobe = 4 gives at most ~1,700 candidates per query, so a shortlist of
    2,048 holds all of them: the exact rerank alone decides, and ids and
    distances must match the oracle's exact IVF search element by element."""
    data, o, g = wide
    q = data["queries"]
    nprobe, k = 4, 60
    ref = oracle_topk(data, o, q, 64, d_s, nprobe, k)
    assert ref["ncand"].max() <= 2048
    gi, gd = A.search_ivf(g, cu(q), 64, d_s, nprobe, k, storage=storage, rerank_k=2048)
    amb = ambiguous_probe_rows(ref["probe_dist"], nprobe)
    n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), ref["ids"], ref["dist"], k,
                          skip_rows=amb)
    assert n > 200 and not fails, f"{len(fails)}/{n} queries differ, e.g. {fails[:2]}"


@pytest.mark.parametrize("d_c,nprobe", [(64, 16), (64, 1), (32, 8), (16, 32)])
def test_tensor_core_cluster_mapping_long_index(A, wide, d_c, nprobe):
    """nlist = 256 >= the tensor-core threshold: BF16 products + certified FP32
    re-score give the FP32 kernels' probes, which equal the oracle's."""
    data, o, g = wide
    q = cu(data["queries"])
    with A.option(A.OPT_COARSE_TC, 0):
        i0, d0, p0 = A.search_ivf(g, q, d_c, 512, nprobe, 20, return_probes=True)
    with A.option(A.OPT_COARSE_TC, 1):
        i1, d1, p1 = A.search_ivf(g, q, d_c, 512, nprobe, 20, return_probes=True)
    assert torch.equal(p0, p1)
    assert torch.equal(i0, i1) and torch.equal(d0, d1)
    ref = oracle.search_ivf(data["db"], o, data["queries"], d_c, 512, nprobe, 20)
    amb = ambiguous_probe_rows(ref["probe_dist"], nprobe)
    gp = p1.cpu().numpy()
    assert (~amb).sum() > 200
    for i in np.nonzero(~amb)[0]:
        assert set(gp[i]) == set(ref["probes"][i]), i


@pytest.mark.parametrize("storage,d_s,nprobe", [(BF16, 512, 16), (FP8, 2048, 8), (BF16, 2048, 32)])
def test_filtered_scan_long_prefix(A, wide, storage, d_s, nprobe):
    """The filtered tensor-core scan (32 and 16 K-blocks) gives the unfiltered
    scan's result bit for bit at the long prefixes."""
    data, o, g = wide
    q = cu(data["queries"])
    with A.option(A.OPT_SCAN_FILTER, 0):
        i0, d0 = A.search_ivf(g, q, 64, d_s, nprobe, 100, storage=storage, rerank_k=400)
    with A.option(A.OPT_SCAN_FILTER, 1):
        i1, d1 = A.search_ivf(g, q, 64, d_s, nprobe, 100, storage=storage, rerank_k=400)
    assert torch.equal(i0, i1)
    assert torch.equal(d0.view(torch.int32), d1.view(torch.int32))
