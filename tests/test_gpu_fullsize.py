"""Oracle parity at the full ImageNet-shaped size, in the benchmark's launch configuration.

The database is the full 1,281,167 x 2048 synthetic stand-in and every search
runs over the whole 50,000-query batch, exactly as the benchmark times it
(d_c = 32, d_s = 512, nprobe = 16, k = 100; BF16 tensor-core scan with an
exact rerank of 4k = 400, and the FP32 scan), plus the largest point of the
ImageNet-shaped grid (d_s = 2048, nprobe = 32).  The oracle then recomputes a
sample of 128 queries spread over the batch, one by one:

* probed lists equal the oracle's for queries with a unique probe set;
* FP32: ids and distances under the parity rule;
* BF16 + rerank: every returned distance is the exact distance of its id, and
  recall@10 against the oracle's exact IVF search.

The index is built by the oracle with two Lloyd iterations (the search does
not depend on how well the centroids converged; two keep the oracle's build
to seconds at this size).
"""
import numpy as np
import pytest

import oracle
import synthdata
from parity import ambiguous_probe_rows, check_topk, full_groups, recall, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BF16 = 2
SAMPLE = 128


@pytest.fixture(scope="module")
def A():
    import paper_2305_19435_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    return P


@pytest.fixture(scope="module")
def full(A):
    data = synthdata.make("imagenet")
    N, nlist = data["db"].shape[0], 1024
    o = oracle.build_ivf(data["db"], 32, nlist, 2, min(N, 256 * nlist), seed=42)
    db = torch.from_numpy(data["db"]).cuda()
    g = A.index_create(db, torch.from_numpy(o["centroids"]).cuda(),
                       torch.from_numpy(o["assign"].astype(np.int32)).cuda(),
                       storage=1 | BF16)
    del db
    torch.cuda.empty_cache()
    q = torch.from_numpy(data["queries"]).cuda()
    rows = np.linspace(0, q.shape[0] - 1, SAMPLE).astype(np.int64)
    yield data, o, g, q, rows
    g.status()
    g.free()


def exact_dist(db, q, ids, d_s):
    out = np.full(ids.shape, np.inf)
    ok = ids >= 0
    P = oracle.prefix(q[None], d_s)[0]
    X = oracle.prefix(db[ids[ok]], d_s)
    out[ok] = ((X - P) ** 2).sum(1)
    return out


@pytest.mark.parametrize("d_s,nprobe", [(512, 16), (2048, 32)])
def test_fp32_full_batch(A, full, d_s, nprobe):
    data, o, g, q, rows = full
    k = 100
    gi, gd, gp = A.search_ivf(g, q, 32, d_s, nprobe, k, return_probes=True)
    gi, gd, gp = gi[rows].cpu().numpy(), gd[rows].cpu().numpy(), gp[rows].cpu().numpy()
    qs = data["queries"][rows]
    ref = full_groups(oracle.search_ivf(data["db"], o, qs, 32, d_s, nprobe, k + 24),
                      lambda r, kk: oracle.search_ivf(data["db"], o, qs[r], 32, d_s, nprobe, kk),
                      k)
    amb = ambiguous_probe_rows(ref["probe_dist"], nprobe)
    for i in np.nonzero(~amb)[0]:
        assert set(gp[i]) == set(ref["probes"][i]), i
    n, fails = check_topk(gi, gd, ref["ids"], ref["dist"], k, skip_rows=amb)
    assert n > SAMPLE - 8 and not fails, f"{len(fails)}/{n} queries differ, e.g. {fails[:2]}"


@pytest.mark.parametrize("d_s,nprobe", [(512, 16), (2048, 32)])
def test_bf16_rerank_full_batch(A, full, d_s, nprobe):
    data, o, g, q, rows = full
    k = 100
    gi, gd = A.search_ivf(g, q, 32, d_s, nprobe, k, storage=BF16, rerank_k=4 * k)
    g.status()
    gi, gd = gi[rows].cpu().numpy(), gd[rows].cpu().numpy()
    qs = data["queries"][rows]
    for i in range(len(rows)):
        ex = exact_dist(data["db"], qs[i], gi[i], d_s)
        assert np.isfinite(ex).all(), i
        assert np.all(np.abs(gd[i] - ex) <= tol(ex)), i
        assert np.all(np.diff(gd[i]) >= 0) and len(set(gi[i].tolist())) == k, i
    ref = oracle.search_ivf(data["db"], o, qs, 32, d_s, nprobe, k)
    assert recall(gi, ref["ids"], 10) >= 0.995
