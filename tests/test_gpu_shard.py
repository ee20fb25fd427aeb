"""Lists partitioned over G shards, emulated on one GPU (each shard its own
index; no kernel waits on another): per-shard search, id map and the merge
kernel give exactly the single-index FP32 search, and the merge kernel equals
a plain sort on random sorted rows with ties, padding and G up to 128."""
import numpy as np
import pytest

import oracle
import synthdata
from parity import ambiguous_probe_rows, check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2305_19435_gb300 as P
    P.build()
    return P


def ref_merge(ids, dist, k):
    G, B, _ = ids.shape
    oi = np.full((B, k), -1, dtype=np.int64)
    od = np.full((B, k), np.inf, dtype=np.float32)
    for q in range(B):
        a, d = ids[:, q].ravel(), dist[:, q].ravel()
        keep = a >= 0
        a, d = a[keep], d[keep]
        o = np.lexsort((a, d))[:k]
        oi[q, :len(o)], od[q, :len(o)] = a[o], d[o]
    return oi, od


@pytest.mark.parametrize("G,B,k,fill", [(2, 37, 10, 1.0), (5, 300, 100, 0.6), (33, 50, 7, 0.3),
                                        (128, 9, 64, 0.05), (1, 20, 1024, 0.5)])
def test_merge_kernel_matches_sort(P, G, B, k, fill):
    rng = np.random.default_rng(G * 1000 + k)
    ids = np.full((G, B, k), -1, dtype=np.int64)
    dist = np.full((G, B, k), np.inf, dtype=np.float32)
    perm = rng.permutation(G * k * 4)
    for s in range(G):
        for q in range(B):
            n = int(rng.binomial(k, fill))
            # coarse distances so that ties across shards are common
            d = rng.integers(0, 8, size=n).astype(np.float32) / 4
            a = perm[rng.choice(len(perm), size=n, replace=False)] + s  # may repeat across shards
            o = np.lexsort((a, d))
            ids[s, q, :n], dist[s, q, :n] = a[o], d[o]
    gi, gd = P.merge_shards(torch.from_numpy(ids).cuda(), torch.from_numpy(dist).cuda())
    ri, rd = ref_merge(ids, dist, k)
    assert np.array_equal(gi.cpu().numpy(), ri)
    assert np.array_equal(gd.cpu().numpy(), rd)


def test_map_ids(P):
    m = torch.tensor([5, 9, 11, 40], dtype=torch.int64, device="cuda")
    ids = torch.tensor([[0, 3, -1], [2, 1, 4]], dtype=torch.int64, device="cuda")
    P.map_ids(ids, m)
    assert ids.cpu().tolist() == [[5, 40, -1], [11, 9, -1]]


@pytest.fixture(scope="module")
def case():
    oracle.build()
    data = synthdata.small(30_000, 700, 128, 64, 77)
    oidx = oracle.build_ivf(data["db"], 32, 64, 6, 20_000, seed=9)
    return data, oidx


@pytest.mark.parametrize("G", [2, 3, 8])
def test_partitioned_equals_single_index(P, case, G):
    from paper_2305_19435_gb300.shard import ShardedIndex
    data, oidx = case
    d_c, d_s, nprobe, k = 32, 128, 6, 50
    q = torch.from_numpy(data["queries"]).cuda()
    one = P.index_create(torch.from_numpy(data["db"]).cuda(),
                         torch.from_numpy(oidx["centroids"]).cuda(),
                         torch.from_numpy(oidx["assign"].astype(np.int32)).cuda())
    ids1, d1 = P.search_ivf(one, q, d_c, d_s, nprobe, k)
    shards = [ShardedIndex(data["db"], oidx["centroids"], oidx["assign"], G, r) for r in range(G)]
    assert sum(s.n_rows for s in shards) == data["db"].shape[0]
    parts = [s.search_partial(q, d_c, d_s, nprobe, k) for s in shards]
    gi, gd = P.merge_shards(torch.stack([p[0] for p in parts]), torch.stack([p[1] for p in parts]))
    assert torch.equal(gi, ids1)
    assert torch.equal(gd, d1)
    # and against the oracle under the acceptance rule
    ref = oracle.search_ivf(data["db"], oidx, data["queries"], d_c, d_s, nprobe, k + 20)
    amb = ambiguous_probe_rows(ref["probe_dist"], nprobe)
    n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), ref["ids"], ref["dist"], k,
                          skip_rows=amb)
    assert n > 0 and not fails, fails[:2]
    for s in shards:
        s.free()
    one.free()


def test_partitioned_bf16_rerank_recall(P, case):
    from paper_2305_19435_gb300.shard import ShardedIndex
    data, oidx = case
    d_c, d_s, nprobe, k, G = 32, 128, 6, 10, 4
    q = torch.from_numpy(data["queries"]).cuda()
    shards = [ShardedIndex(data["db"], oidx["centroids"], oidx["assign"], G, r,
                           storage=1 | P.STORE_BF16) for r in range(G)]
    parts = [s.search_partial(q, d_c, d_s, nprobe, k, storage=P.STORE_BF16, rerank_k=4 * k)
             for s in shards]
    gi, _ = P.merge_shards(torch.stack([p[0] for p in parts]), torch.stack([p[1] for p in parts]))
    ref = oracle.search_ivf(data["db"], oidx, data["queries"], d_c, d_s, nprobe, k)
    gi = gi.cpu().numpy()
    rec = np.mean([len(set(a) & set(b)) / k for a, b in zip(gi, ref["ids"])])
    assert rec >= 0.99
    for s in shards:
        s.free()
