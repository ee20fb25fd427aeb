"""Lists partitioned over ranks, on CPU with gloo (world sizes 2 and 3): the
host side of the multi-GPU path (list partition, row selection, query
slices, the all-to-all exchange of per-rank top-k).  Each rank searches its
own lists with the FP64 oracle; after the exchange and a merge by
(distance, id) every rank's query slice equals the unpartitioned oracle
search exactly (Alg. 1 probes and scans each list independently, so the
partition cannot change a member's distance or the probed lists)."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle
import synthdata
from paper_2305_19435_gb300.shard import exchange_topk, partition_lists, query_slices, shard_rows


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def ref_merge(ids, dist, k):
    """[G, B, k] -> [B, k] by (dist, id) ascending, padding (-1, inf) last."""
    G, B, _ = ids.shape
    oi = np.full((B, k), -1, dtype=np.int64)
    od = np.full((B, k), np.inf)
    for q in range(B):
        a, d = ids[:, q].ravel(), dist[:, q].ravel()
        keep = a >= 0
        a, d = a[keep], d[keep]
        o = np.lexsort((a, d))[:k]
        oi[q, :len(o)], od[q, :len(o)] = a[o], d[o]
    return oi, od


def rank_main(rank, world, port, payload, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        db, oidx, q, (d_c, d_s, nprobe, k) = payload
        nlist = oidx["nlist"]
        owner = partition_lists(np.bincount(oidx["assign"], minlength=nlist), world)
        rows = shard_rows(oidx["assign"], owner, rank)
        off, lids = oracle.lists_from_assignment(oidx["assign"][rows], nlist)
        r = oracle.search_ivf(db[rows], dict(oidx, list_off=off, list_ids=lids), q, d_c, d_s,
                              nprobe, k, nthreads=1)
        gid = np.where(r["ids"] >= 0, rows[np.maximum(r["ids"], 0)], -1)
        ri, rd = exchange_topk(torch.from_numpy(gid), torch.from_numpy(r["dist"]), world, rank)
        mi, md = ref_merge(ri.numpy(), rd.numpy(), k)
        out.put((rank, mi, md, len(rows)))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def case():
    oracle.build()
    data = synthdata.small(6000, 41, 64, 24, 321)
    oidx = oracle.build_ivf(data["db"], 16, 24, 5, 6000, seed=5)
    return data, oidx


@pytest.mark.parametrize("world,B,nprobe,k", [(2, 41, 3, 10), (3, 41, 5, 20), (2, 1, 24, 10)])
def test_partitioned_search_equals_unpartitioned(case, world, B, nprobe, k):
    data, oidx = case
    q = data["queries"][:B]
    d_c, d_s = 16, 64
    full = oracle.search_ivf(data["db"], oidx, q, d_c, d_s, nprobe, k)
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main,
                         args=(r, world, port, (data["db"], oidx, q, (d_c, d_s, nprobe, k)), out))
             for r in range(world)]
    for p in procs:
        p.start()
    got = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert sum(g[3] for g in got) == data["db"].shape[0]      # every row on exactly one rank
    sl = query_slices(B, world)
    for rank, mi, md, _ in got:
        lo, hi = sl[rank]
        assert np.array_equal(mi, full["ids"][lo:hi])
        assert np.array_equal(md, full["dist"][lo:hi])


def test_partition_is_complete_balanced_and_deterministic():
    rng = np.random.default_rng(3)
    sizes = rng.integers(0, 500, size=300)
    for world in (1, 2, 3, 8):
        owner = partition_lists(sizes, world)
        assert owner.min() >= 0 and owner.max() < world
        load = np.bincount(owner, weights=sizes, minlength=world)
        assert load.sum() == sizes.sum()
        # longest-first greedy: no rank exceeds the lightest by more than one list
        assert load.max() - load.min() <= sizes.max()
        assert np.array_equal(owner, partition_lists(sizes, world))


def test_shard_rows_and_query_slices():
    assign = np.array([2, 0, 1, 2, 2, 0, 1])
    owner = np.array([1, 0, 1])
    assert shard_rows(assign, owner, 0).tolist() == [2, 6]
    assert shard_rows(assign, owner, 1).tolist() == [0, 1, 3, 4, 5]
    for B, world in ((10, 3), (2, 4), (0, 2), (7, 7)):
        sl = query_slices(B, world)
        assert sl[0][0] == 0 and sl[-1][1] == B
        assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
        sizes = [h - l for l, h in sl]
        assert max(sizes) - min(sizes) <= 1
