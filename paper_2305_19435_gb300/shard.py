"""AdANNS-IVF with its inverted lists partitioned over several ranks (one GPU
each).

Probing and scanning are independent per inverted list (Alg. 1; Sec. 4.2
scans only the probed lists), so the lists of one index can live on
different devices.  Every rank keeps the full centroid table, so all ranks
choose the same n_p lists for a query, and an index over the database rows of
the lists it owns.  One search then runs in three steps:

1. every rank searches the whole query batch over its own lists and maps the
   local row ids of the results to global database ids (`adanns_map_ids`);
2. the rows of query slice r (queries are split into `world` contiguous
   slices) are sent to rank r: one all-to-all of B*k (id, distance) pairs per
   rank;
3. each rank merges the `world` sorted top-k rows of each of its queries by
   (distance, id) (`adanns_merge_shards`).

With the FP32 path the merged result is the single-device search's: a
member's distance does not depend on where its list lives, the merge order is
the search's order, and global ids are assigned so that ascending local ids
stay ascending.  With a low-precision tier each rank shortlists rerank_k
candidates of its own lists, so the union over ranks holds the single-device
shortlist and the result is at least as close.

Only the partitioning and the exchange are host code; the searches, the id
map and the merge are the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import STORE_F32, index_create, map_ids, merge_shards, search_ivf


def partition_lists(sizes, world: int) -> np.ndarray:
    """Owner rank of each list: longest lists first, each to the rank with the
    fewest rows so far (ties: lower list id first, then lower rank)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    owner = np.zeros(len(sizes), dtype=np.int32)
    load = np.zeros(world, dtype=np.int64)
    for l in np.lexsort((np.arange(len(sizes)), -sizes)):
        r = int(np.argmin(load))
        owner[l] = r
        load[r] += sizes[l]
    return owner


def shard_rows(assign, owner, rank: int) -> np.ndarray:
    """Global ids (ascending) of the database rows whose list rank owns."""
    assign = np.asarray(assign)
    return np.nonzero(np.asarray(owner)[assign] == rank)[0].astype(np.int64)


def query_slices(B: int, world: int) -> list[tuple[int, int]]:
    """Contiguous split of B queries into `world` slices (sizes differ by <= 1)."""
    base, extra = divmod(B, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def exchange_topk(ids: torch.Tensor, dist: torch.Tensor, world: int, rank: int, group=None):
    """All-to-all of per-rank [B, k] results: rank r receives the rows of its
    query slice from every rank, returned as [world, B_r, k] (sender-major)."""
    import torch.distributed as tdist
    B, k = ids.shape
    sl = query_slices(B, world)
    lo, hi = sl[rank]
    if world == 1:
        return ids.unsqueeze(0), dist.unsqueeze(0)
    dev = ids.device
    if tdist.get_backend(group) == "gloo" and dev.type != "cpu":
        ids, dist = ids.cpu(), dist.cpu()
    send = [(h - l) * k for l, h in sl]
    recv = [(hi - lo) * k] * world
    ri = torch.empty(world * (hi - lo) * k, dtype=ids.dtype, device=ids.device)
    rd = torch.empty(world * (hi - lo) * k, dtype=dist.dtype, device=dist.device)
    tdist.all_to_all_single(ri, ids.contiguous().view(-1), recv, send, group=group)
    tdist.all_to_all_single(rd, dist.contiguous().view(-1), recv, send, group=group)
    return ri.view(world, hi - lo, k).to(dev), rd.view(world, hi - lo, k).to(dev)


class ShardedIndex:
    """This rank's part of an index whose lists are partitioned over `world`
    ranks (see the module docstring)."""

    def __init__(self, db: np.ndarray, centroids: np.ndarray, assign: np.ndarray, world: int,
                 rank: int, storage: int = STORE_F32, group=None, device=None):
        nlist = centroids.shape[0]
        self.world, self.rank, self.group = world, rank, group
        sizes = np.bincount(np.asarray(assign), minlength=nlist)
        self.owner = partition_lists(sizes, world)
        rows = shard_rows(assign, self.owner, rank)
        device = device or torch.device("cuda", torch.cuda.current_device())
        self.gids = torch.from_numpy(rows).to(device)
        self.n_rows = len(rows)
        self.index = index_create(
            torch.from_numpy(np.ascontiguousarray(db[rows])).to(device),
            torch.from_numpy(np.ascontiguousarray(centroids, dtype=np.float32)).to(device),
            torch.from_numpy(np.asarray(assign)[rows].astype(np.int32)).to(device),
            storage=storage)

    def search_partial(self, queries: torch.Tensor, d_c: int, d_s: int, nprobe: int, k: int,
                       storage: int = STORE_F32, rerank_k: int = 0):
        """Top-k of every query over this rank's lists, with global ids."""
        ids, dist = search_ivf(self.index, queries, d_c, d_s, nprobe, k, storage=storage,
                               rerank_k=rerank_k)
        return map_ids(ids, self.gids), dist

    def search(self, queries: torch.Tensor, d_c: int, d_s: int, nprobe: int, k: int,
               storage: int = STORE_F32, rerank_k: int = 0):
        """Merged top-k of this rank's query slice (`query_slices(B, world)[rank]`)."""
        ids, dist = self.search_partial(queries, d_c, d_s, nprobe, k, storage, rerank_k)
        ri, rd = exchange_topk(ids, dist, self.world, self.rank, self.group)
        return merge_shards(ri, rd)

    def free(self):
        self.index.free()
