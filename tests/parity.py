"""Acceptance rule for GPU-vs-oracle comparisons of top-k results.

Distances: |gpu - oracle| <= REL * |oracle| + ABS_FLOOR * scale.  REL = 1e-5 is
the stated FP32 tolerance.  The floor covers distances near zero: the GPU
rounds the normalised inputs to FP32 (relative 2^-24 per coordinate), and for a
near-duplicate pair the squared difference of two such roundings leaves an
absolute error of about 4 * 2^-24 * sqrt(dist) <= 2.4e-7 for unit-norm
prefixes, which no relative bound can absorb as dist -> 0.  `scale` is 1 for
prefix-normalised distances and the squared query norm for raw L2.

Ids: the oracle's ranking is split into tie groups, consecutive ranks whose
distance gap is within the same tolerance.  Inside a group the ids are
compared as sets; the group that straddles rank k must contribute a subset of
its ids; every other rank must match exactly.
"""
from __future__ import annotations

import numpy as np

REL = 1e-5
ABS_FLOOR = 2.4e-7


def tol(d_ref, scale=1.0):
    d_ref = np.asarray(d_ref, dtype=np.float64)
    return REL * np.abs(d_ref) + ABS_FLOOR * scale


def tie_groups(dist: np.ndarray, scale=1.0) -> list[tuple[int, int]]:
    """Half-open rank ranges of near-equal oracle distances (ascending input)."""
    groups = []
    a = 0
    n = len(dist)
    for r in range(1, n + 1):
        if r == n:
            groups.append((a, r))
            break
        d0, d1 = dist[r - 1], dist[r]
        same = (not np.isfinite(d0) and not np.isfinite(d1)) or \
            (np.isfinite(d1) and d1 - d0 <= tol(d1, scale))
        if not same:
            groups.append((a, r))
            a = r
    return groups


def check_row(g_ids, g_dist, o_ids, o_dist, k, scale=1.0):
    """Return a list of problems for one query (empty when it passes)."""
    probs = []
    o_ids = np.asarray(o_ids)
    o_dist = np.asarray(o_dist, dtype=np.float64)
    g_ids = np.asarray(g_ids)
    g_dist = np.asarray(g_dist, dtype=np.float64)
    for r in range(k):
        od, gd = o_dist[r], g_dist[r]
        if not np.isfinite(od):
            if np.isfinite(gd) or g_ids[r] != -1:
                probs.append(f"rank {r}: expected padding, got id {g_ids[r]} dist {gd}")
            continue
        if not np.isfinite(gd) or abs(gd - od) > tol(od, scale):
            probs.append(f"rank {r}: dist {gd!r} vs oracle {od!r}")
    for a, b in tie_groups(o_dist, scale):
        if a >= k:
            break
        hi = min(b, k)
        gs = set(int(v) for v in g_ids[a:hi])
        if b <= k:
            if gs != set(int(v) for v in o_ids[a:b]):
                probs.append(f"ranks [{a},{b}): ids {sorted(gs)} vs oracle {sorted(o_ids[a:b])}")
        else:
            if not gs <= set(int(v) for v in o_ids[a:b]):
                probs.append(f"ranks [{a},{k}) (tie group to {b}): ids {sorted(gs)} not within "
                             f"oracle {sorted(o_ids[a:b])}")
    return probs


def ambiguous_probe_rows(probe_dist: np.ndarray, nprobe: int, scale=1.0) -> np.ndarray:
    """Queries whose n_p-th and (n_p+1)-th centroid distances are within tolerance:
    their probe set is not unique, so their ids are excluded from the strict check."""
    if probe_dist.shape[1] <= nprobe:
        return np.zeros(probe_dist.shape[0], dtype=bool)
    a = probe_dist[:, nprobe - 1]
    b = probe_dist[:, nprobe]
    return np.isfinite(b) & (b - a <= tol(b, scale))


def check_topk(g_ids, g_dist, o_ids, o_dist, k, skip_rows=None, scale=None, max_report=5):
    """Check every row; returns (n_checked, failures[list of (row, problems)])."""
    B = g_ids.shape[0]
    fails = []
    n = 0
    for i in range(B):
        if skip_rows is not None and skip_rows[i]:
            continue
        n += 1
        s = 1.0 if scale is None else float(scale[i])
        p = check_row(g_ids[i], g_dist[i], o_ids[i], o_dist[i], k, s)
        if p:
            fails.append((i, p[:max_report]))
    return n, fails


def recall(g_ids, o_ids, k):
    """|top-k(gpu) ∩ top-k(oracle)| / k averaged over queries (k-Recall@k)."""
    tot = 0.0
    for a, b in zip(g_ids[:, :k], o_ids[:, :k]):
        bs = set(int(v) for v in b if v >= 0)
        if not bs:
            tot += 1.0
            continue
        tot += len(bs & set(int(v) for v in a if v >= 0)) / len(bs)
    return tot / len(g_ids)


def full_groups(o, rerun, k):
    """Rows whose tie group at rank k-1 runs to the end of the oracle's list are
    searched again with every candidate returned, so that group is complete."""
    d = o["dist"]
    last = d[:, -1]
    trunc = np.isfinite(last) & (last - d[:, k - 1] <= tol(last))
    if not trunc.any():
        return o
    rows = np.nonzero(trunc)[0]
    kk = int(o["ncand"][rows].max()) if "ncand" in o else 4 * d.shape[1]
    o2 = rerun(rows, max(kk, d.shape[1]))
    K = o2["ids"].shape[1]
    ids = np.full((d.shape[0], K), -1, dtype=np.int64)
    dist = np.full((d.shape[0], K), np.inf)
    ids[:, :d.shape[1]], dist[:, :d.shape[1]] = o["ids"], d
    ids[rows], dist[rows] = o2["ids"], o2["dist"]
    o = dict(o)
    o["ids"], o["dist"] = ids, dist
    return o
