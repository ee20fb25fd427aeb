"""FP64 CPU oracle for AdANNS-IVF / AdANNS-IVF-OPQ (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
use this package.  It shares no code with the GPU library: the heavy loops are
plain C in ``oracle_core.c`` (FP64, pthreads over queries), the orchestration
below is numpy FP64.  Library primitives serve as single steps only: a sort
(``np.argsort``), a matrix product and an SVD (``np.linalg.svd``).

Definitions (each function names the passage it follows):

* P_m(v) = v[0:m] / ||v[0:m]||, P_m(0) = 0 -- an m-prefix of a Matryoshka
  representation used as an m-dim representation (Sec. 3 "MR").  With the raw
  ``L2`` metric the prefix is used unnormalised.
* dist_m(q, x) = sum_{j<m} (P_m(q)_j - P_m(x)_j)^2 (squared L2).
* IVF build: Lloyd k-means on the d_c prefix of a seeded training sample,
  then every point joins the list of its nearest FP32 centroid (Sec. 3 "IVF",
  Algorithm 1 adannsConstruction).
* IVF search: n_p nearest centroids at d_c, exhaustive scan of those lists at
  d_s, k best by (distance, id) (Algorithm 1 adannsInference, Table "formula").
* OPQ: rotation R and M x 256 codebooks on the d_s prefix, trained by
  alternating Lloyd steps and an orthogonal Procrustes update; ADC search by M
  lookups (Sec. 3 "OPQ", Sec. 4.2, Sec. 4.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

METRIC_L2 = 0
METRIC_L2_PREFIXNORM = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_liboracle.so")
_SRC = os.path.join(_HERE, "oracle_core.c")
_SRCS = [_SRC, os.path.join(_HERE, "graph_core.c")]
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle in place (gcc, no arch-specific flags)."""
    if force or not os.path.exists(_SO) or \
            any(os.path.getmtime(_SO) < os.path.getmtime(f) for f in _SRCS):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64, i32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
        lib.orc_splitmix64_next.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        lib.orc_splitmix64_next.restype = u64
        lib.orc_sample.argtypes = [u64, i64, i64, P]
        lib.orc_prefix_normalize.argtypes = [P, i64, i64, i32, i32, P]
        lib.orc_prefix_normalize.restype = None
        lib.orc_assign.argtypes = [P, i64, i32, P, i32, P, P, P, i32]
        lib.orc_assign.restype = None
        lib.orc_ivf_search.argtypes = [P, i64, i32, P, i32, i32, P, P, P, i64, i32, i32, i32, i32,
                                       i32, P, P, P, P, P, i32]
        lib.orc_pq_encode.argtypes = [P, i64, i64, i32, i32, i32, P, P, P, P, P, i32]
        lib.orc_ivfopq_search.argtypes = [P, i64, i32, P, i32, i32, P, P, P, P, P, i32, P, i64,
                                          i32, i32, i32, i32, i32, i32, P, P, P, P, P, i32]
        lib.orc_knn_graph.argtypes = [P, i64, i32, i32, ctypes.c_double, ctypes.c_double, P, P, P,
                                      i32]
        lib.orc_graph_build.argtypes = [P, i64, i32, i32, i32, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, P, P, P, i32]
        lib.orc_graph_search.argtypes = [P, i64, i32, P, i32, i64, P, i64, i32, i32,
                                         ctypes.c_double, ctypes.c_double, P, P, P, P, i32]
        _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------
# seeded sampling (splitmix64 + partial Fisher-Yates)
# ----------------------------------------------------------------------------
def splitmix64(seed: int, count: int) -> list[int]:
    """First `count` outputs of splitmix64 started at `seed`."""
    lib = _load()
    st = ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF)
    return [int(lib.orc_splitmix64_next(ctypes.byref(st))) for _ in range(count)]


def sample(seed: int, n: int, take: int) -> np.ndarray:
    """First `take` entries of a splitmix64-seeded Fisher-Yates shuffle of [0, n)."""
    out = np.empty(take, dtype=np.int64)
    if _load().orc_sample(seed & 0xFFFFFFFFFFFFFFFF, n, take, _p(out)) != 0:
        raise ValueError("bad sample arguments")
    return out


# ----------------------------------------------------------------------------
# prefixes, distances
# ----------------------------------------------------------------------------
def prefix(x: np.ndarray, m: int, metric: int = METRIC_L2_PREFIXNORM) -> np.ndarray:
    """P_m of every row (FP64) for the prefix-normalised metric, else the raw prefix."""
    x = _c(x, np.float32)
    out = np.empty((x.shape[0], m), dtype=np.float64)
    _load().orc_prefix_normalize(_p(x), x.shape[0], x.shape[1], m,
                                 int(metric == METRIC_L2_PREFIXNORM), _p(out))
    return out


def assign(T: np.ndarray, C: np.ndarray, nthreads: int | None = None):
    """Nearest centroid by squared L2, ties to the smallest index (Lloyd step 1).

    Returns (assignment int32, best distance, second-best distance), FP64."""
    T = _c(T, np.float64)
    C = _c(C, np.float64)
    n, dim = T.shape
    a = np.empty(n, dtype=np.int32)
    b = np.empty(n, dtype=np.float64)
    s = np.empty(n, dtype=np.float64)
    _load().orc_assign(_p(T), n, dim, _p(C), C.shape[0], _p(a), _p(b), _p(s), _threads(nthreads))
    return a, b, s


def update(T: np.ndarray, a: np.ndarray, C_prev: np.ndarray) -> np.ndarray:
    """Lloyd step 2: each centroid becomes the FP64 mean of its members; an
    empty cluster keeps its previous centroid."""
    nc = C_prev.shape[0]
    sums = np.zeros_like(C_prev, dtype=np.float64)
    np.add.at(sums, a, T)
    cnt = np.bincount(a, minlength=nc)
    C = np.array(C_prev, dtype=np.float64, copy=True)
    ne = cnt > 0
    C[ne] = sums[ne] / cnt[ne, None]
    return C


def lloyd(T: np.ndarray, C0: np.ndarray, niter: int, nthreads: int | None = None):
    """`niter` Lloyd iterations from C0.  Returns (C, objectives) where
    objectives[t] = sum of squared distances at the assignment of iteration t."""
    C = np.array(C0, dtype=np.float64, copy=True)
    objs = []
    for _ in range(niter):
        a, b, _ = assign(T, C, nthreads)
        objs.append(float(b.sum()))
        C = update(T, a, C)
    return C, objs


# ----------------------------------------------------------------------------
# AdANNS-IVF
# ----------------------------------------------------------------------------
def lists_from_assignment(assign_: np.ndarray, nlist: int):
    """CSR inverted lists: offsets int64 [nlist+1], ids int32 ascending in each list."""
    cnt = np.bincount(assign_, minlength=nlist).astype(np.int64)
    off = np.zeros(nlist + 1, dtype=np.int64)
    np.cumsum(cnt, out=off[1:])
    ids = np.argsort(assign_, kind="stable").astype(np.int32)
    return off, ids


def build_ivf(db: np.ndarray, d_c: int, nlist: int, niter: int, train_n: int, seed: int,
              metric: int = METRIC_L2_PREFIXNORM, nthreads: int | None = None) -> dict:
    """AdANNS-IVF construction (Algorithm 1 adannsConstruction, Sec. 4.1).

    1. S = sample(seed, N, train_n); T = P_dc(db[S]).
    2. Forgy init: mu_h = T[sample(seed + 1, train_n, nlist)[h]].
    3. `niter` Lloyd iterations (ties -> smallest h, empty -> keep).
    4. Round the centroids to FP32: those values are the index.
    5. Assign all N points (P_dc, FP64 arithmetic) to the FP32 centroids.
    6. CSR lists with ids ascending in each list.
    """
    db = _c(db, np.float32)
    N = db.shape[0]
    if not (1 <= nlist <= train_n <= N) or d_c < 1 or d_c > db.shape[1]:
        raise ValueError("bad IVF build arguments")
    S = sample(seed, N, train_n)
    T = prefix(db[S], d_c, metric)
    init = sample(seed + 1, train_n, nlist)
    C, objs = lloyd(T, T[init], niter, nthreads)
    cent = C.astype(np.float32)
    X = prefix(db, d_c, metric)
    a, best, second = assign(X, cent.astype(np.float64), nthreads)
    off, ids = lists_from_assignment(a, nlist)
    return {"centroids": cent, "assign": a, "assign_best": best, "assign_second": second,
            "list_off": off, "list_ids": ids, "objectives": objs, "train_idx": S,
            "init_idx": init, "d_c": d_c, "nlist": nlist, "metric": metric}


def search_ivf(db: np.ndarray, index: dict, queries: np.ndarray, d_c: int, d_s: int, nprobe: int,
               k: int, metric: int | None = None, nthreads: int | None = None) -> dict:
    """AdANNS-IVF search (Algorithm 1 adannsInference; Table "formula").

    Returns ids int64 [B, k], dist FP64 [B, k] (padded with -1 / +inf),
    probes int32 [B, nprobe] and the nprobe+1 smallest coarse distances."""
    metric = index["metric"] if metric is None else metric
    db = _c(db, np.float32)
    queries = _c(queries, np.float32)
    cent = _c(index["centroids"], np.float32)
    B, d = queries.shape
    ids = np.empty((B, k), dtype=np.int64)
    dist = np.empty((B, k), dtype=np.float64)
    probes = np.empty((B, nprobe), dtype=np.int32)
    pd = np.full((B, nprobe + 1), np.inf, dtype=np.float64)
    ncand = np.empty(B, dtype=np.int64)
    rc = _load().orc_ivf_search(_p(db), db.shape[0], d, _p(cent), cent.shape[0], cent.shape[1],
                                _p(_c(index["list_off"], np.int64)),
                                _p(_c(index["list_ids"], np.int32)), _p(queries), B, d_c, d_s,
                                nprobe, k, int(metric == METRIC_L2_PREFIXNORM), _p(ids), _p(dist),
                                _p(probes), _p(pd), _p(ncand), _threads(nthreads))
    if rc != 0:
        raise ValueError("bad IVF search arguments")
    return {"ids": ids, "dist": dist, "probes": probes, "probe_dist": pd, "ncand": ncand}


# ----------------------------------------------------------------------------
# OPQ on the d_s prefix, ADC search
# ----------------------------------------------------------------------------
def procrustes(Y: np.ndarray, Zhat: np.ndarray) -> np.ndarray:
    """argmin over orthogonal R of ||Y R - Zhat||_F: R = U V^T with
    U S V^T = svd(Y^T Zhat) (orthogonal Procrustes, the OPQ rotation step)."""
    U, _, Vt = np.linalg.svd(Y.T @ Zhat)
    return U @ Vt


def pq_assign(Z: np.ndarray, C: np.ndarray, M: int, nthreads: int | None = None) -> np.ndarray:
    """codes [n, M]: per subspace the nearest of 256 codewords (ties -> smallest)."""
    n, d_s = Z.shape
    dsub = d_s // M
    codes = np.empty((n, M), dtype=np.uint8)
    for m in range(M):
        a, _, _ = assign(Z[:, m * dsub:(m + 1) * dsub], C[m], nthreads)
        codes[:, m] = a
    return codes


def pq_decode(codes: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Reconstruction: concatenation of the chosen codewords."""
    M = C.shape[0]
    return np.concatenate([C[m][codes[:, m]] for m in range(M)], axis=1)


def distortion(Z: np.ndarray, C: np.ndarray, codes: np.ndarray) -> float:
    return float(((Z - pq_decode(codes, C)) ** 2).sum() / Z.shape[0])


def list_centroids(db: np.ndarray, index: dict, d_s: int,
                   metric: int = METRIC_L2_PREFIXNORM) -> np.ndarray:
    """Residual centres of the IVF-OPQ composite: for every inverted list the
    FP64 mean of its members' P_ds prefixes, rounded to FP32 (an empty list
    gets the zero vector).  The coarse centroids live at d_c only, so the
    residual that the codes of the d_s prefix encode is taken against these
    d_s-dimensional list means (the reading of residual encoding used here)."""
    X = prefix(db, d_s, metric)
    nlist = index["nlist"]
    a = np.asarray(index["assign"])
    sums = np.zeros((nlist, d_s))
    np.add.at(sums, a, X)
    cnt = np.bincount(a, minlength=nlist)
    out = np.zeros((nlist, d_s))
    ne = cnt > 0
    out[ne] = sums[ne] / cnt[ne, None]
    return out.astype(np.float32)


def train_opq(db: np.ndarray, d_s: int, M: int, opq_iters: int, pq_iters: int, final_iters: int,
              train_n: int, seed: int, metric: int = METRIC_L2_PREFIXNORM,
              nthreads: int | None = None, residual: dict | None = None) -> dict:
    """AdANNS-OPQ training on the d_s prefix (Sec. 3 "OPQ", Sec. 4.2).

    Y = P_ds(db[sample(seed + 2, N, train_n)]), R_0 = I.  Each outer iteration:
    Z = Y R; per subspace `pq_iters` Lloyd steps with 256 codewords (Forgy
    init from sample(seed + 3, n, .) on the first iteration, warm start
    after); encode; R <- Procrustes(Y, Zhat).  Then `final_iters` Lloyd steps
    on Y R.  R and the codebooks are rounded to FP32 (the index values).
    `trace` records the distortion after every half-step; it never increases.
    With residual = dict(lcent=list centroids [nlist, d_s], assign=list of each
    row), the training rows are the residuals P_ds(x) - lcent[list(x)].
    """
    db = _c(db, np.float32)
    N = db.shape[0]
    if M < 1 or d_s % M != 0 or not (1 <= train_n <= N):
        raise ValueError("bad OPQ arguments")
    dsub = d_s // M
    S = sample(seed + 2, N, train_n)
    Y = prefix(db[S], d_s, metric)
    if residual is not None:
        Y = Y - np.asarray(residual["lcent"], dtype=np.float32)[
            np.asarray(residual["assign"])[S]].astype(np.float64)
    n = Y.shape[0]
    perm = sample(seed + 3, n, min(256, n))
    init_rows = perm[np.arange(256) % len(perm)]
    R = np.eye(d_s)
    C = None
    trace = []
    for _ in range(opq_iters):
        Z = Y @ R
        if C is None:
            C = np.stack([Z[init_rows, m * dsub:(m + 1) * dsub] for m in range(M)])
        else:
            trace.append(distortion(Z, C, pq_assign(Z, C, M, nthreads)))
        C = np.stack([lloyd(Z[:, m * dsub:(m + 1) * dsub], C[m], pq_iters, nthreads)[0]
                      for m in range(M)])
        codes = pq_assign(Z, C, M, nthreads)
        trace.append(distortion(Z, C, codes))
        Zhat = pq_decode(codes, C)
        R = procrustes(Y, Zhat)
        trace.append(float(((Y @ R - Zhat) ** 2).sum() / n))
    Z = Y @ R
    if C is None:
        C = np.stack([Z[init_rows, m * dsub:(m + 1) * dsub] for m in range(M)])
    C = np.stack([lloyd(Z[:, m * dsub:(m + 1) * dsub], C[m], final_iters, nthreads)[0]
                  for m in range(M)])
    trace.append(distortion(Z, C, pq_assign(Z, C, M, nthreads)))
    out = {"R": R.astype(np.float32), "codebooks": C.astype(np.float32), "R64": R,
           "codebooks64": C, "trace": trace, "train_idx": S, "d_s": d_s, "M": M,
           "metric": metric}
    if residual is not None:
        out["lcent"] = np.asarray(residual["lcent"], dtype=np.float32)
    return out


def pq_encode(db: np.ndarray, d_s: int, M: int, R: np.ndarray, codebooks: np.ndarray,
              metric: int = METRIC_L2_PREFIXNORM, nthreads: int | None = None,
              lcent: np.ndarray | None = None, assign: np.ndarray | None = None) -> np.ndarray:
    """codes uint8 [N, M] of z = P_ds(x) R under the given (FP32) R / codebooks;
    with list centroids lcent and the rows' lists assign, of the residual
    z = (P_ds(x) - lcent[assign[x]]) R."""
    db = _c(db, np.float32)
    R64 = _c(np.asarray(R, dtype=np.float32).astype(np.float64), np.float64)
    C64 = _c(np.asarray(codebooks, dtype=np.float32).astype(np.float64), np.float64)
    lc = None if lcent is None else _c(lcent, np.float32)
    asg = None if lcent is None else _c(assign, np.int32)
    codes = np.empty((db.shape[0], M), dtype=np.uint8)
    rc = _load().orc_pq_encode(_p(db), db.shape[0], db.shape[1], d_s, M,
                               int(metric == METRIC_L2_PREFIXNORM), _p(R64), _p(C64), _p(lc),
                               _p(asg), _p(codes), _threads(nthreads))
    if rc != 0:
        raise ValueError("bad encode arguments")
    return codes


def search_ivfopq(db: np.ndarray, index: dict, opq: dict, codes: np.ndarray, queries: np.ndarray,
                  d_c: int, nprobe: int, k: int, rerank_k: int = 0, metric: int | None = None,
                  nthreads: int | None = None) -> dict:
    """AdANNS-IVFOPQ search: IVF at d_c, ADC distances on the rotated d_s
    prefix inside the probed lists, optional exact rerank of the rerank_k
    best (Sec. 4.3; Table "formula" IVFOPQ row read as asymmetric lookup).
    When `opq` holds list centroids ("lcent"), the codes are of residuals and
    each probed list l gets its own table from (P_ds(q) - lcent[l]) R."""
    metric = index["metric"] if metric is None else metric
    db = _c(db, np.float32)
    queries = _c(queries, np.float32)
    cent = _c(index["centroids"], np.float32)
    R = _c(opq["R"], np.float32)
    C = _c(opq["codebooks"], np.float32)
    codes = _c(codes, np.uint8)
    B, d = queries.shape
    d_s, M = int(opq["d_s"]), int(opq["M"])
    ids = np.empty((B, k), dtype=np.int64)
    dist = np.empty((B, k), dtype=np.float64)
    probes = np.empty((B, nprobe), dtype=np.int32)
    pd = np.full((B, nprobe + 1), np.inf, dtype=np.float64)
    rc = _load().orc_ivfopq_search(_p(db), db.shape[0], d, _p(cent), cent.shape[0], cent.shape[1],
                                   _p(_c(index["list_off"], np.int64)),
                                   _p(_c(index["list_ids"], np.int32)), _p(R), _p(C), _p(codes),
                                   M, _p(queries), B, d_c, d_s, nprobe, k, rerank_k,
                                   int(metric == METRIC_L2_PREFIXNORM),
                                   _p(_c(opq["lcent"], np.float32)) if "lcent" in opq else None,
                                   _p(ids), _p(dist), _p(probes), _p(pd), _threads(nthreads))
    if rc != 0:
        raise ValueError("bad IVF-OPQ search arguments")
    return {"ids": ids, "dist": dist, "probes": probes, "probe_dist": pd}


# ----------------------------------------------------------------------------
# cost model (App. "Inference Compute Cost")
# ----------------------------------------------------------------------------
def mflops_per_query(d_c: int, d_s: int, nlist: int, nprobe: int, N: int) -> dict:
    """The paper prints C = d_s*k + n_p*d_s*N/k (k = #clusters) while defining
    d_c as the cluster-construction dimension; the first term is read here as
    the cluster-mapping cost d_c*k.  Both forms are returned, in MFLOPs."""
    read = d_c * nlist + nprobe * d_s * N / nlist
    literal = d_s * nlist + nprobe * d_s * N / nlist
    return {"mflops": read / 1e6, "mflops_literal": literal / 1e6}


# ----------------------------------------------------------------------------
# low-d graph shortlist + high-d rerank (AdANNS-DiskANN, Sec. 4.3)
# ----------------------------------------------------------------------------
# Ties within this tolerance make a decision "ambiguous" for a comparison with
# an FP32 implementation (the parity rule's relative tolerance and floor).
AMB_REL, AMB_ABS = 1e-5, 2.4e-7


def knn_graph(db: np.ndarray, d_g: int, K: int, metric: int = METRIC_L2_PREFIXNORM,
              nthreads: int | None = None):
    """The K nearest other rows of every row at the d_g prefix, by (distance,
    id): (ids int32 [N, K], distances FP64, ambiguity flag of the K-th cut)."""
    X = prefix(db, d_g, metric)
    N = X.shape[0]
    nbr = np.empty((N, K), dtype=np.int32)
    dist = np.empty((N, K), dtype=np.float64)
    amb = np.empty(N, dtype=np.uint8)
    if _load().orc_knn_graph(_p(X), N, d_g, K, AMB_REL, AMB_ABS, _p(nbr), _p(dist), _p(amb),
                             _threads(nthreads)) != 0:
        raise ValueError("bad kNN graph arguments")
    return nbr, dist, amb.astype(bool)


def build_graph(db: np.ndarray, d_g: int, K: int, R: int, alpha: float,
                metric: int = METRIC_L2_PREFIXNORM, nthreads: int | None = None) -> dict:
    """AdANNS-DiskANN graph formed with the low-d MR (Sec. 4.3): at the d_g
    prefix, every row's K nearest other rows are robust-pruned (factor alpha)
    to at most R out-neighbours, every edge offers its source to its target,
    and rows holding more than R are pruned again over the union.  Returns
    dict(graph int32 [N, R] (-1 padding, rows by (distance, id)), entry (row
    nearest to the mean), amb (rows with a decision within tolerance))."""
    X = prefix(db, d_g, metric)
    N = X.shape[0]
    g = np.empty((N, R), dtype=np.int32)
    amb = np.empty(N, dtype=np.uint8)
    entry = ctypes.c_int64()
    if _load().orc_graph_build(_p(X), N, d_g, K, R, float(alpha), AMB_REL, AMB_ABS, _p(g),
                               _p(amb), ctypes.byref(entry), _threads(nthreads)) != 0:
        raise ValueError("bad graph build arguments")
    return {"graph": g, "entry": int(entry.value), "amb": amb.astype(bool), "d_g": d_g, "R": R,
            "K": K, "alpha": alpha, "metric": metric}


def search_graph(db: np.ndarray, gr: dict, queries: np.ndarray, L: int, d_s: int, k: int,
                 rerank_k: int, nthreads: int | None = None) -> dict:
    """Best-first search of the graph at the d_g prefix with a candidate list
    of L, then the rerank_k nearest of the list re-scored with dist_ds (the
    high-d MR, Sec. 4.3 shortlist-rerank) and the k best by (distance, id).
    Returns ids, dist (FP64, -1 / +inf padding), the graph stage's shortlist
    (short_ids, short_dist), amb (a traversal decision within tolerance) and
    the number of expanded rows per query."""
    metric = gr["metric"]
    X = prefix(db, gr["d_g"], metric)
    Q = prefix(queries, gr["d_g"], metric)
    B = Q.shape[0]
    sid = np.empty((B, rerank_k), dtype=np.int64)
    sd = np.empty((B, rerank_k), dtype=np.float64)
    amb = np.empty(B, dtype=np.uint8)
    nexp = np.empty(B, dtype=np.int64)
    if _load().orc_graph_search(_p(X), X.shape[0], gr["d_g"], _p(_c(gr["graph"], np.int32)),
                                gr["R"], gr["entry"], _p(Q), B, L, rerank_k, AMB_REL, AMB_ABS,
                                _p(sid), _p(sd), _p(amb), _p(nexp), _threads(nthreads)) != 0:
        raise ValueError("bad graph search arguments")
    ids = np.full((B, k), -1, dtype=np.int64)
    dist = np.full((B, k), np.inf)
    Ps = prefix(queries, d_s, metric)
    for i in range(B):
        c = sid[i][sid[i] >= 0]
        if len(c) == 0:
            continue
        d = ((prefix(db[c], d_s, metric) - Ps[i][None]) ** 2).sum(1)
        o = np.lexsort((c, d))[:k]
        ids[i, :len(o)], dist[i, :len(o)] = c[o], d[o]
    return {"ids": ids, "dist": dist, "short_ids": sid, "short_dist": sd,
            "amb": amb.astype(bool), "expanded": nexp}
