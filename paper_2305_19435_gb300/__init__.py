"""Python binding of the AdANNS GB300 library (libadanns.so, C ABI in include/adanns.h).

Argument marshalling only: tensors must already be CUDA tensors of the stated
dtype; every step of every operation runs in the library's CUDA kernels on
the current torch stream.  There is no CPU path: if the compiled library is
missing, importing this module still works but every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

METRIC_L2 = 0
METRIC_L2_PREFIXNORM = 1
STORE_F32 = 1
GRANULARITIES = (8, 16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 2048)

ERRORS = {-1: "ARG", -2: "DIM", -3: "OOM", -4: "CUDA", -5: "TIMEOUT", -6: "STATE"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libadanns.so")
_lib = None


class AdannsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"adanns error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({LIB_PATH} missing); run "
                               "paper_2305_19435_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
        L.adanns_last_error.restype = ctypes.c_char_p
        L.adanns_version.restype = i32
        L.adanns_launch_count.restype = i64
        L.adanns_profile_enable.argtypes = [i32]
        L.adanns_profile_read.argtypes = [P, P, i32]
        L.adanns_profile_read_host.argtypes = [P, i32]
        L.adanns_profile_read_counters.argtypes = [P, i32]
        L.adanns_build_ivf.argtypes = [P, i64, i32, i32, i32, i32, i64, u64, i32, i32, P, P, P]
        L.adanns_index_create.argtypes = [P, i64, i32, P, i32, i32, P, i32, i32, P, P]
        L.adanns_index_info.argtypes = [P, P, P, P, P, P]
        L.adanns_index_get_lists.argtypes = [P, P, P, P]
        L.adanns_index_get_centroids.argtypes = [P, P, P]
        L.adanns_index_free.argtypes = [P]
        L.adanns_index_free.restype = None
        L.adanns_kmeans_assign.argtypes = [P, i64, i32, i32, i32, P, i32, P, P, P]
        L.adanns_kmeans_update.argtypes = [P, i64, i32, i32, i32, P, i32, P, P]
        L.adanns_search_ivf.argtypes = [P, P, i64, i32, i32, i32, i32, i32, i32, P, P, P, P]
        L.adanns_search_ivf_budgets.argtypes = [P, P, i64, i32, P, P, P, i32, i32, i32, P, P, P]
        L.adanns_search_ivf_host.argtypes = [P, P, i64, i32, i32, i32, i32, i32, i32, P, P, i64, P]
        L.adanns_search_ivfopq_budgets.argtypes = [P, P, i64, i32, P, P, i32, i32, P, P, P]
        L.adanns_opq_encode.argtypes = [P, i64, i32, i32, i32, i32, P, P, P, P]
        L.adanns_pq_update.argtypes = [P, i64, i32, i32, P, P, P]
        L.adanns_procrustes.argtypes = [P, P, i64, i32, P, P]
        L.adanns_build_opq.argtypes = [P, P, i32, i32, i32, i32, i32, i64, u64, P, P]
        L.adanns_index_set_opq.argtypes = [P, i32, i32, P, P, P, P]
        L.adanns_index_get_opq.argtypes = [P, P, P, P, P]
        L.adanns_search_ivfopq.argtypes = [P, P, i64, i32, i32, i32, i32, P, P, P, P]
        L.adanns_index_status.argtypes = [P, P]
        L.adanns_search_scratch_bytes.argtypes = [P, i64, i32, i32, i32, i32, i32, i32]
        L.adanns_search_scratch_bytes.restype = i64
        L.adanns_autotune_search.argtypes = [P, P, i64, i32, i32, i32, i32, P, P, P, P, P]
        L.adanns_autotune_search_lowp.argtypes = [P, P, i64, i32, i32, i32, i32, i32, i32, P, P,
                                                  P, P, P]
        L.adanns_tune_save.argtypes = [ctypes.c_char_p]
        L.adanns_tune_load.argtypes = [ctypes.c_char_p]
        L.adanns_tune_clear.argtypes = []
        L.adanns_plan_create.argtypes = [P, P, i64, i32, i32, i32, i32, i32, i32, P, P, P, P]
        L.adanns_plan_launch.argtypes = [P, P]
        L.adanns_plan_free.argtypes = [P]
        L.adanns_plan_free.restype = None
        L.adanns_map_ids.argtypes = [P, i64, P, i64, P]
        L.adanns_merge_shards.argtypes = [P, P, i32, i64, i32, P, P, P]
        L.adanns_index_opq_info.argtypes = [P, P, P]
        L.adanns_build_opq_residual.argtypes = [P, P, i32, i32, i32, i32, i32, i64, u64, P, P]
        L.adanns_index_set_opq_residual.argtypes = [P, i32, i32, P, P, P, P, P]
        L.adanns_index_get_list_centres.argtypes = [P, P, P]
        L.adanns_index_export.argtypes = [P, ctypes.c_char_p, P]
        L.adanns_index_import.argtypes = [ctypes.c_char_p, P, P]
        L.adanns_server_create.argtypes = [P, i32, i32, i64, i64, P]
        L.adanns_server_submit.argtypes = [P, i32, P, i64, P, P]
        L.adanns_server_poll.argtypes = [P, i64, i32, P, P, P]
        L.adanns_server_stats.argtypes = [P, P, P, P, P, P, P, P]
        L.adanns_server_destroy.argtypes = [P]
        L.adanns_graph_build.argtypes = [P, i64, i32, i32, i32, i32, ctypes.c_float, i32, P, P]
        L.adanns_graph_create.argtypes = [P, i64, i32, i32, P, i32, i64, i32, P, P]
        L.adanns_graph_info.argtypes = [P, P, P, P, P, P]
        L.adanns_graph_get.argtypes = [P, P, P]
        L.adanns_graph_search.argtypes = [P, P, i64, i32, i32, i32, i32, P, P, P, P]
        L.adanns_graph_free.argtypes = [P]
        L.adanns_graph_free.restype = None
        L.adanns_set_option.argtypes = [i32, i64]
        L.adanns_get_option.argtypes = [i32, P]
        _lib = L
    return _lib


# runtime options (include/adanns.h ADANNS_OPT_*)
OPT_FP32_STREAM = 0
OPT_ADC_SELECT = 1
OPT_COARSE_TC = 2
OPT_RERANK_PRUNE = 3
OPT_SCRATCH_BYTES = 4
OPT_WAIT_LIMIT_NS = 5
OPT_TEST_SKIP_LOAD = 6
OPT_SCAN_FILTER = 7
OPT_NARROW_SCAN = 8


def set_option(opt: int, value: int):
    """Set a process-wide runtime option (kernel choices, scratch and wait bounds)."""
    _check(lib().adanns_set_option(int(opt), int(value)))


def get_option(opt: int) -> int:
    v = ctypes.c_int64()
    _check(lib().adanns_get_option(int(opt), ctypes.byref(v)))
    return int(v.value)


class option:
    """Context manager: `with option(OPT_X, v): ...` sets an option and restores it."""

    def __init__(self, opt: int, value: int):
        self.opt, self.value = opt, value

    def __enter__(self):
        self.old = get_option(self.opt)
        set_option(self.opt, self.value)
        return self

    def __exit__(self, *exc):
        set_option(self.opt, self.old)


class BudgetC(ctypes.Structure):
    """adanns_budget (include/adanns.h)."""
    _fields_ = [("method", ctypes.c_int), ("d_c", ctypes.c_int), ("d_s", ctypes.c_int),
                ("nprobe", ctypes.c_int), ("k", ctypes.c_int), ("storage", ctypes.c_int),
                ("rerank_k", ctypes.c_int)]


METHOD_IVF = 0
METHOD_IVFOPQ = 1
PENDING = 1


def launch_count() -> int:
    """Kernels launched by the library since load (host-side counter)."""
    return int(lib().adanns_launch_count())


STAGES = ("prep", "coarse", "invert", "scan", "merge", "lut", "adc", "rerank", "mma", "select",
          "rr_sort", "rr_pairs", "rr_final")
STORE_BF16 = 2
STORE_FP8 = 4


def profile_enable(on: bool = True):
    """Start (or stop) recording per-stage CUDA-event timings; clears records."""
    _check(lib().adanns_profile_enable(int(on)))


def profile_read(nstage: int = 16) -> dict:
    """{stage: (total ms, records)} for the recorded stages (synchronises)."""
    ms = (ctypes.c_double * nstage)()
    cnt = (ctypes.c_int64 * nstage)()
    _check(lib().adanns_profile_read(ms, cnt, nstage))
    names = list(STAGES) + [f"stage{i}" for i in range(len(STAGES), nstage)]
    return {names[i]: (ms[i], cnt[i]) for i in range(nstage) if cnt[i]}


def profile_read_host(nstage: int = 16) -> dict:
    """{stage: host microseconds spent issuing it} since profiling was enabled."""
    us = (ctypes.c_double * nstage)()
    _check(lib().adanns_profile_read_host(us, nstage))
    names = list(STAGES) + [f"stage{i}" for i in range(len(STAGES), nstage)]
    return {names[i]: us[i] for i in range(nstage) if us[i]}


COUNTERS = ("rerank_pairs", "shortlist_slots", "scan_survivors", "select_slow_queries")


def profile_read_counters() -> dict:
    """{counter: total} of the work counters since profiling was enabled (synchronises)."""
    v = (ctypes.c_int64 * 8)()
    _check(lib().adanns_profile_read_counters(v, 8))
    return {name: int(v[i]) for i, name in enumerate(COUNTERS)}


def _check(rc: int):
    if rc != 0:
        raise AdannsError(rc, lib().adanns_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, dtype, name: str, ndim: int | None = None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dims")


class Index:
    """An index owned by the library (device memory), freed by `free()` or GC."""

    def __init__(self, handle: ctypes.c_void_p, objective=None):
        self._h = handle
        self.objective = objective
        N, d, dc, nl, m = (ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(),
                           ctypes.c_int())
        _check(lib().adanns_index_info(self._h, ctypes.byref(N), ctypes.byref(d), ctypes.byref(dc),
                                       ctypes.byref(nl), ctypes.byref(m)))
        self.N, self.d, self.d_c, self.nlist, self.metric = N.value, d.value, dc.value, nl.value, m.value
        ods, om = ctypes.c_int(), ctypes.c_int()
        _check(lib().adanns_index_opq_info(handle, ctypes.byref(ods), ctypes.byref(om)))
        self.opq = (ods.value, om.value) if om.value else None

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("index already freed")
        return self._h

    def free(self):
        if self._h is not None and _lib is not None:
            _lib.adanns_index_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def lists(self):
        off = torch.empty(self.nlist + 1, dtype=torch.int64, device="cuda")
        ids = torch.empty(self.N, dtype=torch.int32, device="cuda")
        _check(lib().adanns_index_get_lists(self.handle, _ptr(off), _ptr(ids), _stream()))
        return off, ids

    def status(self):
        """Raise if a tensor-core pipeline wait timed out since the last check (synchronises)."""
        _check(lib().adanns_index_status(self.handle, _stream()))

    def centroids(self):
        c = torch.empty(self.nlist, self.d_c, dtype=torch.float32, device="cuda")
        _check(lib().adanns_index_get_centroids(self.handle, _ptr(c), _stream()))
        return c


def build_ivf(db: torch.Tensor, d_c: int, nlist: int, niter: int, train_n: int, seed: int,
              metric: int = METRIC_L2_PREFIXNORM, storage: int = STORE_F32) -> Index:
    """AdANNS-IVF construction (k-means at d_c + CSR prefix-major lists)."""
    _need(db, torch.float32, "db", 2)
    obj = (ctypes.c_double * max(niter, 1))()
    h = ctypes.c_void_p()
    _check(lib().adanns_build_ivf(_ptr(db), db.shape[0], db.shape[1], d_c, nlist, niter, train_n,
                                  seed, metric, storage, obj, _stream(), ctypes.byref(h)))
    return Index(h, objective=list(obj)[:niter])


def index_create(db: torch.Tensor, centroids: torch.Tensor, assign: torch.Tensor,
                 metric: int = METRIC_L2_PREFIXNORM, storage: int = STORE_F32) -> Index:
    """Index from given FP32 centroids [nlist, d_c] and list assignment int32 [N]."""
    _need(db, torch.float32, "db", 2)
    _need(centroids, torch.float32, "centroids", 2)
    _need(assign, torch.int32, "assign", 1)
    h = ctypes.c_void_p()
    _check(lib().adanns_index_create(_ptr(db), db.shape[0], db.shape[1], _ptr(centroids),
                                     centroids.shape[0], centroids.shape[1], _ptr(assign), metric,
                                     storage, _stream(), ctypes.byref(h)))
    return Index(h)


def index_export(index: Index, path: str):
    """Write the index to a file (synchronises)."""
    _check(lib().adanns_index_export(index.handle, os.fsencode(path), _stream()))


def index_import(path: str) -> Index:
    """Load an index written by index_export (synchronises)."""
    h = ctypes.c_void_p()
    _check(lib().adanns_index_import(os.fsencode(path), _stream(), ctypes.byref(h)))
    return Index(h)


class Graph:
    """A low-d proximity graph with the rows for the high-d rerank (library-owned)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        N, d, dg, R, e = (ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(),
                          ctypes.c_int64())
        _check(lib().adanns_graph_info(handle, ctypes.byref(N), ctypes.byref(d), ctypes.byref(dg),
                                       ctypes.byref(R), ctypes.byref(e)))
        self.N, self.d, self.d_g, self.R, self.entry = N.value, d.value, dg.value, R.value, e.value

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("graph already freed")
        return self._h

    def neighbours(self) -> torch.Tensor:
        out = torch.empty(self.N, self.R, dtype=torch.int32, device="cuda")
        _check(lib().adanns_graph_get(self.handle, _ptr(out), _stream()))
        return out

    def free(self):
        if self._h is not None:
            lib().adanns_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def graph_build(db: torch.Tensor, d_g: int, K: int, R: int, alpha: float,
                metric: int = METRIC_L2_PREFIXNORM) -> Graph:
    """AdANNS-DiskANN graph on the d_g prefix (K candidates, R out-degree, prune factor alpha)."""
    _need(db, torch.float32, "db", 2)
    h = ctypes.c_void_p()
    _check(lib().adanns_graph_build(_ptr(db), db.shape[0], db.shape[1], d_g, K, R, float(alpha),
                                    metric, _stream(), ctypes.byref(h)))
    return Graph(h)


def graph_create(db: torch.Tensor, d_g: int, graph: torch.Tensor, entry: int,
                 metric: int = METRIC_L2_PREFIXNORM) -> Graph:
    """A graph from given neighbour lists (int32 [N, R], -1 padding) and entry point."""
    _need(db, torch.float32, "db", 2)
    _need(graph, torch.int32, "graph", 2)
    h = ctypes.c_void_p()
    _check(lib().adanns_graph_create(_ptr(db), db.shape[0], db.shape[1], d_g, _ptr(graph),
                                     graph.shape[1], int(entry), metric, _stream(),
                                     ctypes.byref(h)))
    return Graph(h)


def graph_search(g: Graph, queries: torch.Tensor, L: int, d_s: int, k: int, rerank_k: int,
                 return_shortlist: bool = False):
    """Graph shortlist at d_g, exact rerank at d_s -> (ids, dist[, shortlist])."""
    _need(queries, torch.float32, "queries", 2)
    B = queries.shape[0]
    ids = torch.empty(B, k, dtype=torch.int64, device=queries.device)
    dist = torch.empty(B, k, dtype=torch.float32, device=queries.device)
    sl = torch.empty(B, rerank_k, dtype=torch.int64, device=queries.device) \
        if return_shortlist else None
    _check(lib().adanns_graph_search(g.handle, _ptr(queries), B, L, d_s, k, rerank_k, _ptr(ids),
                                     _ptr(dist), _ptr(sl), _stream()))
    return (ids, dist, sl) if return_shortlist else (ids, dist)


def flat_index(db: torch.Tensor, metric: int = METRIC_L2_PREFIXNORM,
               storage: int = STORE_F32) -> Index:
    """Index whose single list holds every row.  IVF-OPQ search on it (d_c = 8,
    nprobe = 1) is the exhaustive AdANNS-OPQ search of Sec. 4.2 (OPQ on the d_s
    prefix, ADC over all N quantized vectors); the FP32 search is exact brute
    force at d_s."""
    _need(db, torch.float32, "db", 2)
    cent = torch.zeros(1, 8, dtype=torch.float32, device=db.device)
    assign = torch.zeros(db.shape[0], dtype=torch.int32, device=db.device)
    return index_create(db, cent, assign, metric=metric, storage=storage)


def kmeans_assign(points: torch.Tensor, centroids: torch.Tensor, dim: int,
                  metric: int = METRIC_L2_PREFIXNORM):
    """Nearest centroid of each point on the `dim` prefix -> (assign int32, dist f32)."""
    _need(points, torch.float32, "points", 2)
    _need(centroids, torch.float32, "centroids", 2)
    n = points.shape[0]
    a = torch.empty(n, dtype=torch.int32, device=points.device)
    dd = torch.empty(n, dtype=torch.float32, device=points.device)
    _check(lib().adanns_kmeans_assign(_ptr(points), n, points.shape[1], dim, metric,
                                      _ptr(centroids), centroids.shape[0], _ptr(a), _ptr(dd),
                                      _stream()))
    return a, dd


def kmeans_update(points: torch.Tensor, assign: torch.Tensor, centroids: torch.Tensor, dim: int,
                  metric: int = METRIC_L2_PREFIXNORM) -> torch.Tensor:
    """One Lloyd update in place on `centroids` [nc, dim]; returns it."""
    _need(points, torch.float32, "points", 2)
    _need(assign, torch.int32, "assign", 1)
    _need(centroids, torch.float32, "centroids", 2)
    _check(lib().adanns_kmeans_update(_ptr(points), points.shape[0], points.shape[1], dim, metric,
                                      _ptr(assign), centroids.shape[0], _ptr(centroids), _stream()))
    return centroids


def scratch_bytes(index: Index, B: int, d_c: int, d_s: int, nprobe: int, k: int,
                  storage: int = STORE_F32, rerank_k: int = 0) -> int:
    """Upper bound of the device scratch a search with these arguments holds."""
    return int(lib().adanns_search_scratch_bytes(index.handle, B, d_c, d_s, nprobe, k, storage,
                                                 rerank_k))


def search_ivf(index: Index, queries: torch.Tensor, d_c: int, d_s: int, nprobe: int, k: int,
               storage: int = STORE_F32, rerank_k: int = 0, return_probes: bool = False,
               out: tuple | None = None):
    """AdANNS-IVF search -> (ids int64 [B,k], dist f32 [B,k][, probes int32 [B,nprobe]])."""
    _need(queries, torch.float32, "queries", 2)
    if queries.shape[1] != index.d:
        raise ValueError(f"queries must have {index.d} columns")
    B = queries.shape[0]
    if out is None:
        ids = torch.empty(B, k, dtype=torch.int64, device=queries.device)
        dist = torch.empty(B, k, dtype=torch.float32, device=queries.device)
    else:
        ids, dist = out
    probes = torch.empty(B, nprobe, dtype=torch.int32, device=queries.device) if return_probes else None
    _check(lib().adanns_search_ivf(index.handle, _ptr(queries), B, d_c, d_s, nprobe, k, storage,
                                   rerank_k, _ptr(ids), _ptr(dist), _ptr(probes), _stream()))
    return (ids, dist, probes) if return_probes else (ids, dist)


def search_ivf_host(index: Index, queries: torch.Tensor, d_c: int, d_s: int, nprobe: int, k: int,
                    storage: int = STORE_F32, rerank_k: int = 0, out: tuple | None = None,
                    slice_rows: int = 0):
    """AdANNS-IVF search of HOST queries (a CPU float32 tensor) into HOST results
    (ids int64 [B,k], dist f32 [B,k]).  Page-locked buffers (and slice_rows 0)
    are read and written in place by the GPU; others go through copies in
    slices that overlap the neighbouring searches.  Returns when the work is
    queued: synchronise the current stream before reading the results."""
    if not isinstance(queries, torch.Tensor) or queries.is_cuda or queries.dtype != torch.float32:
        raise TypeError("queries must be a CPU float32 tensor")
    if queries.dim() != 2 or queries.shape[1] != index.d or not queries.is_contiguous():
        raise ValueError(f"queries must be contiguous [B, {index.d}]")
    B = queries.shape[0]
    if out is None:
        ids = torch.empty(B, k, dtype=torch.int64, pin_memory=True)
        dist = torch.empty(B, k, dtype=torch.float32, pin_memory=True)
    else:
        ids, dist = out
        if ids.is_cuda or dist.is_cuda:
            raise TypeError("results must be CPU tensors")
    _check(lib().adanns_search_ivf_host(index.handle, _ptr(queries), B, d_c, d_s, nprobe, k,
                                        storage, rerank_k, _ptr(ids), _ptr(dist), slice_rows,
                                        _stream()))
    return ids, dist


def search_ivf_budgets(index: Index, queries: torch.Tensor, d_c: int, d_s, nprobe, k,
                       k_max: int | None = None, storage: int = STORE_F32, rerank_k: int = 0,
                       out: tuple | None = None):
    """AdANNS-IVF search with a budget per query (d_s, nprobe, k: sequences of B
    ints, or one int for all) -> (ids int64 [B,k_max], dist f32 [B,k_max]); row i
    holds query i's k[i] results, then (-1, +inf)."""
    _need(queries, torch.float32, "queries", 2)
    if queries.shape[1] != index.d:
        raise ValueError(f"queries must have {index.d} columns")
    B = queries.shape[0]

    ds_a = _budget_array(d_s, B, "d_s")
    np_a, k_a = _budget_array(nprobe, B, "nprobe"), _budget_array(k, B, "k")
    if k_max is None:
        k_max = max(k_a) if B else 1
    if out is None:
        ids = torch.empty(B, k_max, dtype=torch.int64, device=queries.device)
        dist = torch.empty(B, k_max, dtype=torch.float32, device=queries.device)
    else:
        ids, dist = out
    _check(lib().adanns_search_ivf_budgets(index.handle, _ptr(queries), B, d_c, ds_a, np_a, k_a,
                                           k_max, storage, rerank_k, _ptr(ids), _ptr(dist),
                                           _stream()))
    return ids, dist


def search_ivfopq_budgets(index: Index, queries: torch.Tensor, d_c: int, nprobe, k,
                          k_max: int | None = None, rerank_k: int = 0, out: tuple | None = None):
    """AdANNS-IVFOPQ search with nprobe and k per query (sequences of B ints,
    or one int for all) -> (ids int64 [B,k_max], dist f32 [B,k_max]); row i
    holds query i's k[i] results, then (-1, +inf)."""
    _need(queries, torch.float32, "queries", 2)
    if queries.shape[1] != index.d:
        raise ValueError(f"queries must have {index.d} columns")
    B = queries.shape[0]
    np_a, k_a = _budget_array(nprobe, B, "nprobe"), _budget_array(k, B, "k")
    if k_max is None:
        k_max = max(k_a) if B else 1
    if out is None:
        ids = torch.empty(B, k_max, dtype=torch.int64, device=queries.device)
        dist = torch.empty(B, k_max, dtype=torch.float32, device=queries.device)
    else:
        ids, dist = out
    _check(lib().adanns_search_ivfopq_budgets(index.handle, _ptr(queries), B, d_c, np_a, k_a,
                                              k_max, rerank_k, _ptr(ids), _ptr(dist), _stream()))
    return ids, dist


def _budget_array(v, B: int, what: str):
    """a ctypes int32 array of B entries from one int or a sequence"""
    a = (ctypes.c_int32 * B)()
    if isinstance(v, int):
        for i in range(B):
            a[i] = v
    else:
        v = [int(x) for x in v]
        if len(v) != B:
            raise ValueError(f"{what} needs {B} entries")
        a[:] = v
    return a


# ---------------------------------------------------------------- OPQ / IVF-OPQ
def opq_encode(x: torch.Tensor, d_s: int, M: int, R: torch.Tensor, codebooks: torch.Tensor,
               metric: int = METRIC_L2_PREFIXNORM) -> torch.Tensor:
    """codes uint8 [n, M] of z = P_ds(x) R under the given rotation / codebooks."""
    _need(x, torch.float32, "x", 2)
    _need(R, torch.float32, "R", 2)
    _need(codebooks, torch.float32, "codebooks", 3)
    codes = torch.empty(x.shape[0], M, dtype=torch.uint8, device=x.device)
    _check(lib().adanns_opq_encode(_ptr(x), x.shape[0], x.shape[1], d_s, M, metric, _ptr(R),
                                   _ptr(codebooks), _ptr(codes), _stream()))
    return codes


def pq_update(z: torch.Tensor, codes: torch.Tensor, codebooks: torch.Tensor) -> torch.Tensor:
    """One PQ Lloyd update in place on codebooks [M, 256, d_s/M]; returns it."""
    _need(z, torch.float32, "z", 2)
    _need(codes, torch.uint8, "codes", 2)
    _need(codebooks, torch.float32, "codebooks", 3)
    _check(lib().adanns_pq_update(_ptr(z), z.shape[0], z.shape[1], codes.shape[1], _ptr(codes),
                                  _ptr(codebooks), _stream()))
    return codebooks


def procrustes(Y: torch.Tensor, Zhat: torch.Tensor) -> torch.Tensor:
    """Orthogonal R minimising ||Y R - Zhat||_F (polar factor of Y^T Zhat)."""
    _need(Y, torch.float32, "Y", 2)
    _need(Zhat, torch.float32, "Zhat", 2)
    d = Y.shape[1]
    R = torch.empty(d, d, dtype=torch.float32, device=Y.device)
    _check(lib().adanns_procrustes(_ptr(Y), _ptr(Zhat), Y.shape[0], d, _ptr(R), _stream()))
    return R


def build_opq(index: Index, db: torch.Tensor, d_s: int, M: int, opq_iters: int, pq_iters: int,
              final_iters: int, train_n: int, seed: int) -> list:
    """Train AdANNS-OPQ on the d_s prefix and encode the index; returns the trace."""
    _need(db, torch.float32, "db", 2)
    tr = (ctypes.c_double * max(3 * opq_iters, 1))()
    _check(lib().adanns_build_opq(index.handle, _ptr(db), d_s, M, opq_iters, pq_iters, final_iters,
                                  train_n, seed, tr, _stream()))
    index.opq = (d_s, M)
    return list(tr)


def build_opq_residual(index: Index, db: torch.Tensor, d_s: int, M: int, opq_iters: int,
                       pq_iters: int, final_iters: int, train_n: int, seed: int) -> list:
    """Residual-encoded AdANNS-OPQ: codes of P_ds(x) minus its list's d_s centre."""
    _need(db, torch.float32, "db", 2)
    tr = (ctypes.c_double * max(3 * opq_iters, 1))()
    _check(lib().adanns_build_opq_residual(index.handle, _ptr(db), d_s, M, opq_iters, pq_iters,
                                           final_iters, train_n, seed, tr, _stream()))
    index.opq = (d_s, M)
    return list(tr)


def set_opq_residual(index: Index, d_s: int, M: int, R: torch.Tensor, codebooks: torch.Tensor,
                     codes_by_id: torch.Tensor, list_centres: torch.Tensor):
    """Attach residual OPQ data (codes by database id, list centres [nlist, d_s])."""
    _need(R, torch.float32, "R", 2)
    _need(codebooks, torch.float32, "codebooks", 3)
    _need(codes_by_id, torch.uint8, "codes", 2)
    _need(list_centres, torch.float32, "list_centres", 2)
    _check(lib().adanns_index_set_opq_residual(index.handle, d_s, M, _ptr(R), _ptr(codebooks),
                                               _ptr(codes_by_id), _ptr(list_centres), _stream()))
    index.opq = (d_s, M)


def list_centres(index: Index) -> torch.Tensor:
    """The residual list centres [nlist, d_s] of an index with residual codes."""
    d_s, _ = index.opq
    out = torch.empty(index.nlist, d_s, dtype=torch.float32, device="cuda")
    _check(lib().adanns_index_get_list_centres(index.handle, _ptr(out), _stream()))
    return out


def set_opq(index: Index, d_s: int, M: int, R: torch.Tensor, codebooks: torch.Tensor,
            codes_by_id: torch.Tensor):
    """Attach OPQ data (codes indexed by database id)."""
    _need(R, torch.float32, "R", 2)
    _need(codebooks, torch.float32, "codebooks", 3)
    _need(codes_by_id, torch.uint8, "codes", 2)
    _check(lib().adanns_index_set_opq(index.handle, d_s, M, _ptr(R), _ptr(codebooks),
                                      _ptr(codes_by_id), _stream()))
    index.opq = (d_s, M)


def get_opq(index: Index):
    """(R, codebooks, codes in list order) of the index's OPQ data."""
    d_s, M = index.opq
    R = torch.empty(d_s, d_s, dtype=torch.float32, device="cuda")
    C = torch.empty(M, 256, d_s // M, dtype=torch.float32, device="cuda")
    codes = torch.empty(index.N, M, dtype=torch.uint8, device="cuda")
    _check(lib().adanns_index_get_opq(index.handle, _ptr(R), _ptr(C), _ptr(codes), _stream()))
    return R, C, codes


def search_ivfopq(index: Index, queries: torch.Tensor, d_c: int, nprobe: int, k: int,
                  rerank_k: int = 0, return_probes: bool = False, out: tuple | None = None):
    """AdANNS-IVFOPQ search -> (ids int64 [B,k], dist f32 [B,k][, probes])."""
    _need(queries, torch.float32, "queries", 2)
    if queries.shape[1] != index.d:
        raise ValueError(f"queries must have {index.d} columns")
    B = queries.shape[0]
    if out is None:
        ids = torch.empty(B, k, dtype=torch.int64, device=queries.device)
        dist = torch.empty(B, k, dtype=torch.float32, device=queries.device)
    else:
        ids, dist = out
    probes = torch.empty(B, nprobe, dtype=torch.int32, device=queries.device) if return_probes else None
    _check(lib().adanns_search_ivfopq(index.handle, _ptr(queries), B, d_c, nprobe, k, rerank_k,
                                      _ptr(ids), _ptr(dist), _ptr(probes), _stream()))
    return (ids, dist, probes) if return_probes else (ids, dist)


# ---------------------------------------------------------------- graph plans
class Plan:
    """A fixed-shape search captured into a CUDA graph; `launch()` replays it
    on the current contents of `queries`, writing `ids` / `dist`."""

    def __init__(self, index: Index, queries: torch.Tensor, d_c: int, d_s: int, nprobe: int,
                 k: int, storage: int = STORE_F32, rerank_k: int = 0):
        _need(queries, torch.float32, "queries", 2)
        self.index, self.queries = index, queries
        B = queries.shape[0]
        self.ids = torch.empty(B, k, dtype=torch.int64, device=queries.device)
        self.dist = torch.empty(B, k, dtype=torch.float32, device=queries.device)
        h = ctypes.c_void_p()
        _check(lib().adanns_plan_create(index.handle, _ptr(queries), B, d_c, d_s, nprobe, k,
                                        storage, rerank_k, _ptr(self.ids), _ptr(self.dist),
                                        _stream(), ctypes.byref(h)))
        self._h = h

    def launch(self):
        _check(lib().adanns_plan_launch(self._h, _stream()))
        return self.ids, self.dist

    def free(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.adanns_plan_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- autotuner
def autotune(index: Index, queries: torch.Tensor, d_c: int, d_s: int, nprobe: int, k: int):
    """Time the FP32 list-scan variants on this batch and record the faster
    for its shape bucket; returns (queries per thread, ms per call)."""
    _need(queries, torch.float32, "queries", 2)
    B = queries.shape[0]
    ids = torch.empty(B, k, dtype=torch.int64, device=queries.device)
    dist = torch.empty(B, k, dtype=torch.float32, device=queries.device)
    ch, ms = ctypes.c_int(), ctypes.c_float()
    _check(lib().adanns_autotune_search(index.handle, _ptr(queries), B, d_c, d_s, nprobe, k,
                                        _ptr(ids), _ptr(dist), _stream(), ctypes.byref(ch),
                                        ctypes.byref(ms)))
    return ch.value, ms.value


def autotune_lowp(index: Index, queries: torch.Tensor, d_c: int, d_s: int, nprobe: int, k: int,
                  storage: int, rerank_k: int):
    """Time the BF16 / FP8 tensor-core scan's two tile shapes on this batch
    and record the faster for its bucket; returns (queries per tile: 128 or
    32, ms per call)."""
    _need(queries, torch.float32, "queries", 2)
    B = queries.shape[0]
    ids = torch.empty(B, k, dtype=torch.int64, device=queries.device)
    dist = torch.empty(B, k, dtype=torch.float32, device=queries.device)
    ch, ms = ctypes.c_int(), ctypes.c_float()
    _check(lib().adanns_autotune_search_lowp(index.handle, _ptr(queries), B, d_c, d_s, nprobe, k,
                                             storage, rerank_k, _ptr(ids), _ptr(dist), _stream(),
                                             ctypes.byref(ch), ctypes.byref(ms)))
    return ch.value, ms.value


def tune_save(path: str):
    _check(lib().adanns_tune_save(path.encode()))


def tune_load(path: str):
    _check(lib().adanns_tune_load(path.encode()))


def tune_clear():
    _check(lib().adanns_tune_clear())


# ---------------------------------------------------------------- lists on several GPUs
def map_ids(ids: torch.Tensor, id_map: torch.Tensor) -> torch.Tensor:
    """In place: local row ids of a shard index -> global ids (padding kept)."""
    _need(ids, torch.int64, "ids")
    _need(id_map, torch.int64, "id_map", 1)
    _check(lib().adanns_map_ids(_ptr(id_map), id_map.numel(), _ptr(ids), ids.numel(), _stream()))
    return ids


def merge_shards(ids: torch.Tensor, dist: torch.Tensor, out: tuple | None = None):
    """[G, B, k] per-shard sorted top-k -> merged (ids [B, k], dist [B, k])."""
    _need(ids, torch.int64, "ids", 3)
    _need(dist, torch.float32, "dist", 3)
    if ids.shape != dist.shape:
        raise ValueError("ids and dist must have the same shape")
    G, B, k = ids.shape
    if out is None:
        oi = torch.empty(B, k, dtype=torch.int64, device=ids.device)
        od = torch.empty(B, k, dtype=torch.float32, device=ids.device)
    else:
        oi, od = out
    _check(lib().adanns_merge_shards(_ptr(ids), _ptr(dist), G, B, k, _ptr(oi), _ptr(od),
                                     _stream()))
    return oi, od
