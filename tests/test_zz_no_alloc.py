"""The allocation-free search entry point (adanns_search_ivf_noalloc).

It serves callers that cannot allocate device memory during a search (a
framework that owns the whole memory budget, a latency-critical serving
loop).  Called through the C ABI, its results must equal those of
adanns_search_ivf on the same index and queries, on two calls in a row (the
shared scratch array keeps the previous call's contents), and a request
larger than its fixed scratch must be refused with an error.  This file is
collected last so that a failure here leaves the rest of the suite already
run.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synthdata
from parity import check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2305_19435_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    L = P.lib()
    fn = L.adanns_search_ivf_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                   ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    data = synthdata.small(20_000, 600, 128, 32, 707)
    o = oracle.build_ivf(data["db"], 32, 64, 8, 20_000, seed=11)
    idx = P.index_create(torch.from_numpy(data["db"]).cuda(),
                         torch.from_numpy(o["centroids"]).cuda(),
                         torch.from_numpy(o["assign"].astype(np.int32)).cuda())
    yield P, L, fn, data, idx
    idx.free()


def call_noalloc(fn, idx, q, d_c, d_s, nprobe, k):
    B = q.shape[0]
    ids = torch.full((B, k), -7, dtype=torch.int64, device="cuda")
    dist = torch.full((B, k), -7.0, dtype=torch.float32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(idx.handle, ctypes.c_void_p(q.data_ptr()), B, d_c, d_s, nprobe, k,
            ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dist.data_ptr()), st)
    return rc, ids, dist


def same_within_tolerance(ids, dist, ref_ids, ref_dist, k):
    """The parity rule of the oracle comparison, with adanns_search_ivf's
    result as the reference: distances within the FP32 tolerance, ids equal
    outside tie groups and set-equal inside them."""
    n, fails = check_topk(ids, dist, ref_ids, ref_dist.astype(np.float64), k)
    assert n == ids.shape[0] and not fails, fails[:2]


# (d_s, nprobe, k): the second call has other sizes, so it meets the first
# call's leftovers in the shared array; nprobe = 40 is above the register
# top-k of the fast cluster-mapping kernel, so the general scan maps the queries
@pytest.mark.parametrize("first,second", [((128, 8, 50), (64, 4, 10)),
                                          ((96, 40, 20), (128, 8, 50))])
def test_noalloc_matches_allocating_search_twice(setup, first, second):
    P, L, fn, data, idx = setup
    qa = torch.from_numpy(data["queries"][:300]).cuda()
    qb = torch.from_numpy(data["queries"][300:]).cuda()
    for q, (d_s, nprobe, k) in ((qa, first), (qb, second)):
        rc, ids, dist = call_noalloc(fn, idx, q, 32, d_s, nprobe, k)
        assert rc == 0, L.adanns_last_error()
        ref_ids, ref_dist = P.search_ivf(idx, q, 32, d_s, nprobe, k)
        torch.cuda.synchronize()
        same_within_tolerance(ids.cpu().numpy(), dist.cpu().numpy(), ref_ids.cpu().numpy(),
                              ref_dist.cpu().numpy(), k)


def test_noalloc_takes_no_device_memory(setup):
    """After a first call (which loads the kernels' code), further calls leave
    the device's free memory unchanged: no allocation, no pool growth."""
    P, L, fn, data, idx = setup
    q = torch.from_numpy(data["queries"]).cuda()
    ids = torch.empty(q.shape[0], 50, dtype=torch.int64, device="cuda")
    dist = torch.empty(q.shape[0], 50, dtype=torch.float32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(nprobe):
        rc = fn(idx.handle, ctypes.c_void_p(q.data_ptr()), q.shape[0], 32, 128, nprobe, 50,
                ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dist.data_ptr()), st)
        assert rc == 0, L.adanns_last_error()

    for nprobe in (8, 40):
        call(nprobe)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for nprobe in (8, 40, 8):
        call(nprobe)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_refuses_requests_beyond_its_scratch(setup):
    P, L, fn, data, idx = setup
    q = torch.from_numpy(np.repeat(data["queries"], 20, axis=0)).cuda()   # 12,000 queries
    rc, ids, _ = call_noalloc(fn, idx, q, 32, 128, 64, 100)
    assert rc == -1
    assert b"scratch" in L.adanns_last_error()
    torch.cuda.synchronize()
    assert bool((ids == -7).all())        # nothing was launched
