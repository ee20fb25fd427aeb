"""CUDA-graph search plans and the list-scan autotuner against the oracle."""
import os

import numpy as np
import pytest

import oracle
import synthdata
from parity import ambiguous_probe_rows, check_topk, recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    data = synthdata.small(30_000, 512, 128, 32, 501)
    o = oracle.build_ivf(data["db"], 32, 40, 8, 20_000, seed=23)
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                       storage=3)
    yield data, o, g
    g.free()


def oracle_check(data, o, q, gi, gd, d_s, nprobe, k):
    ref = oracle.search_ivf(data["db"], o, q, 32, d_s, nprobe, k + 24)
    amb = ambiguous_probe_rows(ref["probe_dist"], nprobe)
    n, fails = check_topk(gi, gd, ref["ids"], ref["dist"], k, skip_rows=amb)
    assert n > 0 and not fails, fails[:2]


def test_fp32_plan_replays_search(A, case):
    data, o, g = case
    q = cu(data["queries"][:256])
    plan = A.Plan(g, q, 32, 128, 6, 20)
    ids, dist = plan.launch()
    torch.cuda.synchronize()
    ref_i, ref_d = A.search_ivf(g, q, 32, 128, 6, 20)
    assert torch.equal(ids, ref_i) and torch.equal(dist, ref_d)
    # new contents of the bound query buffer are searched by the same plan
    q.copy_(cu(data["queries"][256:512]))
    ids, dist = plan.launch()
    torch.cuda.synchronize()
    oracle_check(data, o, data["queries"][256:512], ids.cpu().numpy(), dist.cpu().numpy(), 128, 6, 20)
    for _ in range(3):
        plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(plan.ids, ids)
    plan.free()


def test_mixed_plan_replays_search(A, case):
    data, o, g = case
    q = cu(data["queries"])
    plan = A.Plan(g, q, 32, 128, 8, 10, storage=A.STORE_BF16, rerank_k=40)
    ids, dist = plan.launch()
    torch.cuda.synchronize()
    g.status()
    ref = oracle.search_ivf(data["db"], o, data["queries"], 32, 128, 8, 10)
    assert recall(ids.cpu().numpy(), ref["ids"], 10) >= 0.99
    plan.free()


def test_autotune_choice_is_correct_and_used(A, case, tmp_path):
    data, o, g = case
    q = cu(data["queries"])
    tq, ms = A.autotune(g, q, 32, 128, 6, 20)
    assert tq in (1, 4, 16) and ms > 0     # tiled 64- or 16-query items, or the streaming scan
    # the tuned search still matches the oracle
    gi, gd = A.search_ivf(g, q, 32, 128, 6, 20)
    oracle_check(data, o, data["queries"], gi.cpu().numpy(), gd.cpu().numpy(), 128, 6, 20)
    # k above 128: the 16-query tile or the streaming scan
    tq2, _ = A.autotune(g, q[:64], 32, 64, 4, 200)
    assert tq2 in (1, 16)
    path = os.path.join(tmp_path, "tune.txt")
    A.tune_save(path)
    lines = open(path).read().split("\n")
    assert any(l.endswith(f" {tq}") for l in lines if "|k32|ds128|" in l)
    A.tune_load(path)


def test_last_autotune_variant_matches_oracle(A, case):
    """The streaming scan is what autotune runs last; its output is checked."""
    data, o, g = case
    q = cu(data["queries"][:300])
    B = 300
    import ctypes
    ids = torch.empty(B, 50, dtype=torch.int64, device="cuda")
    dist = torch.empty(B, 50, dtype=torch.float32, device="cuda")
    ch, ms = ctypes.c_int(), ctypes.c_float()
    rc = A.lib().adanns_autotune_search(g.handle, ctypes.c_void_p(q.data_ptr()), B, 32, 96, 10, 50,
                                        ctypes.c_void_p(ids.data_ptr()),
                                        ctypes.c_void_p(dist.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                        ctypes.byref(ch), ctypes.byref(ms))
    assert rc == 0
    torch.cuda.synchronize()
    oracle_check(data, o, data["queries"][:300], ids.cpu().numpy(), dist.cpu().numpy(), 96, 10, 50)
