"""GPU-vs-oracle parity for AdANNS-OPQ and AdANNS-IVFOPQ.

Encoding, the PQ update and the Procrustes step are teacher-forced from the
oracle's values; the search runs on the oracle's index and OPQ data imported
to the GPU, so both sides look up the same codes.
"""
import numpy as np
import pytest

import oracle
import synthdata
from parity import ambiguous_probe_rows, check_topk, recall, tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PN = oracle.METRIC_L2_PREFIXNORM


@pytest.fixture(scope="module")
def A():
    import paper_2305_19435_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    return P


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def case():
    data = synthdata.small(12_000, 300, 96, 48, 301)
    db = data["db"]
    idx = oracle.build_ivf(db, 32, 24, 6, 12_000, seed=9)
    out = {"data": data, "idx": idx}
    for d_s, M in ((64, 16), (96, 32), (48, 16), (32, 4)):
        opq = oracle.train_opq(db, d_s, M, 3, 3, 5, 4000, seed=13)
        codes = oracle.pq_encode(db, d_s, M, opq["R"], opq["codebooks"])
        out[(d_s, M)] = (opq, codes)
    return out


def gpu_index(A, case, d_s, M):
    data, o = case["data"], case["idx"]
    opq, codes = case[(d_s, M)]
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)))
    A.set_opq(g, d_s, M, cu(opq["R"]), cu(opq["codebooks"]), cu(codes))
    return g


@pytest.mark.parametrize("d_s,M", [(64, 16), (96, 32), (48, 16), (32, 4)])
def test_encode_matches_oracle(A, case, d_s, M):
    db = case["data"]["db"][:3000]
    opq, codes = case[(d_s, M)]
    got = A.opq_encode(cu(db), d_s, M, cu(opq["R"]), cu(opq["codebooks"])).cpu().numpy()
    Z = oracle.prefix(db, d_s) @ opq["R"].astype(np.float64)
    C = opq["codebooks"].astype(np.float64)
    dsub = d_s // M
    for m in range(M):
        D = ((Z[:, None, m * dsub:(m + 1) * dsub] - C[m][None]) ** 2).sum(-1)
        srt = np.sort(D, axis=1)
        tied = srt[:, 1] - srt[:, 0] <= tol(srt[:, 1])
        assert tied.mean() < 0.01
        assert np.array_equal(got[~tied, m], codes[:3000][~tied, m]), m


def test_pq_update_matches_oracle(A, case):
    opq, codes = case[(64, 16)]
    db = case["data"]["db"][:5000]
    Z = (oracle.prefix(db, 64) @ opq["R"].astype(np.float64)).astype(np.float32)
    C0 = opq["codebooks"].copy()
    got = A.pq_update(cu(Z), cu(codes[:5000]), cu(C0.copy())).cpu().numpy()
    for m in range(16):
        want = oracle.update(Z[:, 4 * m:4 * m + 4].astype(np.float64), codes[:5000, m].astype(np.int32),
                             C0[m].astype(np.float64))
        assert np.all(np.abs(got[m] - want) <= 1e-6 * np.abs(want) + 1e-8)


def test_procrustes_matches_oracle(A):
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((4096, 48)) * np.linspace(1.0, 0.3, 48)
    Q = np.linalg.qr(rng.standard_normal((48, 48)))[0]
    Zh = Y @ Q + 0.05 * rng.standard_normal((4096, 48))
    Y32, Z32 = Y.astype(np.float32), Zh.astype(np.float32)
    R = A.procrustes(cu(Y32), cu(Z32)).cpu().numpy().astype(np.float64)
    Ro = oracle.procrustes(Y32.astype(np.float64), Z32.astype(np.float64))
    assert np.abs(R.T @ R - np.eye(48)).max() < 1e-5
    assert np.abs(R - Ro).max() < 1e-4
    fo = ((Y32 @ Ro - Z32) ** 2).sum()
    fg = ((Y32 @ R - Z32) ** 2).sum()
    assert abs(fg - fo) <= 1e-6 * fo


@pytest.mark.parametrize("d_s,M,nprobe,k,d_c", [(64, 16, 4, 20, 32), (96, 32, 8, 100, 32),
                                                (48, 16, 2, 10, 32), (32, 4, 24, 50, 32),
                                                (64, 16, 4, 20, 16), (96, 32, 8, 10, 8)])
def test_ivfopq_search_parity(A, case, d_s, M, nprobe, k, d_c):
    """d_c below the built 32 is the IVF-D coarse step in front of the ADC scan."""
    data, o = case["data"], case["idx"]
    opq, codes = case[(d_s, M)]
    g = gpu_index(A, case, d_s, M)
    q = data["queries"]
    gi, gd, gp = A.search_ivfopq(g, cu(q), d_c, nprobe, k, return_probes=True)
    gi, gd, gp = gi.cpu().numpy(), gd.cpu().numpy(), gp.cpu().numpy()
    orr = oracle.search_ivfopq(data["db"], o, opq, codes, q, d_c, nprobe, k + 40)
    amb = ambiguous_probe_rows(orr["probe_dist"], nprobe)
    for i in np.nonzero(~amb)[0]:
        assert set(gp[i]) == set(orr["probes"][i])
    n, fails = check_topk(gi, gd, orr["ids"], orr["dist"], k, skip_rows=amb)
    assert not fails, f"{len(fails)}/{n}: {fails[:2]}"
    g.free()


@pytest.mark.parametrize("d_s,M,nprobe,k,kr", [(64, 16, 4, 10, 40), (96, 32, 8, 20, 80),
                                               (32, 4, 2, 10, 2048)])
def test_ivfopq_rerank_parity(A, case, d_s, M, nprobe, k, kr):
    data, o = case["data"], case["idx"]
    opq, codes = case[(d_s, M)]
    g = gpu_index(A, case, d_s, M)
    q = data["queries"]
    gi, gd = A.search_ivfopq(g, cu(q), 32, nprobe, k, rerank_k=kr)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    orr = oracle.search_ivfopq(data["db"], o, opq, codes, q, 32, nprobe, k + 20, rerank_k=kr)
    adc = oracle.search_ivfopq(data["db"], o, opq, codes, q, 32, nprobe, kr + 1)
    # the shortlist is ambiguous when the ADC scores at ranks kr-1 and kr are
    # nearly but not exactly equal (identical codes tie exactly on both sides
    # and are ordered by id on both)
    a, b = adc["dist"][:, kr - 1], adc["dist"][:, kr]
    near = np.isfinite(b) & (b - a > 0) & (b - a <= tol(b))
    amb = ambiguous_probe_rows(adc["probe_dist"], nprobe) | near
    n, fails = check_topk(gi, gd, orr["ids"], orr["dist"], k, skip_rows=amb)
    assert n > 0.8 * len(q)
    assert not fails, f"{len(fails)}/{n}: {fails[:2]}"
    # reranking every candidate equals the exact IVF search
    if kr >= 2048:
        exact = oracle.search_ivf(data["db"], o, q, 32, d_s, nprobe, k + 20)
        n, fails = check_topk(gi, gd, exact["ids"], exact["dist"], k, skip_rows=amb)
        assert not fails
    g.free()


def test_build_opq_trace_and_codes(A, case):
    data, o = case["data"], case["idx"]
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)))
    tr = np.array(A.build_opq(g, cu(data["db"]), 64, 16, 3, 3, 5, 4000, 13))
    opq, _ = case[(64, 16)]
    to = np.array(opq["trace"])
    assert tr.shape == to.shape
    assert np.all(tr[1:] <= tr[:-1] * (1 + 1e-5))
    assert abs(tr[0] - to[0]) <= 1e-4 * to[0]          # same sample, same init
    assert abs(tr[-1] - to[-1]) <= 2e-2 * to[-1]        # free-running: close, not equal
    R, C, codes_lo = A.get_opq(g)
    R = R.cpu().numpy().astype(np.float64)
    assert np.abs(R.T @ R - np.eye(64)).max() < 1e-5
    # the stored codes are the nearest codewords under the GPU's own R, C
    off, ids = g.lists()
    ids = ids.cpu().numpy()
    sub = ids[:2000]
    Z = oracle.prefix(data["db"][sub], 64) @ R
    Cg = C.cpu().numpy().astype(np.float64)
    cl = codes_lo.cpu().numpy()[:2000]
    for m in range(16):
        D = ((Z[:, None, 4 * m:4 * m + 4] - Cg[m][None]) ** 2).sum(-1)
        srt = np.sort(D, axis=1)
        tied = srt[:, 1] - srt[:, 0] <= tol(srt[:, 1])
        assert np.array_equal(cl[~tied, m], np.argmin(D, axis=1)[~tied])
    # and the GPU-trained index searches close to the oracle-trained one
    gi, _ = A.search_ivfopq(g, cu(data["queries"]), 32, 8, 10, rerank_k=100)
    exact = oracle.search_ivf(data["db"], o, data["queries"], 32, 64, 8, 10)
    assert recall(gi.cpu().numpy(), exact["ids"], 10) > 0.9
    g.free()


def test_opq_errors(A, case):
    data, o = case["data"], case["idx"]
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)))
    q = cu(data["queries"][:4])
    with pytest.raises(A.AdannsError) as e:
        A.search_ivfopq(g, q, 32, 4, 10)         # no OPQ data yet
    assert e.value.code == -6
    opq, codes = case[(64, 16)]
    with pytest.raises(A.AdannsError) as e:
        A.set_opq(g, 64, 7, cu(opq["R"]), cu(opq["codebooks"]), cu(codes))   # M does not divide
    assert e.value.code == -1
    A.set_opq(g, 64, 16, cu(opq["R"]), cu(opq["codebooks"]), cu(codes))
    with pytest.raises(A.AdannsError) as e:
        A.search_ivfopq(g, q, 32, 4, 10, rerank_k=5)   # shortlist shorter than k
    assert e.value.code == -1
    g.free()


def _search_both(A, g, q, d_c, nprobe, k, kr=0):
    """The same IVF-OPQ search through the distance-then-select ADC stage and
    through the running per-(query, list) top-k ADC stage."""
    a = [t.cpu().numpy() for t in A.search_ivfopq(g, q, d_c, nprobe, k, rerank_k=kr)]
    with A.option(A.OPT_ADC_SELECT, 0):
        b = [t.cpu().numpy() for t in A.search_ivfopq(g, q, d_c, nprobe, k, rerank_k=kr)]
    return a, b


@pytest.mark.parametrize("d_s,M,nprobe,k,kr", [(64, 16, 24, 10, 0), (64, 16, 24, 100, 0),
                                               (96, 32, 20, 10, 400), (32, 4, 24, 50, 2000),
                                               (48, 16, 3, 20, 0), (64, 16, 1, 10, 700)])
def test_adc_select_equals_running_topk(A, case, d_s, M, nprobe, k, kr):
    """Both ADC stages score members with the same FP32 arithmetic and keep
    the best by (score, id), so ids and distances agree bit for bit: sampled
    threshold + buffer select (24 lists of ~500), the whole-region select
    (few lists), and k' at or above the probed members."""
    g = gpu_index(A, case, d_s, M)
    (ai, ad), (bi, bd) = _search_both(A, g, cu(case["data"]["queries"]), 32, nprobe, k, kr)
    assert np.array_equal(ai, bi)
    assert np.array_equal(ad.view(np.uint32), bd.view(np.uint32))
    g.free()


@pytest.fixture(scope="module")
def dup_case():
    """1,200 copies of one vector (identical codes, so exactly equal ADC
    scores) in a 12k database; queries are that vector plus small noise."""
    data = synthdata.small(12_000, 40, 96, 48, 303)
    db = data["db"].copy()
    rng = np.random.default_rng(5)
    dup = np.sort(rng.choice(12_000, 1_200, replace=False))
    db[dup] = db[dup[0]]
    q = (db[dup[0]][None, :] + 1e-3 * rng.standard_normal((40, 96))).astype(np.float32)
    idx = oracle.build_ivf(db, 32, 24, 6, 12_000, seed=9)
    opq = oracle.train_opq(db, 64, 16, 3, 3, 5, 4000, seed=13)
    codes = oracle.pq_encode(db, 64, 16, opq["R"], opq["codebooks"])
    return {"db": db, "q": q, "dup": dup, "idx": idx, "opq": opq, "codes": codes}


@pytest.mark.parametrize("nprobe,k,kr", [(24, 100, 0), (24, 10, 1000), (2, 300, 0),
                                         (24, 1000, 0)])
def test_adc_select_tie_rule(A, dup_case, nprobe, k, kr):
    """The cut falls inside a group of >512 exactly equal scores (the second,
    id-keyed radix select, in the shared buffer and over the whole region):
    the group's smallest ids are kept, as the oracle's (score, id) order
    does."""
    c = dup_case
    g = A.index_create(cu(c["db"]), cu(c["idx"]["centroids"]),
                       cu(c["idx"]["assign"].astype(np.int32)))
    A.set_opq(g, 64, 16, cu(c["opq"]["R"]), cu(c["opq"]["codebooks"]), cu(c["codes"]))
    q = cu(c["q"])
    kk = kr or k
    (ai, ad), (bi, bd) = _search_both(A, g, q, 32, nprobe, k, kr)
    assert np.array_equal(ai, bi)
    assert np.array_equal(ad.view(np.uint32), bd.view(np.uint32))
    orr = oracle.search_ivfopq(c["db"], c["idx"], c["opq"], c["codes"], c["q"], 32, nprobe,
                               kk + 20)
    dupset = set(c["dup"].tolist())
    for i in range(len(c["q"])):
        if kr == 0:
            # the duplicates returned are the smallest ids of the group
            got = sorted(x for x in ai[i].tolist() if x in dupset)
            assert got == sorted(c["dup"].tolist())[:len(got)]
            want = [x for x in orr["ids"][i, :k].tolist() if x in dupset]
            assert len(got) == len(want)
    if kr == 0:
        amb = ambiguous_probe_rows(orr["probe_dist"], nprobe)
        n, fails = check_topk(ai, ad, orr["ids"], orr["dist"], k, skip_rows=amb)
        assert not fails, f"{len(fails)}/{n}: {fails[:2]}"
    g.free()


@pytest.mark.parametrize("d_s,M,opq_iters", [(64, 16, 3), (32, 8, 3), (96, 32, 2), (64, 16, 0),
                                             (48, 8, 0)])
def test_flat_opq_exhaustive_parity(A, case, d_s, M, opq_iters):
    """Exhaustive AdANNS-OPQ (Sec. 4.2: OPQ on the d_s prefix, ADC over every
    quantized vector) as IVF-OPQ over an index with one list; opq_iters = 0 is
    plain PQ (identity rotation).  Against the oracle's ADC over the same
    one-list index and the same codes, at byte budgets 8 to 32."""
    data = case["data"]
    db, q = data["db"], data["queries"]
    N = db.shape[0]
    opq = oracle.train_opq(db, d_s, M, opq_iters, 3, 5, 4000, seed=21)
    if opq_iters == 0:
        assert np.array_equal(opq["R"], np.eye(d_s, dtype=np.float32))
    codes = oracle.pq_encode(db, d_s, M, opq["R"], opq["codebooks"])
    one = {"centroids": np.zeros((1, 8), np.float32), "list_off": np.array([0, N], np.int64),
           "list_ids": np.arange(N, dtype=np.int32), "assign": np.zeros(N, np.int32),
           "metric": PN}
    g = A.flat_index(cu(db))
    A.set_opq(g, d_s, M, cu(opq["R"]), cu(opq["codebooks"]), cu(codes))
    for k in (10, 100):
        gi, gd = A.search_ivfopq(g, cu(q), 8, 1, k)
        orr = oracle.search_ivfopq(db, one, opq, codes, q, 8, 1, k + 40)
        n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), orr["ids"], orr["dist"], k)
        assert n == len(q)
        assert not fails, f"{len(fails)}/{n}: {fails[:2]}"
    g.free()


def test_flat_index_fp32_is_brute_force(A, case):
    """The FP32 search over the one-list index is exact brute force at d_s."""
    data = case["data"]
    db, q = data["db"], data["queries"][:64]
    N = db.shape[0]
    one = {"centroids": np.zeros((1, 8), np.float32), "list_off": np.array([0, N], np.int64),
           "list_ids": np.arange(N, dtype=np.int32), "assign": np.zeros(N, np.int32),
           "metric": PN}
    g = A.flat_index(cu(db))
    gi, gd = A.search_ivf(g, cu(q), 8, 64, 1, 20)
    exact = oracle.search_ivf(db, one, q, 8, 64, 1, 40)   # one list: brute force
    n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), exact["ids"], exact["dist"], 20)
    assert n == len(q) and not fails, fails[:2]
    g.free()


# ---------------------------------------------------------------- residual codes
@pytest.fixture(scope="module")
def res_case(case):
    data, o = case["data"], case["idx"]
    db = data["db"]
    out = {}
    for d_s, M in ((64, 16), (96, 32), (32, 4)):
        lc = oracle.list_centroids(db, o, d_s)
        opq = oracle.train_opq(db, d_s, M, 3, 3, 5, 4000, seed=17,
                               residual={"lcent": lc, "assign": o["assign"]})
        codes = oracle.pq_encode(db, d_s, M, opq["R"], opq["codebooks"], lcent=lc,
                                 assign=o["assign"])
        out[(d_s, M)] = (opq, codes, lc)
    return out


def gpu_res_index(A, case, res_case, d_s, M):
    data, o = case["data"], case["idx"]
    opq, codes, lc = res_case[(d_s, M)]
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)))
    A.set_opq_residual(g, d_s, M, cu(opq["R"]), cu(opq["codebooks"]), cu(codes), cu(lc))
    return g


@pytest.mark.parametrize("d_s,M,nprobe,k,d_c", [(64, 16, 4, 20, 32), (96, 32, 8, 100, 32),
                                                (32, 4, 24, 50, 32), (64, 16, 6, 10, 16)])
def test_residual_ivfopq_search_parity(A, case, res_case, d_s, M, nprobe, k, d_c):
    """Residual codes: one table per (query, probed list) built from
    (P_ds(q) - lcent[l]) R on the oracle's side, the list table S_l and the
    constant |w_l|^2 - 2 <w_l, z_q> on the GPU's; scores and ids agree."""
    data, o = case["data"], case["idx"]
    opq, codes, lc = res_case[(d_s, M)]
    g = gpu_res_index(A, case, res_case, d_s, M)
    q = data["queries"]
    gi, gd = A.search_ivfopq(g, cu(q), d_c, nprobe, k)
    orr = oracle.search_ivfopq(data["db"], o, opq, codes, q, d_c, nprobe, k + 40)
    amb = ambiguous_probe_rows(orr["probe_dist"], nprobe)
    n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), orr["ids"], orr["dist"], k,
                          skip_rows=amb)
    assert n > 0.8 * len(q) and not fails, f"{len(fails)}/{n}: {fails[:2]}"
    # the list centres round-trip
    assert torch.equal(A.list_centres(g).cpu(), torch.from_numpy(lc))
    g.free()


@pytest.mark.parametrize("d_s,M,nprobe,k,kr", [(64, 16, 4, 10, 40), (32, 4, 2, 10, 2048)])
def test_residual_ivfopq_rerank_parity(A, case, res_case, d_s, M, nprobe, k, kr):
    data, o = case["data"], case["idx"]
    opq, codes, lc = res_case[(d_s, M)]
    g = gpu_res_index(A, case, res_case, d_s, M)
    q = data["queries"]
    gi, gd = A.search_ivfopq(g, cu(q), 32, nprobe, k, rerank_k=kr)
    orr = oracle.search_ivfopq(data["db"], o, opq, codes, q, 32, nprobe, k + 20, rerank_k=kr)
    adc = oracle.search_ivfopq(data["db"], o, opq, codes, q, 32, nprobe, kr + 1)
    a, b = adc["dist"][:, kr - 1], adc["dist"][:, kr]
    near = np.isfinite(b) & (b - a > 0) & (b - a <= tol(b))
    amb = ambiguous_probe_rows(adc["probe_dist"], nprobe) | near
    n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), orr["ids"], orr["dist"], k,
                          skip_rows=amb)
    assert n > 0.8 * len(q) and not fails, f"{len(fails)}/{n}: {fails[:2]}"
    g.free()


def test_residual_build_on_gpu(A, case):
    """The GPU residual trainer: its list centres are the oracle's list means
    of the same lists, the distortion trace does not increase, and residual
    codes quantise better than plain codes of the same byte budget."""
    data, o = case["data"], case["idx"]
    db = cu(data["db"])
    g = A.index_create(db, cu(o["centroids"]), cu(o["assign"].astype(np.int32)))
    tr = A.build_opq_residual(g, db, 64, 8, 3, 3, 5, 6000, 21)
    lc = A.list_centres(g).cpu().numpy()
    ref = oracle.list_centroids(data["db"], o, 64)
    assert np.allclose(lc, ref, rtol=1e-5, atol=1e-6)
    tr = np.array(tr)
    assert np.all(np.diff(tr) <= 1e-6 * tr[:-1] + 1e-9), tr
    h = A.index_create(db, cu(o["centroids"]), cu(o["assign"].astype(np.int32)))
    tr0 = np.array(A.build_opq(h, db, 64, 8, 3, 3, 5, 6000, 21))
    assert tr[-1] < tr0[-1]
    # both searchable; residual recall against exact IVF at least that of plain codes
    q = cu(data["queries"])
    ex = oracle.search_ivf(data["db"], o, data["queries"], 32, 64, 6, 10)
    r1 = recall(A.search_ivfopq(g, q, 32, 6, 10)[0].cpu().numpy(), ex["ids"], 10)
    r0 = recall(A.search_ivfopq(h, q, 32, 6, 10)[0].cpu().numpy(), ex["ids"], 10)
    assert r1 >= r0 - 0.02, (r1, r0)
    g.free()
    h.free()
