"""The narrow-tile tensor-core scan: when few queries share a probed list, the
BF16 / FP8 scan takes tiles of 128 members x 32 queries (members on the MMA's
M side) instead of 128 queries x 256 members.  It only chooses the shortlist,
so every returned distance must still be the exact FP32 distance of its id,
the ids must reach the oracle's recall, and a shortlist that holds every
candidate must give exactly the wide tiles' result."""
import numpy as np
import pytest

import oracle
import synthdata
from test_gpu_mixed import BF16, FP8, check, cu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import paper_2305_19435_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    return P


@pytest.fixture(scope="module")
def case(A):
    # 48 lists of ~830 members: seven 128-member tiles per list
    data = synthdata.small(40_000, 400, 256, 64, 431)
    o = oracle.build_ivf(data["db"], 32, 48, 8, 20_000, seed=33)
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                       storage=1 | BF16 | FP8)
    yield data, o, g
    g.free()


@pytest.mark.parametrize("storage,d_s,nprobe,k,kr,B", [
    (BF16, 256, 4, 10, 40, 64), (BF16, 64, 8, 100, 400, 33), (BF16, 128, 2, 10, 40, 1),
    (BF16, 256, 4, 50, 200, 250), (FP8, 256, 4, 10, 40, 64), (FP8, 128, 8, 10, 40, 100)])
def test_narrow_scan_matches_oracle(A, case, storage, d_s, nprobe, k, kr, B):
    """Batches with at most 24 queries per probed list on average (B = 250 with
    4 probes over 48 lists gives lists with more than 32 queries, so several
    query tiles per list), narrow tiles forced at these short prefixes: exact
    distances of the returned ids, recall@10."""
    data, o, g = case
    assert B * nprobe <= 24 * 48
    with A.option(A.OPT_NARROW_SCAN, 2):
        check(A, case, storage, d_s, nprobe, k, kr, 0.97 if storage == FP8 else 0.99, B=B)
    g.status()


@pytest.mark.parametrize("storage", [BF16, FP8])
def test_narrow_and_wide_tiles_agree(A, case, storage):
    """The two tile shapes give the same shortlists up to the rounding of the
    tensor cores' dot products: the same ids almost everywhere, the same
    distance bits wherever the ids agree, and, with a shortlist that holds
    every candidate, exactly the same result."""
    data, o, g = case
    q = cu(data["queries"][:96])
    args = (32, 256, 4, 20)
    full = (32, 256, 2, 20)  # two lists of ~830 members: a 2,048 shortlist holds them all
    with A.option(A.OPT_NARROW_SCAN, 0):
        iw, dw = A.search_ivf(g, q, *args, storage=storage, rerank_k=80)
        iwf, dwf = A.search_ivf(g, q, *full, storage=storage, rerank_k=2048)
    with A.option(A.OPT_NARROW_SCAN, 2):
        i_n, d_n = A.search_ivf(g, q, *args, storage=storage, rerank_k=80)
        inf, dnf = A.search_ivf(g, q, *full, storage=storage, rerank_k=2048)
    g.status()
    iw, dw, i_n, d_n = (x.cpu().numpy() for x in (iw, dw, i_n, d_n))
    same = iw == i_n
    assert same.mean() >= 0.99, same.mean()
    assert np.array_equal(dw.view(np.int32)[same], d_n.view(np.int32)[same])
    assert torch.equal(iwf, inf)
    assert torch.equal(dwf.view(torch.int32), dnf.view(torch.int32))


@pytest.fixture(scope="module")
def long_case(A):
    # a 1024-coordinate prefix: 16 BF16 K-blocks, where the narrow tiles are
    # taken by default
    data = synthdata.small(16_000, 200, 1024, 32, 437)
    o = oracle.build_ivf(data["db"], 32, 32, 6, 16_000, seed=35)
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                       storage=1 | BF16 | FP8)
    yield data, o, g
    g.free()


@pytest.mark.parametrize("storage,opt", [(BF16, 1), (FP8, 2)])
def test_narrow_scan_long_prefix(A, long_case, storage, opt):
    """d_s = 1024 with a few queries per list: BF16 on the default rule (16
    K-blocks), FP8 forced (8 K-blocks); exact distances of the returned ids and
    recall@10 against the oracle, and the same result as the wide tiles when
    the shortlist holds every candidate."""
    data, o, g = long_case
    with A.option(A.OPT_NARROW_SCAN, opt):
        check(A, long_case, storage, 1024, 3, 10, 40, 0.97 if storage == FP8 else 0.99, B=120)
        i_n, d_n = A.search_ivf(g, cu(data["queries"][:40]), 32, 1024, 1, 10, storage=storage,
                                rerank_k=2048)
    with A.option(A.OPT_NARROW_SCAN, 0):
        iw, dw = A.search_ivf(g, cu(data["queries"][:40]), 32, 1024, 1, 10, storage=storage,
                              rerank_k=2048)
    g.status()
    sizes = np.diff(o["list_off"])
    assert sizes.max() <= 2048  # one list per query: the shortlist holds every candidate
    assert torch.equal(i_n, iw)
    assert torch.equal(d_n.view(torch.int32), dw.view(torch.int32))


def test_autotune_lowp_records_and_uses_a_tile_shape(A, case, tmp_path):
    """The tile-shape autotuner times both shapes on a batch with few queries
    per probed list and records the faster; later searches in that bucket take
    it, giving exactly the result of the same shape forced by the option, with
    exact distances and the oracle's recall; the table survives a save, clear
    and load."""
    data, o, g = case
    q = cu(data["queries"][:64])
    args = (32, 256, 4, 10)
    chosen = {}
    try:
        for storage in (BF16, FP8):
            qt, ms = A.autotune_lowp(g, q, *args, storage, 40)
            assert qt in (128, 32) and ms > 0
            chosen[storage] = qt
            ti, td = A.search_ivf(g, q, *args, storage=storage, rerank_k=40)
            with A.option(A.OPT_NARROW_SCAN, 2 if qt == 32 else 0):
                fi, fd = A.search_ivf(g, q, *args, storage=storage, rerank_k=40)
            assert torch.equal(ti, fi)
            assert torch.equal(td.view(torch.int32), fd.view(torch.int32))
        # the tuned search against the oracle (exact distances, recall@10)
        check(A, case, BF16, 256, 4, 10, 40, 0.99, B=64)
        path = str(tmp_path / "tune.txt")
        A.tune_save(path)
        lines = open(path).read().split("\n")
        assert any("|lpbf16|ds256|" in l and l.endswith(f" {chosen[BF16]}") for l in lines)
        assert any("|lpfp8|ds256|" in l and l.endswith(f" {chosen[FP8]}") for l in lines)
        A.tune_clear()
        A.tune_load(path)
        ti2, td2 = A.search_ivf(g, q, *args, storage=BF16, rerank_k=40)
        with A.option(A.OPT_NARROW_SCAN, 2 if chosen[BF16] == 32 else 0):
            fi2, fd2 = A.search_ivf(g, q, *args, storage=BF16, rerank_k=40)
        assert torch.equal(ti2, fi2)
        assert torch.equal(td2.view(torch.int32), fd2.view(torch.int32))
        # nothing to tune: a forced shape, or the exact FP32 scan
        with A.option(A.OPT_NARROW_SCAN, 0):
            with pytest.raises(A.AdannsError):
                A.autotune_lowp(g, q, *args, BF16, 40)
        with pytest.raises(A.AdannsError):
            A.autotune_lowp(g, q, *args, 1, 0)
    finally:
        A.tune_clear()  # later modules take the built-in rule
    g.status()
