"""Index files: export, import, and the file format against an independent writer.

* A GPU-built index (BF16 and FP8 tiers, OPQ) exported and imported again
  searches bit-identically on every path (FP32, BF16 / FP8 with rerank,
  IVF-OPQ with and without rerank), and its lists, centroids and OPQ data are
  equal.
* The exported file, parsed by tests/indexfile.py, holds the database rows
  exactly and the index's own centroids and lists.
* An index file written by tests/indexfile.py from the FP64 oracle's index and
  OPQ training imports into an index whose searches match the oracle's.
"""
import numpy as np
import pytest

import indexfile
import oracle
import synthdata
from parity import ambiguous_probe_rows, check_topk, full_groups

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BF16, FP8 = 2, 4


@pytest.fixture(scope="module")
def A():
    import paper_2305_19435_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    return P


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def data():
    return synthdata.small(30_000, 300, 256, 48, 601)


def test_export_import_roundtrip(A, data, tmp_path):
    db = cu(data["db"])
    g = A.build_ivf(db, 32, 64, 6, 20_000, 5, storage=1 | BF16 | FP8)
    A.build_opq(g, db, 128, 16, 3, 2, 4, 8_000, 9)
    path = str(tmp_path / "ivf.idx")
    A.index_export(g, path)
    h = A.index_import(path)
    assert (h.N, h.d, h.d_c, h.nlist) == (g.N, g.d, g.d_c, g.nlist)
    for a, b in zip(g.lists(), h.lists()):
        assert torch.equal(a, b)
    assert torch.equal(g.centroids(), h.centroids())
    for a, b in zip(A.get_opq(g), A.get_opq(h)):
        assert torch.equal(a, b)
    q = cu(data["queries"])
    for d_c, d_s, nprobe, k, storage, kr in ((32, 256, 8, 50, 1, 0), (16, 128, 4, 10, BF16, 40),
                                             (32, 256, 12, 100, FP8, 400)):
        i0, d0 = A.search_ivf(g, q, d_c, d_s, nprobe, k, storage=storage, rerank_k=kr)
        i1, d1 = A.search_ivf(h, q, d_c, d_s, nprobe, k, storage=storage, rerank_k=kr)
        assert torch.equal(i0, i1)
        assert torch.equal(d0.view(torch.int32), d1.view(torch.int32))
    for kr in (0, 200):
        i0, d0 = A.search_ivfopq(g, q, 32, 6, 20, rerank_k=kr)
        i1, d1 = A.search_ivfopq(h, q, 32, 6, 20, rerank_k=kr)
        assert torch.equal(i0, i1)
        assert torch.equal(d0.view(torch.int32), d1.view(torch.int32))
    g.status()
    h.status()
    g.free()
    h.free()


def test_exported_file_layout(A, data, tmp_path):
    db = cu(data["db"])
    g = A.build_ivf(db, 16, 40, 3, 10_000, 3, storage=1)
    path = str(tmp_path / "plain.idx")
    A.index_export(g, path)
    f = indexfile.read(path)
    assert f["magic"] == b"ADANNSIX" and f["version"] == 1 and f["trailing_bytes"] == 0
    assert (f["N"], f["d"], f["d_c"], f["nlist"], f["metric"], f["storage"]) == \
        (30_000, 256, 16, 40, 1, 1)
    assert f["opq_M"] == 0
    assert np.array_equal(f["rows"], data["db"])          # the rows come back exactly
    assert np.array_equal(f["centroids"], g.centroids().cpu().numpy())
    off, ids = (t.cpu().numpy() for t in g.lists())
    lists = np.repeat(np.arange(40), np.diff(off))
    assert np.array_equal(f["assign"][ids], lists)
    g.free()


def test_import_of_an_oracle_index_file(A, data, tmp_path):
    """The file written independently from the oracle's index and OPQ: the
    imported index searches like the oracle (FP32 IVF and IVF-OPQ)."""
    o = oracle.build_ivf(data["db"], 32, 48, 6, 20_000, seed=13)
    opq = oracle.train_opq(data["db"], 64, 16, 2, 2, 4, 6_000, seed=17)
    codes = oracle.pq_encode(data["db"], 64, 16, opq["R"], opq["codebooks"])
    path = str(tmp_path / "oracle.idx")
    indexfile.write(path, o["centroids"], o["assign"], data["db"], storage=1,
                    opq={"R": opq["R"], "codebooks": opq["codebooks"], "codes": codes})
    h = A.index_import(path)
    q = data["queries"]
    k, nprobe = 20, 6
    gi, gd = A.search_ivf(h, cu(q), 32, 128, nprobe, k)
    ref = full_groups(oracle.search_ivf(data["db"], o, q, 32, 128, nprobe, k + 24),
                      lambda r, kk: oracle.search_ivf(data["db"], o, q[r], 32, 128, nprobe, kk), k)
    amb = ambiguous_probe_rows(ref["probe_dist"], nprobe)
    n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), ref["ids"], ref["dist"], k,
                          skip_rows=amb)
    assert n > 250 and not fails, fails[:2]
    gi, gd = A.search_ivfopq(h, cu(q), 32, nprobe, k)
    ref = oracle.search_ivfopq(data["db"], o, opq, codes, q, 32, nprobe, k)
    n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), ref["ids"], ref["dist"], k,
                          skip_rows=ambiguous_probe_rows(ref["probe_dist"], nprobe))
    assert n > 250 and not fails, fails[:2]
    h.free()


def test_import_rejects_truncated_file(A, data, tmp_path):
    o = oracle.build_ivf(data["db"][:2000], 16, 8, 2, 2000, seed=3)
    path = tmp_path / "cut.idx"
    indexfile.write(str(path), o["centroids"], o["assign"], data["db"][:2000])
    raw = path.read_bytes()
    path.write_bytes(raw[:-100])
    with pytest.raises(A.AdannsError) as e:
        A.index_import(str(path))
    assert e.value.code == -6
    path.write_bytes(raw + b"x")
    with pytest.raises(A.AdannsError) as e:
        A.index_import(str(path))
    assert e.value.code == -6


def test_residual_index_file_roundtrip_and_oracle_import(A, data, tmp_path):
    """Residual codes survive export / import (flag bit and list centres), and
    an independently written residual file imports into an index whose search
    matches the oracle's."""
    o = oracle.build_ivf(data["db"], 32, 48, 6, 20_000, seed=13)
    lc = oracle.list_centroids(data["db"], o, 64)
    opq = oracle.train_opq(data["db"], 64, 16, 2, 2, 4, 6_000, seed=19,
                           residual={"lcent": lc, "assign": o["assign"]})
    codes = oracle.pq_encode(data["db"], 64, 16, opq["R"], opq["codebooks"], lcent=lc,
                             assign=o["assign"])
    path = str(tmp_path / "res.idx")
    indexfile.write(path, o["centroids"], o["assign"], data["db"],
                    opq={"R": opq["R"], "codebooks": opq["codebooks"], "codes": codes, "lcent": lc})
    h = A.index_import(path)
    q = data["queries"]
    gi, gd = A.search_ivfopq(h, cu(q), 32, 6, 20)
    ref = oracle.search_ivfopq(data["db"], o, opq, codes, q, 32, 6, 20)
    n, fails = check_topk(gi.cpu().numpy(), gd.cpu().numpy(), ref["ids"], ref["dist"], 20,
                          skip_rows=ambiguous_probe_rows(ref["probe_dist"], 6))
    assert n > 250 and not fails, fails[:2]
    path2 = str(tmp_path / "res2.idx")
    A.index_export(h, path2)
    f = indexfile.read(path2)
    assert f["opq_flags"] == 1 and np.array_equal(f["lcent"], lc) and f["trailing_bytes"] == 0
    h2 = A.index_import(path2)
    i2, d2 = A.search_ivfopq(h2, cu(q), 32, 6, 20)
    i1, d1 = A.search_ivfopq(h, cu(q), 32, 6, 20)
    assert torch.equal(i1, i2) and torch.equal(d1.view(torch.int32), d2.view(torch.int32))
    h.free()
    h2.free()
