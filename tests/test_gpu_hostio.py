"""Search of host queries into host results (adanns_search_ivf_host): the batch
runs in slices whose copies overlap the neighbouring searches, and every row
equals the device-memory search of the same rows (ids and distance bits)."""
import numpy as np
import pytest

import oracle
import synthdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2305_19435_gb300 as P
    P.build()
    data = synthdata.small(20_000, 1000, 256, 64, 901)
    o = oracle.build_ivf(data["db"], 32, 48, 5, 20_000, seed=3)
    g = P.index_create(torch.from_numpy(data["db"]).cuda(), torch.from_numpy(o["centroids"]).cuda(),
                       torch.from_numpy(o["assign"].astype(np.int32)).cuda(),
                       storage=1 | P.STORE_BF16)
    yield P, data, g
    g.free()


@pytest.mark.parametrize("tier", ["f32", "bf16"])
@pytest.mark.parametrize("slice_rows", [0, 97, 1000, 4096])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_search_equals_device_search(setup, tier, slice_rows, pinned):
    P, data, g = setup
    q = torch.from_numpy(data["queries"])
    if pinned:
        q = q.pin_memory()
    st, rr = (P.STORE_F32, 0) if tier == "f32" else (P.STORE_BF16, 80)
    di, dd = P.search_ivf(g, q.cuda(), 32, 256, 6, 20, storage=st, rerank_k=rr)
    ids = torch.empty(len(q), 20, dtype=torch.int64, pin_memory=pinned)
    dist = torch.empty(len(q), 20, dtype=torch.float32, pin_memory=pinned)
    P.search_ivf_host(g, q, 32, 256, 6, 20, storage=st, rerank_k=rr, out=(ids, dist),
                      slice_rows=slice_rows)
    torch.cuda.synchronize()
    assert np.array_equal(ids.numpy(), di.cpu().numpy())
    assert np.array_equal(dist.numpy().view(np.int32), dd.cpu().numpy().view(np.int32))


def test_host_search_arguments(setup):
    P, data, g = setup
    q = torch.from_numpy(data["queries"][:8]).pin_memory()
    with pytest.raises(P.AdannsError) as e:
        P.search_ivf_host(g, q, 32, 100, 6, 20)           # d_s not a granularity
    assert e.value.code == -2
    with pytest.raises(P.AdannsError) as e:
        P.search_ivf_host(g, q, 32, 256, 6, 20, storage=P.STORE_BF16, rerank_k=10)
    assert e.value.code == -1
    with pytest.raises(TypeError):
        P.search_ivf_host(g, q.cuda(), 32, 256, 6, 20)    # device queries
    ids, dist = P.search_ivf_host(g, q[:0], 32, 256, 6, 20)
    torch.cuda.synchronize()
    assert ids.shape == (0, 20)
