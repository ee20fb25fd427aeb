"""The tensor-core scan's bounded waits: a wait that runs out is reported, not hung.

Every mbarrier wait of the tensor-core list scan has a wall-time limit.  The
test hook ADANNS_OPT_TEST_SKIP_LOAD leaves one stage of the pipeline unfilled
(no copy is issued and nobody arrives on its barrier), so the MMA issuer's
wait on it runs out: the kernel must record the stage in the index's status
word, stop issuing work, let its copies land, free its tensor memory and
return.  The host then reads ADANNS_ERR_TIMEOUT once, the word is cleared, and
the next search on the same index and context is correct again.
"""
import numpy as np
import pytest

import oracle
import synthdata
from parity import recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BF16 = 2


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
    data = synthdata.small(20_000, 300, 256, 32, 77)
    o = oracle.build_ivf(data["db"], 32, 40, 6, 10_000, seed=5)
    g = A.index_create(cu(data["db"]), cu(o["centroids"]), cu(o["assign"].astype(np.int32)),
                       storage=1 | BF16)
    yield data, o, g
    g.free()


@pytest.mark.parametrize("skip", [0, 5])
def test_wait_runs_out_reports_timeout_and_recovers(A, case, skip):
    data, o, g = case
    q = cu(data["queries"])
    g.status()  # nothing pending
    with A.option(A.OPT_WAIT_LIMIT_NS, 10_000_000):
        A.set_option(A.OPT_TEST_SKIP_LOAD, skip)
        try:
            A.search_ivf(g, q, 32, 256, 6, 10, storage=BF16, rerank_k=40)
            torch.cuda.synchronize()  # the kernel returned: the context is usable
        finally:
            A.set_option(A.OPT_TEST_SKIP_LOAD, -1)
        with pytest.raises(A.AdannsError) as e:
            g.status()
        assert e.value.code == -5
        g.status()  # reported once, then cleared
    # the hook is one-shot, tensor memory was released: the next search is correct
    assert A.get_option(A.OPT_TEST_SKIP_LOAD) == -1
    gi, gd = A.search_ivf(g, q, 32, 256, 6, 10, storage=BF16, rerank_k=40)
    g.status()
    ref = oracle.search_ivf(data["db"], o, data["queries"], 32, 256, 6, 10)
    assert recall(gi.cpu().numpy(), ref["ids"], 10) >= 0.99


def test_option_validation(A):
    with pytest.raises(A.AdannsError):
        A.set_option(A.OPT_WAIT_LIMIT_NS, 10)
    with pytest.raises(A.AdannsError):
        A.set_option(99, 1)
    assert A.get_option(A.OPT_WAIT_LIMIT_NS) == 2_000_000_000
