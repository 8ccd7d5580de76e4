"""Failure detection without a GPU fault: every device-side wait of the
library is bounded.  A grid barrier of the pre-update kernel (k_prep) and
every mbarrier wait of the tensor-core S pass give up after timeout_iters
polls, record SR_ERR_TIMEOUT in the handle's status word and return (the
tensor-core pass first drains the TMA loads and MMAs it has in flight and
frees its TMEM).  Here a limit of one poll makes them run out: the other CTAs
of a grid barrier, and the TMA copies and MMAs of a tile, cannot all arrive
within one poll.  simrank_sync / simrank_multi_sync must report status 7,
and the device must stay usable: a new handle afterwards gives the oracle's
result."""
import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import chung_lu_digraph, update_stream

pytestmark = pytest.mark.gpu

SR_ERR_TIMEOUT = 7


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_00121_gb300 as P

    return P


def graph(n=3000, seed=71):
    s, d = chung_lu_digraph(n, 10 * n, 2.1, 2.1, seed)
    return n, s, d


def expect_timeout(fn):
    import paper_1711_00121_gb300 as P

    with pytest.raises(P.SimrankError) as e:
        fn()
    assert e.value.status == SR_ERR_TIMEOUT, str(e.value)


def still_usable(P):
    """After a timeout, a fresh handle on the same device gives Alg 1's result."""
    n, m, C, K = 400, 2000, 0.6, 8
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 72)
    S0 = O.simrank_fixed_point(O.transition_matrix(n, s, d, sparse=True), C, tol=1e-15)
    ups = update_stream(n, s, d, 3, 73)
    h = P.SimRank(n, s, d, S0=S0, C=C, K=K, s_precision=64)
    h.apply_updates(ups)
    h.sync()
    want, _ = O.sequential_unit_updates(n, s, d, S0, ups.tolist(), C, K)
    assert np.max(np.abs(h.dense() - want)) < 1e-10
    h.close()


def test_prep_grid_barrier_timeout(P):
    """k_prep: the grid barriers between phases and recurrence steps (the S pass
    is the single-role CUDA-core kernel, which has no waits)."""
    n, s, d = graph()
    h = P.SimRank(n, s, d, C=0.6, K=10, s_precision=32, chain=0, tc=0, s_kernel=1, defer=0,
                  timeout_iters=1)
    ups = update_stream(n, s, d, 8, 74)
    expect_timeout(lambda: (h.apply_updates(ups), h.sync()))
    h.close()
    still_usable(P)


@pytest.mark.parametrize("defer", [16, 0])
def test_tensor_core_pass_timeout(P, defer):
    """The tcgen05 S pass (defer = 16: jobs of two tile pairs; defer = 0: one
    tile pair per job); the work before it is the per-step path (chain = 1),
    whose kernels have no waits."""
    n, s, d = graph()
    h = P.SimRank(n, s, d, C=0.6, K=10, s_precision=32, chain=1, tc=2, defer=defer,
                  timeout_iters=1)
    ups = update_stream(n, s, d, 16, 75)
    expect_timeout(lambda: (h.apply_updates(ups), h.sync()))
    h.close()
    still_usable(P)


def test_multi_graph_pass_timeout(P):
    """simrank_multi_*: the tensor-core pass over the tiles of all graphs."""
    graphs = []
    for g in range(4):
        n = 900 + 300 * g
        s, d = chung_lu_digraph(n, 8 * n, 2.1, 2.1, 76 + g)
        graphs.append((n, s, d))
    mh = P.MultiSimRank(graphs, C=0.6, K=8, s_precision=32, tc=1, init_tol=1e-9, timeout_iters=1)
    per = [update_stream(n, s, d, 4, 80 + g) for g, (n, s, d) in enumerate(graphs)]
    expect_timeout(lambda: (mh.apply_updates(per), mh.sync()))
    mh.close()
    still_usable(P)
