"""The autotuner on the GPU: launch knobs changed on a live handle
(simrank_set_launch) keep the results of the oracle, and a stream run with
the knobs the tuner picked matches the oracle (FP32 tolerance)."""
import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import chung_lu_digraph, update_stream

pytestmark = pytest.mark.gpu

TOL32 = 1e-6


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_00121_gb300 as P

    return P


def setup(n=1200, seed=101, count=60, C=0.6):
    s, d = chung_lu_digraph(n, 10 * n, 2.1, 2.1, seed)
    st = update_stream(n, s, d, count, seed + 1)
    S0 = O.simrank_fixed_point(O.transition_matrix(n, s, d, sparse=True), C, tol=1e-15)
    return n, s, d, st, S0


def test_set_launch_mid_stream_keeps_parity(P):
    n, s, d, st, S0 = setup()
    C, K = 0.6, 12
    want, _ = O.sequential_unit_updates(n, s, d, S0, st.tolist(), C, K)
    h = P.SimRank(n, s, d, C=C, K=K, s_precision=32, vec_fp64=1, defer=16, tc=2)
    h.apply_updates(st[:10])
    h.set_launch(defer=8, tc=1, prep_item=512)
    h.apply_updates(st[10:30])
    h.set_launch(defer=0, tc=0, prep_ctas=100, prep_item=2048)
    h.apply_updates(st[30:45])
    h.set_launch(defer=24, tc=2, prep_ctas=0, prep_item=1024)
    h.apply_updates(st[45:])
    got = h.dense()
    h.close()
    assert np.max(np.abs(got - want)) < TOL32


def test_tuned_knobs_keep_parity(P, tmp_path):
    from paper_1711_00121_gb300 import tune

    n, s, d, st, S0 = setup(seed=111)
    C, K = 0.6, 10
    path = str(tmp_path / "tuned.json")
    res = tune.tune_stream(n, s, d, C=C, K=K, updates=48, warmup=16, path=path)
    kn = res["knobs"]
    assert set(kn) == {"defer", "tc", "prep_item", "prep_ctas"} and res["us_per_update"] > 0
    assert tune.lookup("stream", tune.gpu_name(), n, K, 32, 1, path) == kn
    h = P.SimRank(n, s, d, C=C, K=K, s_precision=32, vec_fp64=1, **kn)
    h.apply_updates(st)
    got = h.dense()
    h.close()
    want, _ = O.sequential_unit_updates(n, s, d, S0, st.tolist(), C, K)
    assert np.max(np.abs(got - want)) < TOL32
