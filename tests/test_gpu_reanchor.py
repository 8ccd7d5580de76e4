"""Automatic drift re-anchor (reanchor_every): after every N updates the
library runs Jacobi sweeps of Eq. 1 from the current S and reports the
residual it found.  An FP32-S stream of 240 updates at K = 20, re-anchored
every 60 updates, must end at the FP64 fixed point of the final graph on
sampled columns (within the FP32 tolerance), where the same stream without
re-anchoring carries the truncation drift of its 240 updates."""
import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import chung_lu_digraph, update_stream, EdgeSet

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


@pytest.mark.parametrize("defer,tc", [(0, 0), (16, 2)])
def test_fp32_stream_reanchored_to_fixed_point(P, defer, tc):
    n, m, C, K = 1500, 12000, 0.6, 20
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 91)
    es = EdgeSet(n, s, d)
    st = update_stream(n, s, d, 240, 92, edge_set=es)
    fs = np.array([a for a, _ in es.edges], np.int32)
    fd = np.array([b for _, b in es.edges], np.int32)
    rng = np.random.default_rng(93)
    cols = np.array(sorted(set(rng.choice(n, 24, replace=False).tolist())
                           | {int(x) for x in st[-4:, 1]}), np.int32)
    truth = O.partial_sim_block(O.transition_matrix(n, fs, fd, sparse=True), cols, 80, C)
    drift = P.SimRank(n, s, d, C=C, K=K, s_precision=32, defer=defer, tc=tc)
    drift.apply_updates(st)
    e_drift = float(np.max(np.abs(drift.columns(cols) - truth)))
    drift.close()
    h = P.SimRank(n, s, d, C=C, K=K, s_precision=32, defer=defer, tc=tc, reanchor_every=60,
                  reanchor_sweeps=80, init_tol=1e-12)
    h.apply_updates(st)
    e_anchor = float(np.max(np.abs(h.columns(cols) - truth)))
    stats = h.stats()
    h.close()
    assert stats["reanchors"] == 4
    assert stats["reanchor_residual"] > stats["reanchor_change"]
    assert e_anchor < TOL32, (e_anchor, e_drift)
    assert e_anchor < e_drift
