"""Many graphs advanced together (simrank_multi_*) vs the FP64 CPU oracle.

Each graph's S after its own update stream must equal the oracle's
sequential Alg 1 updates on that graph alone (1e-10 with S in FP64, 1e-6
with S in FP32), whatever the batching: one launch pair per round replayed
from a CUDA graph, or per-graph launches.  Graph sizes span one to several
tiles, with ragged last tiles; some graphs get no update at all.
"""
import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import er_graph, chung_lu_digraph, update_stream, batch_with_new_nodes

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
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


def oracle_S(n, s, d, C, n_total=None):
    S = O.simrank_fixed_point(O.transition_matrix(n, s, d, sparse=True), C, tol=1e-15)
    if n_total is not None and n_total > n:
        T = np.zeros((n_total, n_total))
        T[:n, :n] = S
        T[np.arange(n, n_total), np.arange(n, n_total)] = 1.0 - C
        S = T
    return S


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


def make_graphs(count, seed, n_lo=100, n_hi=520):
    rng = np.random.default_rng(seed)
    out = []
    for g in range(count):
        n = int(rng.integers(n_lo, n_hi))
        m = int(n * rng.uniform(3.0, 7.0))
        if g % 2:
            s, d = chung_lu_digraph(n, m, 2.1, 2.1, seed * 1000 + g)
        else:
            s, d = er_graph(n, m, seed * 1000 + g)
        out.append((n, s, d))
    return out


def streams(graphs, seed, max_len):
    rng = np.random.default_rng(seed)
    ups = []
    for g, (n, s, d) in enumerate(graphs):
        c = int(rng.integers(0, max_len + 1)) if g else 0  # graph 0 gets none
        ups.append(update_stream(n, s, d, c, seed * 77 + g))
    return ups


@pytest.mark.parametrize("prec,launch,tc", [(64, 0, 0), (64, 1, 0), (32, 0, 0), (32, 1, 0),
                                            (32, 0, 1), (32, 1, 1)])
def test_multi_streams_match_oracle(P, prec, launch, tc):
    C, K = 0.6, 10
    graphs = make_graphs(9, 21)
    ups = streams(graphs, 22, 7)
    mh = P.MultiSimRank(graphs, C=C, K=K, s_precision=prec, multi_launch=launch, tc=tc)
    mh.apply_updates(ups)
    mh.sync()
    tol = TOL64 if prec == 64 else TOL32
    for g, (n, s, d) in enumerate(graphs):
        want, _ = O.sequential_unit_updates(n, s, d, oracle_S(n, s, d, C), ups[g].tolist(), C, K)
        got = mh.dense(g)
        assert maxabs(got, want) < tol, g
        assert maxabs(got, got.T) < (1e-12 if prec == 64 else 1e-7)
    st = mh.stats()
    assert st["updates"] == sum(len(u) for u in ups)
    mh.close()


def test_multi_repeated_calls_reuse_the_cuda_graph(P):
    """Two calls of the same shape replay one instantiated CUDA graph; a third
    of another shape re-captures.  Results stay exact."""
    C, K = 0.6, 8
    graphs = make_graphs(6, 31)
    mh = P.MultiSimRank(graphs, C=C, K=K, s_precision=64)
    state = [(n, s, d, oracle_S(n, s, d, C)) for n, s, d in graphs]
    from synth.graphs import EdgeSet

    sets = [EdgeSet(n, s, d) for n, s, d in graphs]
    for call, length in enumerate([3, 3, 5]):
        ups = [update_stream(n, None, None, length, 500 + 10 * call + g, edge_set=sets[g])
               for g, (n, _, _) in enumerate(graphs)]
        mh.apply_updates(ups)
        new_state = []
        for g, (n, s, d, S) in enumerate(state):
            S2, edges = O.sequential_unit_updates(n, s, d, S, ups[g].tolist(), C, K)
            s2 = np.array([a for a, _ in edges], np.int32)
            d2 = np.array([b for _, b in edges], np.int32)
            new_state.append((n, s2, d2, S2))
        state = new_state
        for g, (n, _, _, S) in enumerate(state):
            assert maxabs(mh.dense(g), S) < TOL64, (call, g)
    mh.close()


def test_multi_new_nodes(P):
    """Updates that attach new nodes (pre-allocated capacity per graph)."""
    C, K = 0.6, 10
    base = make_graphs(5, 41, 150, 400)
    graphs, ups, finals = [], [], []
    for g, (n, s, d) in enumerate(base):
        u, n_new = batch_with_new_nodes(n, s, d, 12, 700 + g, frac_new=0.3)
        graphs.append((n, s, d, n + n_new))
        ups.append(u)
        finals.append(n + n_new)
    mh = P.MultiSimRank(graphs, C=C, K=K, s_precision=64, relabel=0)
    mh.apply_updates(ups)
    for g, (n, s, d, nf) in enumerate(graphs):
        want, _ = O.sequential_unit_updates(nf, s, d, oracle_S(n, s, d, C, nf), ups[g].tolist(), C, K)
        assert mh.num_nodes(g) == nf
        assert maxabs(mh.dense(g), want) < TOL64, g
    mh.close()


def test_multi_invalid_update_changes_nothing(P):
    C, K = 0.6, 6
    graphs = make_graphs(4, 51)
    mh = P.MultiSimRank(graphs, C=C, K=K, s_precision=64)
    before = [mh.dense(g) for g in range(4)]
    ups = streams(graphs, 52, 4)
    n3, s3, d3 = graphs[3]
    bad = np.array([[int(s3[0]), int(d3[0]), 1]], np.int32)  # inserting an existing edge
    ups[3] = np.concatenate([ups[3], bad]) if len(ups[3]) else bad
    with pytest.raises(P.SimrankError) as ei:
        mh.apply_updates(ups)
    assert "graph 3" in str(ei.value)
    for g in range(4):
        assert maxabs(mh.dense(g), before[g]) == 0.0
    mh.close()


def test_multi_large_graph_global_path(P):
    """A graph too large for the shared-memory vectors (FP64, > 5120 rows)
    next to a small one: both paths of the prep kernel in one round."""
    C, K = 0.4, 6
    big = (5200,) + er_graph(5200, 3 * 5200, 61)
    small = (300,) + er_graph(300, 1200, 62)
    graphs = [big, small]
    ups = [update_stream(n, s, d, 3, 63 + g) for g, (n, s, d) in enumerate(graphs)]
    mh = P.MultiSimRank(graphs, C=C, K=K, s_precision=64)
    mh.apply_updates(ups)
    for g, (n, s, d) in enumerate(graphs):
        want, _ = O.sequential_unit_updates(n, s, d, oracle_S(n, s, d, C), ups[g].tolist(), C, K)
        assert maxabs(mh.dense(g), want) < TOL64, g
    mh.close()
