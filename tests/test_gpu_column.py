"""Column mode (§7, Alg 7 Inc-SR-All-P with Procedure 1) against the oracle,
through the C ABI."""
import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import er_graph, chung_lu_digraph, update_stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1711_00121_gb300 as P

    return P


def test_column_mode_base_columns_fp64(P):
    n, m, C, K = 700, 3500, 0.6, 9
    s, d = er_graph(n, m, 51)
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=64, mode=P.MODE_COLUMN)
    cols = np.array([0, 3, 129, 300, 699], np.int32)
    Q = O.transition_matrix(n, s, d, sparse=True)
    want = O.partial_sim_block(Q, cols, K, C)
    assert np.max(np.abs(sr.columns(cols) - want)) < 1e-12


def test_column_mode_updates_all_cases_fp64(P):
    n, m, C, K = 500, 2500, 0.6, 8
    s, d = er_graph(n, m, 52)
    edges = set(zip(s.tolist(), d.tolist()))
    deg = np.bincount(d, minlength=n)
    j_big = int(np.argmax(deg))
    i_new = next(x for x in range(n) if x != j_big and (x, j_big) not in edges)
    e_del = next(e for e in sorted(edges) if deg[e[1]] > 1 and e[1] != j_big)
    ups = [
        (i_new, j_big, 1),   # C0 insert
        (e_del[0], e_del[1], -1),  # C0 delete
        (4, n, 1),           # C1: j new
        (n + 1, j_big, 1),   # C2: i new
        (n + 2, n + 3, 1),   # C3: both new
        (9, n, 1),           # C0 into a node created above
    ]
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=64, mode=P.MODE_COLUMN, n_capacity=n + 4)
    sr.apply_updates(ups)
    assert sr.n == n + 4
    cols = np.array([0, j_big, i_new, e_del[1], n, n + 1, n + 3, 257], np.int32)
    got = sr.columns(cols)
    Q0 = O.transition_matrix(n, s, d, sparse=True)
    for c, x in enumerate(cols.tolist()):
        col0 = O.partial_sim(Q0, x, K, C) if x < n else np.zeros(n)
        want = O.inc_sr_all_p(n, s, d, col0, x, ups, C, K)
        assert np.max(np.abs(got[:, c] - want)) < 1e-10, x


def test_column_mode_stream_fp32(P):
    n, m, C, K = 1200, 12000, 0.6, 10
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 53)
    st = update_stream(n, s, d, 12, 54)
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=32, mode=P.MODE_COLUMN)
    sr.apply_updates(st)
    rng = np.random.default_rng(55)
    cols = np.sort(rng.choice(n, size=40, replace=False)).astype(np.int32)
    got = sr.columns(cols)
    Q0 = O.transition_matrix(n, s, d, sparse=True)
    base = O.partial_sim_block(Q0, cols, K, C)
    for c, x in enumerate(cols.tolist()[:6]):
        want = O.inc_sr_all_p(n, s, d, base[:, c], x, st.tolist(), C, K)
        assert np.max(np.abs(got[:, c] - want)) < 1e-6, x


@pytest.mark.parametrize("width", [1, 3, 4, 5, 8])
def test_column_mode_fp32_query_widths(P, width):
    """FP32 queries of every block form: narrow blocks (one warp per four row
    chunks, B <= 4), four columns per thread (B a multiple of 4) and one column
    per thread (other widths), after stored updates, against Alg 7."""
    n, m, C, K = 900, 8000, 0.6, 9
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 61)
    st = update_stream(n, s, d, 6, 62)
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=32, mode=P.MODE_COLUMN)
    sr.apply_updates(st)
    rng = np.random.default_rng(63 + width)
    cols = np.sort(rng.choice(n, size=width, replace=False)).astype(np.int32)
    got = sr.columns(cols)
    Q0 = O.transition_matrix(n, s, d, sparse=True)
    base = O.partial_sim_block(Q0, cols, K, C)
    for c, x in enumerate(cols.tolist()):
        want = O.inc_sr_all_p(n, s, d, base[:, c], x, st.tolist(), C, K)
        assert np.max(np.abs(got[:, c] - want)) < 1e-6, (width, x)


@pytest.mark.parametrize("prec", [64, 32])
def test_column_mode_sink_blocks(P, prec):
    """Alg 7 fed by similar-sink blocks (§8; the closing remark of §7): a batch
    with deletions and new nodes, then a block of 40 insertions into one sink
    (one Procedure-1 column started from the indicator of its 40 sources), against the
    oracle's column form at the same K (old columns by PartialSim at K)."""
    from synth import batch_with_new_nodes

    n, m, C, K = 500, 2500, 0.6, 8
    s, d = er_graph(n, m, 56)
    ups, n_new = batch_with_new_nodes(n, s, d, 60, 57, frac_new=0.2, reuse_target=0.5)
    n_final = n + n_new
    plus, minus = O.net_update(ups.tolist())
    edges1 = (set(zip(s.tolist(), d.tolist())) | set(plus)) - set(minus)
    deg1 = np.bincount(np.array([b for _, b in edges1]), minlength=n_final)
    j0 = int(np.argmax(deg1[:n]))
    big = [(x, j0, 1) for x in range(n_final) if x != j0 and (x, j0) not in edges1][:40]
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=prec, mode=P.MODE_COLUMN, n_capacity=n_final,
                   apply=P.APPLY_SINK_BLOCKS)
    sr.apply_updates(ups)
    sr.apply_updates(big)
    assert sr.n == n_final
    rng = np.random.default_rng(58)
    cols = sorted(set(rng.choice(n_final, 6, replace=False).tolist()) | {j0, big[0][0], n_final - 1})
    got = sr.columns(np.array(cols, np.int32))
    Q0 = O.transition_matrix(n, s, d, sparse=True)
    e1s = np.array([a for a, _ in edges1], np.int64)
    e1d = np.array([b for _, b in edges1], np.int64)
    for c, x in enumerate(cols):
        col0 = O.partial_sim(Q0, x, K, C) if x < n else None
        mid = O.inc_sr_all_p_blocks(n, n_final, s, d, col0, x, ups.tolist(), C, K)
        want = O.inc_sr_all_p_blocks(n_final, n_final, e1s, e1d, mid, x, big, C, K)
        assert np.max(np.abs(got[:, c] - want)) < (1e-10 if prec == 64 else 1e-6), x
