"""One-shot batch form (whole batch as one rank-2r update) against the
oracle's definition (Eq. 23-25 written out: T = Q_new S Q_new^T - Q S Q^T,
Delta S_K = sum_{k<=K} C^{k+1} Q_new^k T Q_new^kT), through the C ABI."""
import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import er_graph, chung_lu_digraph, batch_with_new_nodes

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


def setup(n, m, seed, b, frac_new, C, powerlaw=False):
    if powerlaw:
        s, d = chung_lu_digraph(n, m, 2.2, 2.2, seed)
    else:
        s, d = er_graph(n, m, seed)
    S = O.simrank_fixed_point(O.transition_matrix(n, s, d, sparse=True), C, tol=1e-15)
    ups, n_new = batch_with_new_nodes(n, s, d, b, seed, frac_new=frac_new, reuse_target=0.5)
    n_final = n + n_new
    Sp = np.zeros((n_final, n_final))
    Sp[:n, :n] = S
    for x in range(n, n_final):
        Sp[x, x] = 1 - C
    edges = set(zip(s.tolist(), d.tolist()))
    plus, minus = O.net_update(ups.tolist())
    new = (edges | set(plus)) - set(minus)
    ns = np.array([a for a, _ in new], np.int64)
    nd = np.array([bb for _, bb in new], np.int64)
    return s, d, S, ups, n_final, Sp, ns, nd


def test_one_shot_fp64_vs_definition(P):
    n, m, C, K = 500, 2500, 0.6, 10
    s, d, S, ups, n_final, Sp, ns, nd = setup(n, m, 31, 40, 0.2, C)
    sr = P.SimRank(n, s, d, S0=S, C=C, K=K, s_precision=64, n_capacity=n_final,
                   apply=P.APPLY_ONE_SHOT)
    sr.apply_updates(ups)
    want = O.one_shot_batch(n_final, s, d, ns, nd, Sp, C, K)
    assert maxabs(sr.dense(), want) < TOL64


@pytest.mark.parametrize("tc", [0, 1, 2])
def test_one_shot_fp32_vs_definition(P, tc):
    n, m, C, K = 1100, 8800, 0.8, 12
    s, d, S, ups, n_final, Sp, ns, nd = setup(n, m, 32, 96, 0.1, C, powerlaw=True)
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=32, n_capacity=n_final,
                   apply=P.APPLY_ONE_SHOT, tc=tc)
    sr.apply_updates(ups)
    sr.sync()
    want = O.one_shot_batch(n_final, s, d, ns, nd, Sp, C, K)
    got = sr.dense()
    assert maxabs(got, want) < TOL32
    # S is symmetric (Eq. 1); in FP32 the diagonal tiles of the tensor-core
    # update accumulate D[r][c] and D[c][r] in different orders
    assert maxabs(got, got.T) < TOL32


def test_one_shot_tc_matches_ffma_many_chunks(P):
    """More sinks than one 32-column chunk, several k per S pass, and a sink
    that loses every in-edge: the tensor-core and CUDA-core updates agree."""
    n, m, C, K = 900, 5400, 0.6, 6
    s, d = er_graph(n, m, 33)
    edges = list(zip(s.tolist(), d.tolist()))
    deg = np.bincount(d, minlength=n)
    j_all = int(np.nonzero(deg == 2)[0][0])
    ups = [(a, b, -1) for a, b in edges if b == j_all]
    rng = np.random.default_rng(33)
    have = set(edges)
    while len(ups) < 150:
        i, j = map(int, rng.integers(0, n, 2))
        if i != j and (i, j) not in have and j != j_all:
            have.add((i, j))
            ups.append((i, j, 1))
    res = []
    for tc in (0, 1, 2):
        sr = P.SimRank(n, s, d, C=C, K=K, s_precision=32, apply=P.APPLY_ONE_SHOT, tc=tc)
        sr.apply_updates(ups)
        sr.sync()
        res.append(sr.dense())
    assert maxabs(res[0], res[1]) < TOL32
    assert maxabs(res[0], res[2]) < TOL32
    S = O.simrank_fixed_point(O.transition_matrix(n, s, d, sparse=True), C, tol=1e-15)
    plus, minus = O.net_update(ups)
    new = (set(edges) | set(plus)) - set(minus)
    ns = np.array([a for a, _ in new], np.int64)
    nd = np.array([bb for _, bb in new], np.int64)
    want = O.one_shot_batch(n, s, d, ns, nd, S, C, K)
    assert maxabs(res[1], want) < TOL32
    assert maxabs(res[2], want) < TOL32


def test_one_shot_converges_to_batch_recompute(P):
    n, m, C, K = 600, 3600, 0.6, 70
    s, d, S, ups, n_final, Sp, ns, nd = setup(n, m, 34, 50, 0.15, C)
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=64, n_capacity=n_final, apply=P.APPLY_ONE_SHOT)
    sr.apply_updates(ups)
    truth = O.simrank_fixed_point(O.transition_matrix(n_final, ns, nd, sparse=True), C, tol=1e-15)
    assert maxabs(sr.dense(), truth) < TOL64


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))
