"""simrank_grad (adjoint of the K-truncated series) against the FP64 CPU
oracle's derivative and against central finite differences of the GPU's own
loss, through the C ABI and the torch.autograd.Function."""
import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import chung_lu_digraph, edge_weights, query_pairs

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


def instance(n=260, m=1500, npairs=40, seed=61):
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, seed)
    w = edge_weights(m, seed)
    a, b, t = query_pairs(n, npairs, seed)
    return s, d, w, a, b, t


@pytest.mark.parametrize("mode", [0, 1])
def test_grad_matches_oracle_derivative(P, mode):
    n = 260
    s, d, w, a, b, t = instance(n)
    C, K = 0.6, 9
    sr = P.SimRank(n, s, d, weight=w, C=C, K=K, s_precision=64, mode=mode)
    L, g = sr.grad(a, b, t, s.size)
    L_ref, g_ref, _ = O.pair_loss_and_weight_grad(n, s, d, w.astype(np.float64), a, b, t, C, K)
    assert abs(L - L_ref) < 1e-11 * max(1.0, abs(L_ref))
    assert np.max(np.abs(g - g_ref)) < 1e-10 * max(1.0, np.max(np.abs(g_ref)))


def test_grad_unweighted_graph(P):
    n = 200
    s, d, w, a, b, t = instance(n, 1000, 30, 62)
    C, K = 0.7, 6
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=64, mode=1)
    L, g = sr.grad(a, b, t, s.size)
    L_ref, g_ref, _ = O.pair_loss_and_weight_grad(n, s, d, np.ones(s.size), a, b, t, C, K)
    assert abs(L - L_ref) < 1e-11
    assert np.max(np.abs(g - g_ref)) < 1e-10


def test_grad_vs_central_differences(P):
    n = 240
    s, d, w, a, b, t = instance(n, 1400, 30, 63)
    C, K = 0.6, 8
    w = w.astype(np.float32)

    def loss(wv):
        sr = P.SimRank(n, s, d, weight=wv, C=C, K=K, s_precision=64, mode=1)
        L, _ = sr.grad(a, b, t, s.size)
        sr.close()
        return L

    sr = P.SimRank(n, s, d, weight=w, C=C, K=K, s_precision=64, mode=1)
    _, g = sr.grad(a, b, t, s.size)
    rng = np.random.default_rng(64)
    for e in rng.choice(s.size, size=6, replace=False):
        h = np.float32(2.0 ** -9) * w[e]
        wp = w.copy()
        wp[e] += h
        wm = w.copy()
        wm[e] -= h
        fd = (loss(wp) - loss(wm)) / (float(wp[e]) - float(wm[e]))
        assert abs(fd - g[e]) < 1e-5 * max(1e-3, abs(g[e])) + 1e-9, (e, fd, g[e])


def test_autograd_function(P):
    import torch
    from paper_1711_00121_gb300.autograd import pair_loss

    n = 150
    s, d, w, a, b, t = instance(n, 800, 20, 65)
    C, K = 0.6, 7
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    L = pair_loss(wt, n, s, d, a, b, t, C, K)
    L.backward()
    L_ref, g_ref, _ = O.pair_loss_and_weight_grad(n, s, d, w.astype(np.float64), a, b, t, C, K)
    assert abs(float(L) - L_ref) < 1e-11
    assert np.max(np.abs(wt.grad.numpy() - g_ref)) < 1e-10
