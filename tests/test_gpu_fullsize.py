"""Parity at the full size of the benchmarked workload (directed Chung-Lu,
n = 20,000, in/out exponent 2.1, mean degree 10, C = 0.6, K = 20, S in FP32),
on sampled columns that the oracle computes one by one (Procedure 1 and
Alg 7), plus properties that hold at any size."""
import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import chung_lu_digraph, update_stream, EdgeSet

pytestmark = pytest.mark.gpu

N, M, C, K = 20000, 200000, 0.6, 20
K_CONV = 60  # C^(K+1) / (1 - C) < 1e-13: the truncation has vanished at this K
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


@pytest.fixture(scope="module")
def graph():
    s, d = chung_lu_digraph(N, M, 2.1, 2.1, 2)
    return s, d


def sample_cols(n, k, seed, must=()):
    rng = np.random.default_rng(seed)
    cols = list(must) + rng.choice(n, size=k, replace=False).tolist()
    return np.array(sorted(set(cols)), np.int32)


def test_fullsize_init_and_first_update(P, graph):
    s, d = graph
    sr = P.SimRank(N, s, d, C=C, K=K, s_precision=32)
    Qs = O.transition_matrix(N, s, d, sparse=True)
    cols = sample_cols(N, 16, 21)
    want = O.partial_sim_block(Qs, cols, K_CONV, C)
    got = sr.columns(cols)
    assert np.max(np.abs(got - want)) < TOL32
    # first update of the benchmarked stream, on sampled columns (Alg 7 with
    # converged old columns and the same K)
    st = update_stream(N, s, d, 1, 3)
    i, j, op = map(int, st[0])
    cols = sample_cols(N, 6, 22, must=(i, j))
    sr.apply_updates(st)
    got = sr.columns(cols)
    for c, x in enumerate(cols):
        col0 = O.partial_sim(Qs, int(x), K_CONV, C)
        want = O.inc_sr_all_p(N, s, d, col0, int(x), [(i, j, op)], C, K, K_old=K_CONV)
        assert np.max(np.abs(got[:, c] - want)) < TOL32, x


def test_fullsize_stream_properties(P, graph):
    """1,000 updates at the benchmarked K: symmetry, diag >= 1 - C and
    0 <= s <= 1 up to FP32 rounding, on sampled columns."""
    s, d = graph
    sr = P.SimRank(N, s, d, C=C, K=K, s_precision=32)
    st = update_stream(N, s, d, 1000, 3)
    sr.apply_updates(st)
    cols = sample_cols(N, 64, 23)
    got = sr.columns(cols)
    sub = got[cols, :]
    assert np.max(np.abs(sub - sub.T)) < 1e-7
    assert np.all(got[cols, np.arange(cols.size)] >= 1 - C - 1e-6)
    assert np.all(got >= -1e-6) and np.all(got <= 1 + 1e-6)
    stats = sr.stats()
    assert stats["rank_one_updates"] == 1000


@pytest.mark.parametrize("defer,tc", [(0, 0), (16, 1), (16, 2)])
def test_fullsize_stream_converged_vs_batch(P, graph, defer, tc):
    """The same 1,000-update stream at K_CONV: sampled columns equal an FP64
    batch recomputation (Procedure 1 to convergence) on the final graph, with
    S updated per edge on the CUDA cores, or 16 updates at a time on the
    tensor cores (TF32 or FP16 split)."""
    s, d = graph
    sr = P.SimRank(N, s, d, C=C, K=K_CONV, s_precision=32, defer=defer, tc=tc)
    es = EdgeSet(N, s, d)
    st = update_stream(N, s, d, 1000, 3, edge_set=es)
    sr.apply_updates(st)
    fs = np.array([a for a, _ in es.edges], np.int32)
    fd = np.array([b for _, b in es.edges], np.int32)
    Qf = O.transition_matrix(N, fs, fd, sparse=True)
    cols = sample_cols(N, 24, 24, must=tuple(int(x) for x in st[:4, 1]))
    want = O.partial_sim_block(Qf, cols, K_CONV, C)
    got = sr.columns(cols)
    err = float(np.max(np.abs(got - want)))
    print(f"stream of 1000 at K={K_CONV}: max-abs vs batch = {err:.3e}")
    assert err < TOL32
