"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances: 1e-10 max-abs with S in FP64, 1e-6 with S in FP32 (the stated
targets for the two storage precisions).  Sizes span several 128-wide tiles
with a ragged last tile.
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


def oracle_S(n, s, d, C):
    return O.simrank_fixed_point(O.transition_matrix(n, s, d, sparse=True), C, tol=1e-15)


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


# ----------------------------------------------------------------------- init

def test_init_fp64_config1(P):
    n, m, C = 1000, 5000, 0.6
    s, d = er_graph(n, m, 1)
    sr = P.SimRank(n, s, d, C=C, K=15, s_precision=64)
    assert maxabs(sr.dense(), oracle_S(n, s, d, C)) < TOL64
    st = sr.stats()
    assert st["init_residual"] < 1e-13


def test_init_fp32_powerlaw(P):
    n, m, C = 1500, 15000, 0.6
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 2)
    sr = P.SimRank(n, s, d, C=C, K=20, s_precision=32)
    assert maxabs(sr.dense(), oracle_S(n, s, d, C)) < TOL32


def test_init_accepts_S0_and_isolated_capacity(P):
    n, C = 300, 0.7
    s, d = er_graph(n, 1200, 3)
    S = oracle_S(n, s, d, C)
    sr = P.SimRank(n, s, d, S0=S, C=C, K=5, s_precision=64, n_capacity=n + 7)
    assert sr.n == n
    assert maxabs(sr.dense(), S) == 0.0


# ---------------------------------------------------------- unit updates (C0)

def _cases(n, s, d):
    edges = set(zip(s.tolist(), d.tolist()))
    deg = np.bincount(d, minlength=n)
    outs = {}
    for a, b in edges:
        outs.setdefault(b, []).append(a)
    j_big = int(np.argmax(deg))
    i_new = next(x for x in range(n) if x != j_big and (x, j_big) not in edges)
    j_zero = int(np.nonzero(deg == 0)[0][0])
    i_zero = 0 if j_zero != 0 else 1
    j_one = int(np.nonzero(deg == 1)[0][0])
    return {
        "insert_dj_pos": (i_new, j_big, 1),
        "insert_dj_zero": (i_zero, j_zero, 1),
        "delete_dj_gt1": (outs[j_big][0], j_big, -1),
        "delete_dj_eq1": (outs[j_one][0], j_one, -1),
    }


@pytest.mark.parametrize("case", ["insert_dj_pos", "insert_dj_zero", "delete_dj_gt1", "delete_dj_eq1"])
@pytest.mark.parametrize("K", [0, 15])
def test_unit_update_fp64_config1(P, case, K):
    n, m, C = 1000, 5000, 0.6
    s, d = er_graph(n, m, 1)
    if case == "insert_dj_zero" and np.all(np.bincount(d, minlength=n) > 0):
        pytest.skip("graph has no zero in-degree node")
    i, j, op = _cases(n, s, d)[case]
    S = oracle_S(n, s, d, C)
    sr = P.SimRank(n, s, d, S0=S, C=C, K=K, s_precision=64)
    sr.apply_updates([(i, j, op)])
    want = O.inc_usr(n, s, d, S, j, [i], op, C, K)
    assert maxabs(sr.dense(), want) < TOL64


@pytest.mark.parametrize("case", ["insert_dj_pos", "delete_dj_gt1"])
def test_unit_update_converged_vs_batch_recompute(P, case):
    """At K large enough for the truncation to vanish, one update equals a full
    FP64 batch recomputation on the new graph."""
    n, m, C = 1000, 5000, 0.6
    s, d = er_graph(n, m, 1)
    i, j, op = _cases(n, s, d)[case]
    sr = P.SimRank(n, s, d, C=C, K=75, s_precision=64)
    sr.apply_updates([(i, j, op)])
    edges = set(zip(s.tolist(), d.tolist()))
    edges = edges | {(i, j)} if op > 0 else edges - {(i, j)}
    ns = np.array([a for a, _ in edges])
    nd = np.array([b for _, b in edges])
    assert maxabs(sr.dense(), oracle_S(n, ns, nd, C)) < TOL64


# ------------------------------------------------------------ update streams

@pytest.mark.parametrize("variant", ["fused_aff", "fused_aff_norelabel", "fused_single_role",
                                     "fused_noaff", "plain", "deferred_ffma", "deferred_tc",
                                     "per_step_chain", "prep_multi_tile", "prep_small_items",
                                     "deferred_multi_tile", "full_storage", "deferred_tc_full",
                                     "tc_each", "fp64_vectors", "deferred_fp64_vectors",
                                     "deferred_tc_f16", "tc_each_f16"])
def test_stream_fp32_powerlaw(P, variant):
    n, m, C, K = 1500, 15000, 0.6, 20
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 4)
    st = update_stream(n, s, d, 40, 5)
    kw = dict(aff=1, s_update=P.SUPDATE_FUSED)
    if variant == "fused_aff_norelabel":
        kw = dict(aff=1, relabel=0, s_update=P.SUPDATE_FUSED)
    elif variant == "fused_single_role":
        kw = dict(aff=1, s_kernel=1, s_update=P.SUPDATE_FUSED)
    elif variant == "deferred_ffma":
        kw = dict(aff=1, defer=7, tc=0)
    elif variant == "deferred_tc":
        kw = dict(aff=1, defer=16, tc=1)
    elif variant == "fused_noaff":
        kw = dict(aff=0, s_update=P.SUPDATE_FUSED)
    elif variant == "plain":
        kw = dict(aff=0, s_update=P.SUPDATE_PLAIN)
    elif variant == "per_step_chain":
        kw = dict(aff=1, chain=1)
    elif variant == "prep_multi_tile":
        # 12 tiles on 2 CTAs (6 tiles each) and a 64-entry column cache: the
        # multi-tile and uncached-column paths of the fused launch
        kw = dict(aff=1, prep_ctas=2, prep_cache=64)
    elif variant == "prep_small_items":
        # 48-nonzero work items: every tile split over several CTAs
        kw = dict(aff=1, prep_item=48, prep_ctas=40)
    elif variant == "fp64_vectors":
        kw = dict(aff=1, vec_fp64=1)
    elif variant == "deferred_fp64_vectors":
        kw = dict(aff=1, defer=16, tc=1, vec_fp64=1)
    elif variant == "deferred_tc_f16":
        kw = dict(aff=1, defer=16, tc=2)
    elif variant == "tc_each_f16":
        kw = dict(aff=1, defer=0, tc=2)
    elif variant == "tc_each":
        kw = dict(aff=1, defer=0, tc=1)
    elif variant == "full_storage":
        kw = dict(aff=1, upper_only=0)
    elif variant == "deferred_tc_full":
        kw = dict(aff=1, defer=16, tc=1, upper_only=0)
    elif variant == "deferred_multi_tile":
        kw = dict(aff=1, defer=7, tc=1, prep_ctas=3, prep_cache=128)
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=32, **kw)
    sr.apply_updates(st)
    S = oracle_S(n, s, d, C)
    want, _ = O.sequential_unit_updates(n, s, d, S, st.tolist(), C, K)
    got = sr.dense()
    assert maxabs(got, want) < TOL32
    assert maxabs(got, got.T) < 1e-7


@pytest.mark.parametrize("kw", [{}, {"chain": 1}, {"prep_ctas": 2, "prep_cache": 32},
                                {"prep_item": 40, "prep_ctas": 30}, {"upper_only": 0},
                                {"upper_only": 0, "chain": 1}],
                         ids=["fused", "per_step", "fused_multi_tile", "fused_small_items",
                              "full_storage", "full_storage_per_step"])
def test_stream_fp64_matches_oracle(P, kw):
    n, m, C, K = 700, 4200, 0.8, 12
    s, d = er_graph(n, m, 6)
    st = update_stream(n, s, d, 25, 7)
    S = oracle_S(n, s, d, C)
    sr = P.SimRank(n, s, d, S0=S, C=C, K=K, s_precision=64, **kw)
    sr.apply_updates(st)
    want, _ = O.sequential_unit_updates(n, s, d, S, st.tolist(), C, K)
    assert maxabs(sr.dense(), want) < TOL64


def test_aff_skips_tiles_and_leaves_them_bitwise_unchanged(P):
    """Thm 4 pruning is lossless: tiles outside the affected area are not
    touched (bitwise identical S there), and the result equals the unpruned one."""
    n, C, K = 1024, 0.6, 8
    # two disjoint halves: an update inside the first half cannot reach the second
    s1, d1 = er_graph(512, 2500, 8)
    s = np.concatenate([s1, s1 + 512]).astype(np.int32)
    d = np.concatenate([d1, d1 + 512]).astype(np.int32)
    edges = set(zip(s.tolist(), d.tolist()))
    i, j = next((a, b) for a in range(512) for b in range(512) if a != b and (a, b) not in edges)
    S = oracle_S(n, s, d, C)
    sr = P.SimRank(n, s, d, S0=S, C=C, K=K, s_precision=64, aff=1)
    before = sr.dense()
    sr.apply_updates([(i, j, 1)])
    after = sr.dense()
    assert np.array_equal(after[512:, :], before[512:, :])
    assert np.array_equal(after[:, 512:], before[:, 512:])
    st = sr.stats()
    assert st["tiles_touched"] < st["tiles_total"]
    want = O.inc_usr(n, s, d, S, j, [i], 1, C, K)
    assert maxabs(after, want) < TOL64


# ------------------------------------------------------------- new nodes (§6)

def test_new_node_cases_unit_fp64(P):
    n, m, C, K = 600, 3000, 0.7, 12
    s, d = er_graph(n, m, 9)
    S = oracle_S(n, s, d, C)
    deg = np.bincount(d, minlength=n)
    j_old = int(np.argmax(deg))
    ups = [
        (5, n, 1),           # C1: i in V, j new (id n)
        (n + 1, j_old, 1),   # C2: i new (id n+1), j in V
        (n + 2, n + 3, 1),   # C3: both new
        (7, n, 1),           # C0 into the node created by C1
    ]
    sr = P.SimRank(n, s, d, S0=S, C=C, K=K, s_precision=64, n_capacity=n + 10)
    sr.apply_updates(ups)
    assert sr.n == n + 4
    Sp = np.zeros((n + 4, n + 4))
    Sp[:n, :n] = S
    for x in range(n, n + 4):
        Sp[x, x] = 1 - C
    want, _ = O.sequential_unit_updates(n + 4, s, d, Sp, ups, C, K)
    got = sr.dense()
    assert maxabs(got, want) < TOL64
    # C3 block of Alg 5: the new pair forms its own component
    assert abs(got[n + 3, n + 3] - (1 - C * C)) < TOL64
    assert abs(got[n + 2, n + 2] - (1 - C)) < TOL64


def test_c1_border_exact(P):
    n, m, C, K = 500, 2500, 0.6, 15
    s, d = er_graph(n, m, 10)
    S = oracle_S(n, s, d, C)
    sr = P.SimRank(n, s, d, S0=S, C=C, K=K, s_precision=64, n_capacity=n + 1)
    sr.apply_updates([(17, n, 1)])
    assert maxabs(sr.dense(), O.inc_c1(n, s, d, S, 17, C)) < TOL64


def test_c2_matches_alg4(P):
    n, m, C, K = 500, 2500, 0.6, 15
    s, d = er_graph(n, m, 11)
    S = oracle_S(n, s, d, C)
    j = int(np.argmax(np.bincount(d, minlength=n)))
    sr = P.SimRank(n, s, d, S0=S, C=C, K=K, s_precision=64, n_capacity=n + 1)
    sr.apply_updates([(n, j, 1)])
    assert maxabs(sr.dense(), O.inc_c2(n, s, d, S, j, C, K)) < TOL64


# --------------------------------------------------------- batches (§8, Alg 6)

@pytest.mark.parametrize("defer", [0, 5])
def test_sink_blocks_fp32_deferred_vs_inc_bsr(P, defer):
    n, m, C, K = 600, 3600, 0.6, 10
    s, d = er_graph(n, m, 14)
    ups, n_new = batch_with_new_nodes(n, s, d, 60, 14, frac_new=0.2, reuse_target=0.5)
    S = oracle_S(n, s, d, C)
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=32, n_capacity=n + n_new,
                   apply=P.APPLY_SINK_BLOCKS, defer=defer, tc=1)
    sr.apply_updates(ups)
    want, _ = O.inc_bsr(n, s, d, S, ups.tolist(), C, K)
    assert maxabs(sr.dense(), want) < TOL32


@pytest.mark.parametrize("seed,chain", [(12, 0), (13, 0), (12, 1)])
def test_sink_blocks_fp64_vs_inc_bsr(P, seed, chain):
    n, m, C, K = 500, 2500, 0.6, 10
    s, d = er_graph(n, m, seed)
    ups, n_new = batch_with_new_nodes(n, s, d, 60, seed, frac_new=0.2, reuse_target=0.5)
    S = oracle_S(n, s, d, C)
    sr = P.SimRank(n, s, d, S0=S, C=C, K=K, s_precision=64, n_capacity=n + n_new,
                   apply=P.APPLY_SINK_BLOCKS, chain=chain)
    sr.apply_updates(ups)
    want, _ = O.inc_bsr(n, s, d, S, ups.tolist(), C, K)
    assert maxabs(sr.dense(), want) < TOL64


# ----------------------------------------------------------- validation paths

def test_invalid_batches_leave_state_unchanged(P):
    n, C = 200, 0.6
    s, d = er_graph(n, 800, 14)
    sr = P.SimRank(n, s, d, C=C, K=5, s_precision=64, n_capacity=n + 2)
    before = sr.dense()
    e0 = (int(s[0]), int(d[0]))
    absent = next((a, b) for a in range(n) for b in range(n)
                  if a != b and (a, b) not in set(zip(s.tolist(), d.tolist())))
    bad = {
        "exists": ([(absent[0], absent[1], 1), (e0[0], e0[1], 1)], 2),
        "missing": ([(absent[0], absent[1], -1)], 3),
        "selfloop": ([(3, 3, 1)], 2),
        "gap": ([(1, n + 1, 1)], 1),
        "capacity": ([(1, n, 1), (2, n + 1, 1), (3, n + 2, 1)], 4),
        "op": ([(1, 2, 0)], 1),
    }
    for name, (ups, code) in bad.items():
        with pytest.raises(P.SimrankError) as ei:
            sr.apply_updates(ups)
        assert ei.value.status == code, name
    assert sr.n == n
    assert np.array_equal(sr.dense(), before)
    sr.apply_updates([])  # empty batch is a no-op
    assert np.array_equal(sr.dense(), before)


def test_reanchor_reaches_fixed_point(P):
    n, m, C, K = 800, 4000, 0.6, 6
    s, d = er_graph(n, m, 15)
    st = update_stream(n, s, d, 20, 16)
    sr = P.SimRank(n, s, d, C=C, K=K, s_precision=64)
    sr.apply_updates(st)
    final = set(zip(s.tolist(), d.tolist()))
    for i, j, op in st.tolist():
        final = final | {(i, j)} if op > 0 else final - {(i, j)}
    ns = np.array([a for a, _ in final])
    nd = np.array([b for _, b in final])
    truth = oracle_S(n, ns, nd, C)
    drift = maxabs(sr.dense(), truth)
    change = sr.reanchor(200)
    assert change < 1e-13
    assert maxabs(sr.dense(), truth) < TOL64
    assert drift > TOL64  # K = 6 left a visible truncation drift before the re-anchor
