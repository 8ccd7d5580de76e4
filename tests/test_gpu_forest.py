"""Incremental SimRank as a batch accelerator (§1, Examples 1 and 2), through
the C ABI.  Example 2: S of a forest of arborescences in closed form on the
GPU (init_form = SR_INIT_FOREST) against the FP64 fixed point of Eq. 1, then
the non-tree edges applied as one batch (one-shot rank-2r form and sink
blocks) against the oracle at the same K and against the converged fixed
point of the whole graph.  Example 1: S of the block-diagonal graph, then the
cross-block edges applied as a batch, against the fixed point of the whole
graph."""
import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import random_forest, tree_with_extra_edges, block_graph

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


@pytest.mark.parametrize("prec,relabel,upper", [(64, 1, 1), (64, 0, 0), (32, 1, 1)])
def test_forest_init_matches_fixed_point(P, prec, relabel, upper):
    sizes = [300, 250, 170, 1]
    s, d = random_forest(sizes, 81)
    n = sum(sizes)
    C = 0.7
    h = P.SimRank(n, s, d, C=C, K=5, s_precision=prec, init_form=P.INIT_FOREST,
                  relabel=relabel, upper_only=upper, n_capacity=n + 9)
    got = h.dense()
    assert h.stats()["init_sweeps"] == 0
    h.close()
    want = O.simrank_fixed_point(O.transition_matrix(n, s, d, sparse=True), C, tol=1e-15)
    assert np.max(np.abs(got - want)) < (1e-12 if prec == 64 else TOL32)


def test_forest_init_rejects_non_forests(P):
    # a node with two in-neighbours
    with pytest.raises(P.SimrankError) as e:
        P.SimRank(4, [0, 1, 2], [2, 2, 3], init_form=P.INIT_FOREST)
    assert e.value.status == 1 and "in-degree" in str(e.value)
    # every in-degree is one, but the graph is a cycle
    with pytest.raises(P.SimrankError) as e:
        P.SimRank(3, [0, 1, 2], [1, 2, 0], init_form=P.INIT_FOREST)
    assert e.value.status == 1 and "cycle" in str(e.value)


def edges_arrays(edges):
    return (np.array([a for a, _ in edges], np.int64), np.array([b for _, b in edges], np.int64))


@pytest.mark.parametrize("form", ["one_shot_fp64", "one_shot_tc", "sink_blocks_fp64"])
def test_tree_then_non_tree_edges(P, form):
    """Example 2: closed-form S of the tree, then the non-tree edges as one batch."""
    n, extra, C = 600, 40, 0.6
    ts, td, xs, xd = tree_with_extra_edges(n, extra, 82)
    tree = set(zip(ts.tolist(), td.tolist()))
    ups = np.stack([xs, xd, np.ones(extra, np.int32)], axis=1)
    S_tree = O.simrank_fixed_point(O.transition_matrix(n, ts, td, sparse=True), C, tol=1e-15)
    full = tree | set(zip(xs.tolist(), xd.tolist()))
    fs, fd = edges_arrays(full)
    for K in (6, 70):
        kw = dict(C=C, K=K, init_form=P.INIT_FOREST)
        if form == "one_shot_fp64":
            kw.update(s_precision=64, apply=P.APPLY_ONE_SHOT)
        elif form == "one_shot_tc":
            kw.update(s_precision=32, apply=P.APPLY_ONE_SHOT, tc=1)
        else:
            kw.update(s_precision=64, apply=P.APPLY_SINK_BLOCKS)
        h = P.SimRank(n, ts, td, **kw)
        h.apply_updates(ups)
        got = h.dense()
        h.close()
        tol = TOL32 if form == "one_shot_tc" else TOL64
        if K == 6:
            if form.startswith("one_shot"):
                want = O.one_shot_batch(n, ts, td, fs, fd, S_tree, C, K)
            else:
                want, _ = O.inc_bsr_isolated(n, n, ts, td, S_tree, ups.tolist(), C, K)
        else:
            # C^(K+2) / (1 - C) < 1e-15: the converged S of the whole graph
            want = O.simrank_fixed_point(O.transition_matrix(n, fs, fd, sparse=True), C, tol=1e-15)
        assert np.max(np.abs(got - want)) < tol, (form, K)


@pytest.mark.parametrize("init_form", ["components", "sweeps"])
def test_blocks_then_cross_edges(P, init_form):
    """Example 1: S of the graph without its cross-block edges, computed block
    by block (SR_INIT_COMPONENTS: here two bins, 2,500 nodes and 2,000 + 1,500
    nodes) or by sweeps over the whole matrix, is block diagonal; the
    cross-block edges then applied as sink blocks at K = 70 give the fixed
    point of the whole graph (sampled columns against Procedure 1)."""
    sizes, C, K = [2500, 2000, 1500], 0.6, 70
    bs, bd, xs, xd = block_graph(sizes, 5, 60, 83)
    n = sum(sizes)
    ups = np.stack([xs, xd, np.ones(xs.size, np.int32)], axis=1)
    form = P.INIT_COMPONENTS if init_form == "components" else P.INIT_SWEEPS
    h = P.SimRank(n, bs, bd, C=C, K=K, s_precision=64, apply=P.APPLY_SINK_BLOCKS,
                  init_form=form)
    rng = np.random.default_rng(84)
    cols = np.array(sorted(set(rng.choice(n, 14, replace=False).tolist()) | set(xd[:4].tolist())),
                    np.int32)
    old = h.columns(cols)
    want_old = O.partial_sim_block(O.transition_matrix(n, bs, bd, sparse=True), cols, 80, C)
    assert np.max(np.abs(old - want_old)) < 1e-12
    off = np.cumsum([0] + sizes)
    for c, x in enumerate(cols.tolist()):
        blk = int(np.searchsorted(off, x, side="right") - 1)
        outside = np.ones(n, bool)
        outside[off[blk]:off[blk + 1]] = False
        assert np.all(old[outside, c] == 0.0), x
    h.apply_updates(ups)
    got = h.columns(cols)
    h.close()
    fs = np.concatenate([bs, xs])
    fd = np.concatenate([bd, xd])
    want = O.partial_sim_block(O.transition_matrix(n, fs, fd, sparse=True), cols, 80, C)
    assert np.max(np.abs(got - want)) < TOL64
