"""Pins for the FP64 CPU oracle: each oracle function is checked against
something other than itself (closed forms, printed example values,
brute-force linear solves, independent formulations, invariants)."""
import json
import os

import numpy as np
import pytest

from oracle import simrank_oracle as O
from synth import er_graph, chung_lu_digraph, random_arborescence, update_stream, batch_with_new_nodes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def small_graph(n=12, m=30, seed=0):
    return er_graph(n, m, seed)


# --------------------------------------------------------------------------- O1

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fixed_point_matches_kron_solve(seed):
    n = 9
    s, d = small_graph(n, 20, seed)
    Q = O.transition_matrix(n, s, d)
    for C in (0.6, 0.8):
        S_fp = O.simrank_fixed_point(Q, C)
        S_kr = O.simrank_kron_solve(Q, C)
        assert np.max(np.abs(S_fp - S_kr)) < 1e-12


def test_transition_matrix_by_hand():
    # edges 0->2, 1->2, 2->0 : row 2 has in-neighbours 0 and 1, row 0 has 2
    Q = O.transition_matrix(3, [0, 1, 2], [2, 2, 0])
    expect = np.array([[0, 0, 1.0], [0, 0, 0], [0.5, 0.5, 0]])
    assert np.array_equal(Q, expect)
    Qw = O.transition_matrix(3, [0, 1, 2], [2, 2, 0], weight=[1.0, 3.0, 2.0])
    assert np.allclose(Qw, np.array([[0, 0, 1.0], [0, 0, 0], [0.25, 0.75, 0]]))


@pytest.mark.parametrize("seed", [3, 4])
def test_tree_closed_form(seed):
    """Example 2 (§1): on an arborescence S(a,b) = C^lam (1 - C^{H-lam+1}) for
    a, b on the same level, else 0 (lam = edges from the LCA, H = depth)."""
    n = 25
    par, ch = random_arborescence(n, seed)
    parent = {int(c): int(p) for p, c in zip(par, ch)}
    depth = [0] * n
    for v in range(1, n):
        depth[v] = depth[parent[v]] + 1
    C = 0.7
    S = O.simrank_fixed_point(O.transition_matrix(n, par, ch), C)

    def anc(v, k):
        for _ in range(k):
            v = parent[v]
        return v

    for a in range(n):
        for b in range(n):
            if depth[a] != depth[b]:
                expect = 0.0
            else:
                H = depth[a]
                lam = next(k for k in range(H + 1) if anc(a, k) == anc(b, k))
                expect = C ** lam * (1 - C ** (H - lam + 1))
            assert abs(S[a, b] - expect) < 1e-13


@pytest.mark.parametrize("seed", [5, 6])
def test_invariants(seed):
    n = 40
    s, d = er_graph(n, 120, seed)
    C = 0.6
    S = O.simrank_fixed_point(O.transition_matrix(n, s, d), C)
    assert np.max(np.abs(S - S.T)) < 1e-15
    assert np.all(np.diag(S) >= 1 - C - 1e-15)
    assert np.all(S >= -1e-15) and np.all(S <= 1 + 1e-15)


def test_partial_sim_matches_series_and_fixed_point():
    n = 30
    s, d = er_graph(n, 90, 7)
    C, K = 0.6, 12
    Q = O.transition_matrix(n, s, d)
    S_K = O.simrank_truncated_series(Q, C, K)
    for q in (0, 7, 29):
        assert np.max(np.abs(O.partial_sim(Q, q, K, C) - S_K[:, q])) < 1e-15
    Qs = O.transition_matrix(n, s, d, sparse=True)
    blk = O.partial_sim_block(Qs, [3, 4, 5], K, C)
    assert np.max(np.abs(blk - S_K[:, 3:6])) < 1e-15
    # converged: the truncation error is at most C^{K+1}
    S = O.simrank_kron_solve(Q, C)
    assert np.max(np.abs(O.partial_sim(Q, 11, 60, C) - S[:, 11])) < 1e-13
    assert np.max(np.abs(S_K - S)) <= C ** (K + 1)


# ------------------------------------------------------ printed example values

def test_thm1_example():
    g = load("example_thm1.json")
    # nodes: h=0, i=1, j=2, k=3 ; j's in-neighbours h and k
    Q = O.transition_matrix(4, [0, 3], [2, 2])
    u, v = O.rank_one_factors(Q, g["d_j"], 2, [1], O.INSERT)
    names = {"h": 0, "i": 1, "j": 2, "k": 3}
    eu = np.zeros(4)
    ev = np.zeros(4)
    for k, x in g["u"].items():
        eu[names[k]] = x
    for k, x in g["v"].items():
        ev[names[k]] = x
    assert np.allclose(u, eu) and np.allclose(v, ev)
    # and the factors reproduce the new Q exactly
    Qn = O.transition_matrix(4, [0, 3, 1], [2, 2, 2])
    assert np.max(np.abs(Q + np.outer(u, v) - Qn)) < 1e-15


def test_alg1_example_gamma():
    g = load("example_alg1.json")
    names = ["a", "b", "f", "i", "j"]
    idx = {x: t for t, x in enumerate(names)}
    n = len(names)
    w = np.zeros(n)
    for k, x in g["w"].items():
        w[idx[k]] = x
    col = np.zeros(n)
    for k, x in g["S_col_j"].items():
        col[idx[k]] = x
    gamma, lam = O.gamma_sink_block(w, col, g["S_ii"], g["S_jj"], g["d_j"], 1, O.INSERT, g["C"], idx["j"])
    assert round(lam, g["decimals"]) == g["lambda"]
    for k, x in g["gamma"].items():
        assert round(gamma[idx[k]], g["decimals"]) == pytest.approx(x, abs=1e-12), k


def test_c2_example_z():
    """Eq. 60 through the oracle's Alg 4 step (z is the start of eta)."""
    g = load("example_c2_z.json")
    C, d = g["C"], g["d_j"]
    names = ["f", "i", "j"]
    idx = {x: t for t, x in enumerate(names)}
    col = np.zeros(3)
    for k, x in g["S_col_j"].items():
        col[idx[k]] = x
    j = idx["j"]
    ej = np.eye(3)[j]
    z = ((col[j] - (1 - C) ** 2) / (2 * C * (d + 1)) + (1 - C) / C) * ej - col / C
    for k, x in g["z"].items():
        assert round(z[idx[k]], g["decimals"]) == pytest.approx(x, abs=1e-12)
    # the same z drives the oracle's inc_c2: check it through a graph where
    # j has exactly two in-neighbours and K = 0 (M = e_j z^T)
    n = 4  # nodes 0=f, 1=i, 2=j, 3=x ; j's in-neighbours: f, x
    s, dd = [0, 3], [2, 2]
    S = np.zeros((4, 4))
    S[:3, :3] = np.diag([1, 1, 1]) * 0.0
    S[:, 2] = [0.2064, 0.3104, 0.5104, 0.0]
    S[2, :] = S[:, 2]
    S_new = O.inc_c2(n, s, dd, S, 2, C, 0)
    dS = S_new[:n, :n] - S
    z4 = np.zeros(4)
    z4[:3] = z
    z4[3] = 0.0
    e = np.eye(4)[2]
    assert np.max(np.abs(dS - C / (d + 1) * (np.outer(e, z4) + np.outer(z4, e)))) < 1e-15


def test_c1_example_corner():
    g = load("example_c1_corner.json")
    # graph: node 0 (= i) alone; inc_c1 appends the new node
    S = np.array([[g["S_ii"]]])
    S_new = O.inc_c1(1, [], [], S, 0, g["C"])
    assert round(S_new[1, 1], g["decimals"]) == g["corner"]


def test_batch_example_net_and_partition():
    g = load("example_batch.json")
    names = sorted({x for u in g["updates"] for x in u[:2]})
    new = set(g["new_nodes"])
    old_names = [x for x in names if x not in new]
    ids = {x: t for t, x in enumerate(old_names + sorted(new))}
    ups = [(ids[a], ids[b], 1 if op == "+" else -1) for a, b, op in g["updates"]]
    plus, minus = O.net_update(ups)
    inv = {t: x for x, t in ids.items()}
    assert [[inv[a], inv[b]] for a, b in plus] == g["net_plus"]
    assert [[inv[a], inv[b]] for a, b in minus] == g["net_minus"]
    n_old = len(old_names)
    dels, ins = O.partition_similar_sink(plus, minus, lambda x: x < n_old)
    got_ins = {(inv[j], tuple(sorted(inv[i] for i in srcs))) for j, srcs in ins}
    want_ins = {(j, tuple(sorted(s))) for j, s in g["insertion_blocks"]}
    assert got_ins == want_ins
    got_del = {(inv[j], tuple(sorted(inv[i] for i in srcs))) for j, srcs in dels}
    assert got_del == {(j, tuple(sorted(s))) for j, s in g["deletion_blocks"]}


def test_net_update_rejects_double_insert():
    with pytest.raises(ValueError):
        O.net_update([(0, 1, 1), (0, 1, 1)])


# ------------------------------------------------------------ Thm 2 / Alg 1

def test_li_counterexample_two_cycle():
    """Appendix A, Examples 2-3: Q = [[0,1],[0,0]] (edge 2->1), insert 1->2.
    Old S = diag(1 - C^2, 1 - C); the new graph is a 2-cycle with S = I."""
    C = 0.6
    src, dst = [1], [0]
    Q = O.transition_matrix(2, src, dst)
    S = O.simrank_kron_solve(Q, C)
    assert np.allclose(S, np.diag([1 - C * C, 1 - C]), atol=1e-15)
    S_new = O.inc_usr(2, src, dst, S, 1, [0], O.INSERT, C, 200)
    assert np.max(np.abs(S_new - np.eye(2))) < 1e-13


@pytest.mark.parametrize("op", [O.INSERT, O.DELETE])
@pytest.mark.parametrize("seed", [10, 11, 12])
def test_inc_usr_converges_to_new_fixed_point(op, seed):
    """Alg 1 at large K against a brute-force solve of Eq. 1 on the new graph."""
    n = 10
    s, d = er_graph(n, 26, seed)
    C = 0.6
    rng = np.random.default_rng(seed)
    edges = set(zip(s.tolist(), d.tolist()))
    if op == O.INSERT:
        while True:
            i, j = map(int, rng.integers(0, n, 2))
            if i != j and (i, j) not in edges:
                break
        new = edges | {(i, j)}
    else:
        i, j = list(edges)[int(rng.integers(0, len(edges)))]
        new = edges - {(i, j)}
    S = O.simrank_kron_solve(O.transition_matrix(n, s, d), C)
    S_new = O.inc_usr(n, s, d, S, j, [i], op, C, 120)
    ns = np.array([a for a, _ in new])
    nd = np.array([b for _, b in new])
    S_true = O.simrank_kron_solve(O.transition_matrix(n, ns, nd), C)
    assert np.max(np.abs(S_new - S_true)) < 1e-12


@pytest.mark.parametrize("case", ["ins0", "ins", "del1", "del"])
def test_thm3_gamma_equals_thm2_w(case):
    """At the exact fixed point, Thm 3/9's gamma (built with Eq. 33) equals
    Thm 2's general w scaled by u's factor; and the two M_K agree."""
    n = 14
    C, K = 0.7, 9
    s, d = er_graph(n, 40, 21)
    edges = set(zip(s.tolist(), d.tolist()))
    deg = O.in_degrees(n, d)
    outs = {}
    for a, b in edges:
        outs.setdefault(b, []).append(a)
    if case == "ins0":
        j = int(np.nonzero(deg == 0)[0][0]) if np.any(deg == 0) else None
        if j is None:
            s = s[d != 3]
            d = d[d != 3]
            j = 3
        i = 0 if j != 0 else 1
        op = O.INSERT
    elif case == "ins":
        j = int(np.argmax(deg))
        i = next(x for x in range(n) if x != j and (x, j) not in edges)
        op = O.INSERT
    elif case == "del1":
        j = int(np.nonzero(deg == 1)[0][0])
        i = outs[j][0]
        op = O.DELETE
    else:
        j = int(np.argmax(deg))
        i = outs[j][0]
        op = O.DELETE
    Q = O.transition_matrix(n, s, d)
    S = O.simrank_kron_solve(Q, C)
    dj = int(O.in_degrees(n, d)[j])
    u, v = O.rank_one_factors(Q, dj, j, [i], op)
    w_general = O.thm2_w(Q, S, u, v)
    gamma, _ = O.gamma_sink_block(Q @ S[:, i], S[:, j], S[i, i], S[j, j], dj, 1, op, C, j)
    scale = u[j]
    assert np.max(np.abs(gamma - scale * w_general)) < 1e-13
    # Alg 1's sum of xi eta^T against the conventional dense recurrence
    _, M, _ = O.inc_usr(n, s, d, S, j, [i], op, C, K, return_terms=True)
    Qn = Q + np.outer(u, v)
    M_conv = O.sylvester_conventional(Qn, u, w_general, C, K)
    assert np.max(np.abs(M - M_conv)) < 1e-13


def test_truncation_bound():
    """Footnote of Appendix D.1: ||M_K - M||_max <= C^{K+1} (M = K -> inf)."""
    n = 12
    s, d = er_graph(n, 35, 30)
    C = 0.8
    S = O.simrank_kron_solve(O.transition_matrix(n, s, d), C)
    edges = set(zip(s.tolist(), d.tolist()))
    i, j = next((a, b) for a in range(n) for b in range(n) if a != b and (a, b) not in edges)
    _, M_inf, _ = O.inc_usr(n, s, d, S, j, [i], O.INSERT, C, 300, return_terms=True)
    for K in (3, 8, 15):
        _, M_K, _ = O.inc_usr(n, s, d, S, j, [i], O.INSERT, C, K, return_terms=True)
        assert np.max(np.abs(M_K - M_inf)) <= C ** (K + 1)


@pytest.mark.parametrize("seed", [40, 41])
def test_thm4_affected_areas(seed):
    """Thm 4: M_k is zero outside (A_k x B_k) u (A_0 x B_0)."""
    n = 30
    s, d = er_graph(n, 45, seed)
    C, K = 0.6, 6
    S = O.simrank_fixed_point(O.transition_matrix(n, s, d), C)
    edges = set(zip(s.tolist(), d.tolist()))
    deg = O.in_degrees(n, d)
    j = int(np.argmax(deg))
    i = next(x for x in range(n) if x != j and (x, j) not in edges)
    _, _, terms = O.inc_usr(n, s, d, S, j, [i], O.INSERT, C, K, return_terms=True)
    sets = O.affected_sets(n, s, d, S, i, j, O.INSERT, K, terms)
    M = np.zeros((n, n))
    A0, B0 = sets[0]
    for k in range(K + 1):
        xi, eta = terms[k]
        M = M + np.outer(xi, eta)
        A, B = sets[k]
        allowed = np.outer(A, B) | np.outer(A0, B0)
        assert np.all(M[~allowed] == 0)


# ----------------------------------------------------------- new-node cases

def _dense_new(n_final, edges, C):
    s = np.array([a for a, _ in edges], np.int64)
    d = np.array([b for _, b in edges], np.int64)
    return O.simrank_kron_solve(O.transition_matrix(n_final, s, d), C)


def test_new_node_cases_exact():
    """Alg 3/4/5 (C1/C2/C3) against a brute-force solve of the grown graph."""
    n = 9
    s, d = er_graph(n, 22, 50)
    C = 0.6
    edges = set(zip(s.tolist(), d.tolist()))
    S = O.simrank_kron_solve(O.transition_matrix(n, s, d), C)
    deg = O.in_degrees(n, d)
    i = 2
    S1 = O.inc_c1(n, s, d, S, i, C)
    assert np.max(np.abs(S1 - _dense_new(n + 1, edges | {(i, n)}, C))) < 1e-13
    j = int(np.argmax(deg))
    S2 = O.inc_c2(n, s, d, S, j, C, 150)
    assert np.max(np.abs(S2 - _dense_new(n + 1, edges | {(n, j)}, C))) < 1e-12
    S3 = O.inc_c3(S, C)
    assert np.max(np.abs(S3 - _dense_new(n + 2, edges | {(n, n + 1)}, C))) < 1e-13


@pytest.mark.parametrize("K", [0, 3, 10])
def test_new_nodes_as_isolated_nodes_term_by_term(K):
    """Pre-allocating new nodes as isolated nodes turns C1/C2/C3 into Alg 1
    with d_j = 0 or d_j > 0; the results agree at any K."""
    n = 10
    s, d = er_graph(n, 25, 51)
    C = 0.7
    S = O.simrank_fixed_point(O.transition_matrix(n, s, d), C)
    deg = O.in_degrees(n, d)

    def padded(extra):
        P = np.zeros((n + extra, n + extra))
        P[:n, :n] = S
        for x in range(n, n + extra):
            P[x, x] = 1 - C
        return P

    i = 4
    lit = O.inc_c1(n, s, d, S, i, C)
    red = O.inc_usr(n + 1, s, d, padded(1), n, [i], O.INSERT, C, K)
    assert np.max(np.abs(lit - red)) < 1e-13
    j = int(np.argmax(deg))
    lit = O.inc_c2(n, s, d, S, j, C, K)
    red = O.inc_usr(n + 1, s, d, padded(1), j, [n], O.INSERT, C, K)
    assert np.max(np.abs(lit - red)) < 1e-13
    lit = O.inc_c3(S, C)
    red = O.inc_usr(n + 2, s, d, padded(2), n + 1, [n], O.INSERT, C, K)
    assert np.max(np.abs(lit - red)) < 1e-13


# -------------------------------------------------------------- batch (§8)

@pytest.mark.parametrize("seed", [60, 61, 62])
def test_inc_bsr_literal_vs_isolated_and_exact(seed):
    n = 10
    s, d = er_graph(n, 24, seed)
    C = 0.6
    S = O.simrank_kron_solve(O.transition_matrix(n, s, d), C)
    ups, n_new = batch_with_new_nodes(n, s, d, 9, seed, frac_new=0.45, reuse_target=0.5)
    n_final = n + n_new
    for K in (2, 7):
        lit, e1 = O.inc_bsr(n, s, d, S, ups.tolist(), C, K)
        red, e2 = O.inc_bsr_isolated(n, n_final, s, d, S, ups.tolist(), C, K)
        assert e1 == e2
        assert np.max(np.abs(lit - red)) < 1e-13
    lit, edges = O.inc_bsr(n, s, d, S, ups.tolist(), C, 160)
    assert np.max(np.abs(lit - _dense_new(n_final, edges, C))) < 1e-12


def test_table2_c0_block_exact():
    """A C0 sink block of delta insertions, then the same block deleted."""
    n = 11
    s, d = er_graph(n, 26, 70)
    C = 0.6
    edges = set(zip(s.tolist(), d.tolist()))
    deg = O.in_degrees(n, d)
    j = int(np.argmax(deg))
    srcs = [x for x in range(n) if x != j and (x, j) not in edges][:3]
    S = O.simrank_kron_solve(O.transition_matrix(n, s, d), C)
    S1 = O.inc_usr(n, s, d, S, j, srcs, O.INSERT, C, 160)
    e1 = edges | {(x, j) for x in srcs}
    assert np.max(np.abs(S1 - _dense_new(n, e1, C))) < 1e-12
    s1 = np.array([a for a, _ in e1])
    d1 = np.array([b for _, b in e1])
    S2 = O.inc_usr(n, s1, d1, S1, j, srcs, O.DELETE, C, 160)
    assert np.max(np.abs(S2 - S)) < 1e-12
    # deleting every in-edge of a sink (d_j = delta branch)
    ins_j = sorted(a for a, b in edges if b == j)
    S3 = O.inc_usr(n, s, d, S, j, ins_j, O.DELETE, C, 160)
    assert np.max(np.abs(S3 - _dense_new(n, {e for e in edges if e[1] != j}, C))) < 1e-12


@pytest.mark.parametrize("seed", [80, 81])
def test_one_shot_batch(seed):
    """The one-shot form converges to the new fixed point, and at finite K its
    T equals the low-rank U W^T + W U^T of the proof of Thm 2."""
    n = 10
    s, d = er_graph(n, 24, seed)
    C = 0.6
    S = O.simrank_kron_solve(O.transition_matrix(n, s, d), C)
    ups, n_new = batch_with_new_nodes(n, s, d, 8, seed, frac_new=0.4)
    n_final = n + n_new
    Sp = np.zeros((n_final, n_final))
    Sp[:n, :n] = S
    for x in range(n, n_final):
        Sp[x, x] = 1 - C
    edges = set(zip(s.tolist(), d.tolist()))
    plus, minus = O.net_update(ups.tolist())
    new = (edges | set(plus)) - set(minus)
    ns = np.array([a for a, _ in new])
    nd = np.array([b for _, b in new])
    S_one = O.one_shot_batch(n_final, s, d, ns, nd, Sp, C, 170)
    assert np.max(np.abs(S_one - _dense_new(n_final, new, C))) < 1e-12


# --------------------------------------------------------- column mode (§7)

def test_inc_sr_all_p_matches_sequential_at_large_k():
    n = 9
    s, d = er_graph(n, 20, 90)
    C = 0.6
    S = O.simrank_kron_solve(O.transition_matrix(n, s, d), C)
    ups = [(0, 5, 1), (3, 5, 1), (n, 2, 1), (1, n + 1, 1), (n + 2, n + 3, 1)]
    edges = set(zip(s.tolist(), d.tolist()))
    u = next(e for e in sorted(edges) if e[0] < n and e[1] < n and (e[0], e[1]) not in {(0, 5), (3, 5)})
    ups.append((u[0], u[1], -1))
    final = set(edges)
    for i, j, op in ups:
        if op > 0:
            final.add((i, j))
        else:
            final.discard((i, j))
    n_final = n + 4
    S_true = _dense_new(n_final, final, C)
    for x in (0, 5, n, n + 1, n + 3):
        col0 = S[:, x] if x < n else None
        col = O.inc_sr_all_p(n, s, d, col0 if col0 is not None else np.zeros(n), x, ups, C, 140)
        assert np.max(np.abs(col - S_true[:, x])) < 1e-11, x


# ---------------------------------------------------------------- gradient

def test_pair_loss_gradient_vs_finite_differences():
    n = 14
    s, d = er_graph(n, 40, 95)
    rng = np.random.default_rng(95)
    w = rng.uniform(0.1, 1.0, size=s.size)
    a = rng.integers(0, n, 6)
    b = rng.integers(0, n, 6)
    t = rng.uniform(0, 0.3, 6)
    C, K = 0.6, 7
    L, g, S = O.pair_loss_and_weight_grad(n, s, d, w, a, b, t, C, K)
    assert abs(L - O.pair_loss(n, s, d, w, a, b, t, C, K)) < 1e-13
    assert np.max(np.abs(S - O.simrank_truncated_series(O.transition_matrix(n, s, d, w), C, K))) < 1e-14
    for e in range(0, s.size, 5):
        h = 1e-5
        wp = w.copy()
        wp[e] += h
        wm = w.copy()
        wm[e] -= h
        fd = (O.pair_loss(n, s, d, wp, a, b, t, C, K) - O.pair_loss(n, s, d, wm, a, b, t, C, K)) / (2 * h)
        assert abs(fd - g[e]) < 1e-8 * max(1.0, abs(fd))


def test_generators_are_seeded_and_simple():
    s1, d1 = chung_lu_digraph(500, 2500, 2.1, 2.1, 3)
    s2, d2 = chung_lu_digraph(500, 2500, 2.1, 2.1, 3)
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    assert np.all(s1 != d1)
    assert len(set(zip(s1.tolist(), d1.tolist()))) == 2500
    st = update_stream(500, s1, d1, 50, 4)
    assert st.shape == (50, 3)


def test_sequential_stream_converges_to_final_fixed_point():
    n = 12
    s, d = er_graph(n, 30, 97)
    C = 0.6
    S = O.simrank_kron_solve(O.transition_matrix(n, s, d), C)
    st = update_stream(n, s, d, 6, 98)
    S_seq, edges = O.sequential_unit_updates(n, s, d, S, st.tolist(), C, 150)
    assert np.max(np.abs(S_seq - _dense_new(n, edges, C))) < 1e-12


# ------------------------------------------------ finite-K pins (Thm 2, Alg 7, Thm 4)

def _exact(n, s, d, C):
    return O.simrank_kron_solve(O.transition_matrix(n, s, d), C)


def _edge_arrays(edges):
    return (np.array([a for a, _ in edges], np.int64), np.array([b for _, b in edges], np.int64))


@pytest.mark.parametrize("K", [0, 1, 3, 7])
def test_one_shot_batch_single_block_equals_inc_usr(K):
    """A batch that is one sink block is a rank-one change of Q, so the proof
    of Thm 2 (Eqs 23-28) gives T = Q_new S Q_new^T - Q S Q^T = u w^T + w u^T
    exactly, and the one-shot series equals Alg 1's M_K + M_K^T at the same K
    (insert with d_j > 0, insert into an isolated node, delete with d_j > 1 and
    with d_j = 1, a block of two insertions into one sink)."""
    n = 11
    s, d = er_graph(n, 28, 300)
    C = 0.6
    edges = set(zip(s.tolist(), d.tolist()))
    deg = O.in_degrees(n, d)
    S = _exact(n, s, d, C)
    j = int(np.argmax(deg))
    absent = [x for x in range(n) if x != j and (x, j) not in edges]
    iso = int(np.argmin(deg))
    i_iso = next(x for x in range(n) if x != iso and (x, iso) not in edges)
    e_many = next(e for e in sorted(edges) if deg[e[1]] > 1)
    cases = [(j, [absent[0]], O.INSERT), (iso, [i_iso], O.INSERT),
             (e_many[1], [e_many[0]], O.DELETE), (j, absent[1:3], O.INSERT)]
    d1 = next((e for e in sorted(edges) if deg[e[1]] == 1), None)
    if d1 is not None:
        cases.append((d1[1], [d1[0]], O.DELETE))
    for sink, srcs, op in cases:
        new = (edges | {(x, sink) for x in srcs}) if op > 0 else (edges - {(x, sink) for x in srcs})
        ns, nd = _edge_arrays(new)
        one = O.one_shot_batch(n, s, d, ns, nd, S, C, K)
        alg1 = O.inc_usr(n, s, d, S, sink, srcs, op, C, K)
        assert np.max(np.abs(one - alg1)) < 1e-13, (sink, srcs, op)
    # K and K + 1 differ, so an off-by-one in the series length fails above
    sink, srcs, op = cases[0]
    ns, nd = _edge_arrays(edges | {(srcs[0], sink)})
    gap = np.max(np.abs(O.one_shot_batch(n, s, d, ns, nd, S, C, K + 1) - O.inc_usr(n, s, d, S, sink, srcs, op, C, K)))
    assert gap > 1e-9


@pytest.mark.parametrize("K", [0, 2, 5])
def test_inc_sr_all_p_single_update_finite_k(K):
    """Alg 7 for one update at the same K as Alg 1: with converged old columns
    (K_old large) column x equals column x of Alg 1 applied to the exact S;
    with K_old = K (Alg 7 as printed) it equals Alg 1 applied to the truncated
    S_K of Eq. 17, whose columns are exactly what Procedure 1 returns.  C0
    insert, C0 delete with d_j > 1 and with d_j = 1; C2 against Alg 4, C1
    against Alg 3."""
    n = 10
    s, d = er_graph(n, 24, 301)
    C = 0.6
    edges = set(zip(s.tolist(), d.tolist()))
    deg = O.in_degrees(n, d)
    S = _exact(n, s, d, C)
    S_K = O.simrank_truncated_series(O.transition_matrix(n, s, d), C, K)
    j = int(np.argmax(deg))
    i = next(x for x in range(n) if x != j and (x, j) not in edges)
    e_many = next(e for e in sorted(edges) if deg[e[1]] > 1)
    ups = [(i, j, O.INSERT), (e_many[0], e_many[1], O.DELETE)]
    d1 = next((e for e in sorted(edges) if deg[e[1]] == 1), None)
    if d1 is not None:
        ups.append((d1[0], d1[1], O.DELETE))
    for ii, jj, op in ups:
        conv = O.inc_usr(n, s, d, S, jj, [ii], op, C, K)
        trunc = O.inc_usr(n, s, d, S_K, jj, [ii], op, C, K)
        for x in (0, ii, jj, n - 1):
            col = O.inc_sr_all_p(n, s, d, S[:, x], x, [(ii, jj, op)], C, K, K_old=200)
            assert np.max(np.abs(col - conv[:, x])) < 1e-13, (ii, jj, op, x)
            col = O.inc_sr_all_p(n, s, d, S_K[:, x], x, [(ii, jj, op)], C, K)
            assert np.max(np.abs(col - trunc[:, x])) < 1e-13, (ii, jj, op, x)
    # C2: a new source into j (Alg 4 at the same K)
    lit = O.inc_c2(n, s, d, S, j, C, K)
    for x in (0, j, n - 1, n):
        col = O.inc_sr_all_p(n, s, d, S[:, x] if x < n else np.zeros(n), x, [(n, j, 1)], C, K, K_old=200)
        assert np.max(np.abs(col - lit[:, x])) < 1e-13, ("C2", x)
    # C1: a new sink fed by i (Alg 3; no truncation enters)
    lit = O.inc_c1(n, s, d, S, i, C)
    for x in (0, i, n):
        col = O.inc_sr_all_p(n, s, d, S[:, x] if x < n else np.zeros(n), x, [(i, n, 1)], C, K, K_old=200)
        assert np.max(np.abs(col - lit[:, x])) < 1e-13, ("C1", x)


def _mask(n, nodes):
    m = np.zeros(n, bool)
    m[list(nodes)] = True
    return m


def test_thm4_affected_sets_exact_on_hand_built_tree():
    """Thm 4 (Eqs 39-41) worked by hand on the tree 0->1, 0->2, 1->3, 2->4,
    3->5, 4->6 (levels {0}, {1,2}, {3,4}, {5,6}; S is non-zero exactly on
    pairs of one level).
    Insert (4, 3), d_3 = 1: F1 = O(3) u O(4) = {5, 6}, F2 = {3, 4}, so
    A_0 x B_0 = {3} x {3,4,5,6}; M_0 = xi_0 eta_0^T has rows {3}, columns
    {3,4,5,6} -> A_1 x B_1 = O~(3) x O~({3,4,5,6}) = {5} x {3,5,6}; xi_1 is
    supported on {5} and eta_1 on {3,5,6}, so M_1 has rows {3,5} and columns
    {3,4,5,6} -> A_2 x B_2 = {5} x {3,5,6}; xi_2 = 0, so every later set is
    the same.
    Delete (1, 3), d_3 = 1: F2 is empty, F1 = O(1) u O(2) = {3, 4}:
    A_0 x B_0 = {3} x {3,4}, A_1 x B_1 = {5} x {5,6}, and from k = 2 on
    {5} x {5,6}."""
    n = 7
    tree = [(0, 1), (0, 2), (1, 3), (2, 4), (3, 5), (4, 6)]
    s, d = _edge_arrays(tree)
    C, K = 0.6, 5
    S = O.simrank_fixed_point(O.transition_matrix(n, s, d), C)
    for (i, j, op), want in (
        ((4, 3, O.INSERT), [({3}, {3, 4, 5, 6}), ({5}, {3, 5, 6})] + [({5}, {3, 5, 6})] * (K - 1)),
        ((1, 3, O.DELETE), [({3}, {3, 4}), ({5}, {5, 6})] + [({5}, {5, 6})] * (K - 1)),
    ):
        _, _, terms = O.inc_usr(n, s, d, S, j, [i], op, C, K, return_terms=True)
        sets = O.affected_sets(n, s, d, S, i, j, op, K, terms)
        assert len(sets) == K + 1
        for k, ((A, B), (wa, wb)) in enumerate(zip(sets, want)):
            assert np.array_equal(A, _mask(n, wa)), (op, k, np.nonzero(A)[0])
            assert np.array_equal(B, _mask(n, wb)), (op, k, np.nonzero(B)[0])


@pytest.mark.parametrize("K", [0, 3, 10])
def test_alg1_stream_columns_equals_dense_sequential(K):
    """The column form of a sequential Alg 1 stream equals the dense form
    (sequential_unit_updates, pinned above) column by column at the same K."""
    n = 14
    s, d = er_graph(n, 40, 310)
    C = 0.6
    S = _exact(n, s, d, C)
    st = update_stream(n, s, d, 7, 311)
    dense, _ = O.sequential_unit_updates(n, s, d, S, st.tolist(), C, K)
    query = [0, 3, 7, int(st[0, 1]), n - 1]
    cols = O.alg1_stream_columns(n, s, d, lambda c: S[:, c], st.tolist(), C, K, query)
    assert np.max(np.abs(cols - dense[:, query])) < 1e-13


@pytest.mark.parametrize("K", [0, 2, 5])
def test_inc_sr_all_p_blocks_single_block_finite_k(K):
    """One sink block through the column form of Alg 7 x §8 at the same K as
    Alg 1 on the exact S (converged old columns): a two-edge insertion block, a
    two-edge deletion block, and a block into a new (isolated) sink."""
    n = 11
    s, d = er_graph(n, 30, 320)
    C = 0.6
    edges = set(zip(s.tolist(), d.tolist()))
    deg = O.in_degrees(n, d)
    S = _exact(n, s, d, C)
    j = int(np.argmax(deg))
    ins = [x for x in range(n) if x != j and (x, j) not in edges][:2]
    jd = next(b for b in range(n) if deg[b] >= 3)
    dels = sorted(a for a, b in edges if b == jd)[:2]
    for srcs, sink, op in ((ins, j, O.INSERT), (dels, jd, O.DELETE)):
        want = O.inc_usr(n, s, d, S, sink, srcs, op, C, K)
        ups = [(i, sink, op) for i in srcs]
        for x in (0, sink, srcs[0], n - 1):
            col = O.inc_sr_all_p_blocks(n, n, s, d, S[:, x], x, ups, C, K, K_old=200)
            assert np.max(np.abs(col - want[:, x])) < 1e-13, (op, x)
    # two old sources into a new sink n: Alg 1 on the graph padded with the isolated node
    Sp = np.zeros((n + 1, n + 1))
    Sp[:n, :n] = S
    Sp[n, n] = 1 - C
    want = O.inc_usr(n + 1, s, d, Sp, n, ins, O.INSERT, C, K)
    for x in (0, ins[0], n):
        col = O.inc_sr_all_p_blocks(n, n + 1, s, d, S[:, x] if x < n else None, x,
                                    [(i, n, 1) for i in ins], C, K, K_old=200)
        assert np.max(np.abs(col - want[:, x])) < 1e-13, ("new sink", x)


def test_inc_sr_all_p_blocks_batch_converges():
    """A batch with insertions, deletions and new nodes at large K equals the
    brute-force fixed point of the final graph, column by column."""
    n = 10
    s, d = er_graph(n, 24, 321)
    C = 0.6
    S = _exact(n, s, d, C)
    ups, n_new = batch_with_new_nodes(n, s, d, 9, 322, frac_new=0.4, reuse_target=0.5)
    n_final = n + n_new
    _, edges = O.inc_bsr(n, s, d, S, ups.tolist(), C, 2)
    S_true = _dense_new(n_final, edges, C)
    for x in (0, 4, n - 1, n_final - 1):
        col = O.inc_sr_all_p_blocks(n, n_final, s, d, S[:, x] if x < n else None, x, ups.tolist(),
                                    C, 150)
        assert np.max(np.abs(col - S_true[:, x])) < 1e-11, x
