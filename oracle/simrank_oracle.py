"""Plain FP64 CPU oracle for incremental SimRank (Yu, Lin, Zhang, McCann,
"Dynamical SimRank Search on Time-Varying Networks").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this module: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA library: it builds its own transition matrices
from edge lists and does every step with dense NumPy (or SciPy sparse)
arithmetic in float64.

Conventions (§3.1): an edge (i, j) means i -> j; Q is the backward transition
matrix, [Q]_{a,b} = 1/in-degree(a) if there is an edge b -> a, else 0; the
SimRank matrix is the fixed point of Eq. 1, S = C Q S Q^T + (1-C) I.

Readings of passages where the paper is silent, garbled or inconsistent are
marked "reading:" at the function that takes them.  Every function here is
pinned by a "not gpu" test against something other than itself (closed
forms, printed example values, brute-force solves, or an independent
formulation); none is "parity unpinned".
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

INSERT = 1
DELETE = -1


# ----------------------------------------------------------------------------
# Transition matrix and the SimRank definition
# ----------------------------------------------------------------------------

def transition_matrix(n, src, dst, weight=None, sparse=False):
    """Backward transition matrix Q of §3.1.

    Row a holds a's in-neighbours b (edges b -> a) with value 1/d_a.  With
    ``weight`` given, row a holds w_{ba} / sum_x w_{xa} (reading: the paper
    defines only the unweighted Q; the weighted form normalises each row by
    the total in-weight, which reduces to 1/d_a for unit weights).
    """
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    w = np.ones(src.size) if weight is None else np.asarray(weight, np.float64)
    A = sp.coo_matrix((w, (dst, src)), shape=(n, n)).tocsr()
    rowsum = np.asarray(A.sum(axis=1)).ravel()
    inv = np.zeros(n)
    nz = rowsum != 0
    inv[nz] = 1.0 / rowsum[nz]
    Q = sp.diags(inv) @ A
    return Q.tocsr() if sparse else Q.toarray()


def _row(Q, j):
    """Row j of a dense or SciPy-sparse matrix as a dense 1-D array."""
    if sp.issparse(Q):
        return np.asarray(Q[j, :].toarray()).ravel()
    return np.asarray(Q[j, :]).ravel()


def in_degrees(n, dst):
    """In-degree vector d (Table 1)."""
    return np.bincount(np.asarray(dst, np.int64), minlength=n).astype(np.int64)


def simrank_fixed_point(Q, C, tol=1e-15, max_iter=100000):
    """Batch SimRank: iterate Eq. 1, S <- C Q S Q^T + (1-C) I, to a fixed point.

    Stops when the max-abs change of one sweep is below ``tol``.  Works with a
    dense or SciPy-sparse Q.
    """
    n = Q.shape[0]
    S = (1.0 - C) * np.eye(n)
    for _ in range(max_iter):
        QS = Q @ S
        S_new = C * np.asarray((Q @ QS.T).T) + (1.0 - C) * np.eye(n)
        diff = np.max(np.abs(S_new - S))
        S = S_new
        if diff < tol:
            return 0.5 * (S + S.T)
    raise RuntimeError("fixed-point iteration did not converge")


def simrank_kron_solve(Q, C):
    """Eq. 1 solved exactly as one linear system (brute force, small n only).

    With row-major vectorisation vec(Q S Q^T) = (Q kron Q) vec(S), so Eq. 1
    reads (I - C Q kron Q) vec(S) = (1-C) vec(I).
    """
    Q = np.asarray(Q.toarray() if sp.issparse(Q) else Q, np.float64)
    n = Q.shape[0]
    A = np.eye(n * n) - C * np.kron(Q, Q)
    b = (1.0 - C) * np.eye(n).ravel()
    return np.linalg.solve(A, b).reshape(n, n)


def simrank_truncated_series(Q, C, K):
    """Eq. 17 truncated after k = K: S_K = (1-C) sum_{k=0}^{K} C^k Q^k (Q^T)^k."""
    Q = np.asarray(Q.toarray() if sp.issparse(Q) else Q, np.float64)
    n = Q.shape[0]
    P = np.eye(n)
    S = np.zeros((n, n))
    for k in range(K + 1):
        S += (C ** k) * (P @ P.T)
        P = Q @ P
    return (1.0 - C) * S


def partial_sim(Q, q, K, C):
    """Procedure 1 (PartialSim): column q of S in O(Kn + m) memory.

    reading: the printed loop indices are inconsistent (x_1 is never set);
    taken as x_0 = e_q, x_t = Q^T x_{t-1} for t = 1..K, then y = x_K and
    y <- x_{K-t} + C Q y for t = 1..K, returning (1-C) y, which equals
    (1-C) sum_{k=0}^{K} C^k Q^k (Q^T)^k e_q, the column of Eq. 17.
    """
    n = Q.shape[0]
    x = [np.zeros(n)]
    x[0][q] = 1.0
    QT = Q.T
    for t in range(1, K + 1):
        x.append(np.asarray(QT @ x[t - 1]).ravel())
    y = x[K].copy()
    for t in range(1, K + 1):
        y = x[K - t] + C * np.asarray(Q @ y).ravel()
    return (1.0 - C) * y


def partial_sim_block(Q, cols, K, C):
    """Procedure 1 applied to a block of columns at once (same arithmetic)."""
    n = Q.shape[0]
    X0 = np.zeros((n, len(cols)))
    X0[np.asarray(cols), np.arange(len(cols))] = 1.0
    xs = [X0]
    QT = Q.T
    for t in range(1, K + 1):
        xs.append(np.asarray(QT @ xs[t - 1]))
    Y = xs[K].copy()
    for t in range(1, K + 1):
        Y = xs[K - t] + C * np.asarray(Q @ Y)
    return (1.0 - C) * Y


# ----------------------------------------------------------------------------
# Rank-one change of Q (Thm 1, Thm 9, Table 2) and Thm 2's w
# ----------------------------------------------------------------------------

def rank_one_factors(Q, d, j, sources, op):
    """u, v with Q_new = Q + u v^T for a sink block {(i, j) : i in sources}.

    Thm 1 (insert one edge), Thm 9 (delete one edge) and the C0 rows of
    Table 2 (delta edges into one sink j).  ``d`` is the old in-degree of j.
    reading: Table 2's deletion conditions "d_j = 1 / d_j > 1" are taken as
    "d_j = delta / d_j > delta" for a block of delta deletions, and e_I is the
    indicator of the source set I.
    """
    n = Q.shape[0]
    delta = len(sources)
    eI = np.zeros(n)
    for i in sources:
        eI[i] += 1.0
    ej = np.zeros(n)
    ej[j] = 1.0
    qj = _row(Q, j)
    if op == INSERT:
        if d == 0:
            return ej.copy(), eI / delta
        return (delta / (d + delta)) * ej, eI / delta - qj
    if d == delta:
        return ej.copy(), -eI / delta
    return (delta / (d - delta)) * ej, qj - eI / delta


def thm2_w(Q, S, u, v):
    """Thm 2, Eq. 20: w = y + (lambda/2) u with z = S v, y = Q z, lambda = v^T z."""
    z = S @ v
    y = Q @ z
    lam = float(v @ z)
    return np.asarray(y).ravel() + 0.5 * lam * u


def gamma_sink_block(w, S_col_j, S_II, S_jj, d, delta, op, C, j):
    """The auxiliary vector gamma of Thm 3 (insert), Thm 9 (delete) and Table 2.

    Inputs are taken as the paper names them: w = (1/delta) Q S_{*,I} (the
    old Q, Alg 1 line "memoize w"), S_col_j = S_{*,j}, S_II = sum over
    i, i' in I of S_{i,i'}, S_jj, the old in-degree d of the sink j and the
    block size delta.  Returns (gamma, lambda); lambda follows Eq. 29b in
    its Table 2 form (1/delta^2) S_II + S_jj/C - 2 w_j - 1/C + 1.
    """
    n = w.size
    ej = np.zeros(n)
    ej[j] = 1.0
    lam = S_II / delta ** 2 + S_jj / C - 2.0 * w[j] - 1.0 / C + 1.0
    if op == INSERT:
        if d == 0:
            return w + S_II / (2.0 * delta ** 2) * ej, lam
        r = delta / (d + delta)
        g = r * (w - S_col_j / C + (lam * delta / (2.0 * (d + delta)) + 1.0 / C - 1.0) * ej)
        return g, lam
    if d == delta:
        return -w + S_II / (2.0 * delta ** 2) * ej, lam
    r = delta / (d - delta)
    g = r * (S_col_j / C - w + (lam * delta / (2.0 * (d - delta)) - 1.0 / C + 1.0) * ej)
    return g, lam


# ----------------------------------------------------------------------------
# Inc-uSR (Alg 1) for a unit update or a sink block, on existing nodes
# ----------------------------------------------------------------------------

def inc_usr(n, src, dst, S, j, sources, op, C, K, return_terms=False):
    """Alg 1 (Inc-uSR), generalised to a sink block by Table 2's C0 rows.

    Steps in the paper's order: build Q and d_j of the old graph; memoize
    w = (1/delta) Q S_{*,I}; lambda; u, v and gamma by the d_j branch;
    xi_0 = C e_j, eta_0 = gamma, M_0 = C e_j gamma^T; for k < K:
    xi_{k+1} = C Q xi_k + C (v^T xi_k) u, eta_{k+1} = Q eta_k + (v^T eta_k) u,
    M_{k+1} = xi_{k+1} eta_{k+1}^T + M_k; return S + M_K + M_K^T.
    ``src``/``dst`` describe the OLD graph.
    """
    Q = transition_matrix(n, src, dst)
    d = int(in_degrees(n, dst)[j])
    delta = len(sources)
    S_col_I = np.zeros(n)
    S_II = 0.0
    for i in sources:
        S_col_I += S[:, i]
        for i2 in sources:
            S_II += S[i, i2]
    w = (Q @ S_col_I) / delta
    u, v = rank_one_factors(Q, d, j, sources, op)
    gamma, _ = gamma_sink_block(w, S[:, j], S_II, S[j, j], d, delta, op, C, j)
    xi = np.zeros(n)
    xi[j] = C
    eta = gamma.copy()
    M = np.outer(xi, eta)
    terms = [(xi.copy(), eta.copy())]
    for _ in range(K):
        xi_next = C * (Q @ xi) + C * float(v @ xi) * u
        eta_next = Q @ eta + float(v @ eta) * u
        xi, eta = xi_next, eta_next
        M = np.outer(xi, eta) + M
        terms.append((xi.copy(), eta.copy()))
    S_new = S + M + M.T
    if return_terms:
        return S_new, M, terms
    return S_new


def sylvester_conventional(Q_new, u, w, C, K):
    """M_K by the "conventional way" of §4.1: M_0 = C u w^T,
    M_{k+1} = M_0 + C Q_new M_k Q_new^T (dense matrix-matrix products)."""
    M0 = C * np.outer(u, w)
    M = M0.copy()
    for _ in range(K):
        M = M0 + C * (Q_new @ M @ Q_new.T)
    return M


def affected_sets(n, src_old, dst_old, S, i, j, op, K, terms):
    """Thm 4: the sets A_k x B_k outside which M_k is zero.

    F1 = out-neighbours (old graph) of {y : S_{i,y} != 0}; F2 = {y : S_{j,y} != 0}
    unless d_j = 0 (insert) / d_j = 1 (delete), where it is empty;
    A_0 x B_0 = {j} x (F1 u F2 u {j}); A_k x B_k = out-neighbours (new graph)
    of the row / column support of M_{k-1}.  ``terms`` are the (xi_k, eta_k)
    of :func:`inc_usr`, used only to form the supports of M_{k-1}.
    Returns a list of (A_k, B_k) as boolean masks.
    """
    src_old = np.asarray(src_old)
    dst_old = np.asarray(dst_old)
    d = int(in_degrees(n, dst_old)[j])
    out_old = [[] for _ in range(n)]
    for a, b in zip(src_old.tolist(), dst_old.tolist()):
        out_old[a].append(b)
    if op == INSERT:
        pairs = set(zip(src_old.tolist(), dst_old.tolist())) | {(i, j)}
    else:
        pairs = set(zip(src_old.tolist(), dst_old.tolist())) - {(i, j)}
    out_new = [[] for _ in range(n)]
    for a, b in pairs:
        out_new[a].append(b)
    F1 = np.zeros(n, bool)
    for y in np.nonzero(S[i, :])[0]:
        F1[out_old[y]] = True
    F2 = np.zeros(n, bool)
    empty_branch = (d == 0) if op == INSERT else (d == 1)
    if not empty_branch:
        F2 = S[j, :] != 0
    A0 = np.zeros(n, bool)
    A0[j] = True
    B0 = F1 | F2
    B0[j] = True
    sets = [(A0, B0)]
    M = np.zeros((n, n))
    for k in range(1, K + 1):
        xi, eta = terms[k - 1]
        M = M + np.outer(xi, eta)
        rows = np.nonzero(np.any(M != 0, axis=1))[0]
        cols = np.nonzero(np.any(M != 0, axis=0))[0]
        A = np.zeros(n, bool)
        B = np.zeros(n, bool)
        for x in rows:
            A[out_new[x]] = True
        for y in cols:
            B[out_new[y]] = True
        sets.append((A, B))
    return sets


# ----------------------------------------------------------------------------
# New-node cases (§6: Alg 3, Alg 4, Alg 5) on the bordered matrices
# ----------------------------------------------------------------------------

def inc_c1(n, src, dst, S, i, C):
    """Alg 3 / Thm 8: edge (i, j) with i in V, j new (index n).

    y = C Q S_{*,i}; S_new = [[S, y], [y^T, C S_ii + 1 - C]].
    """
    Q = transition_matrix(n, src, dst)
    y = C * (Q @ S[:, i])
    S_new = np.zeros((n + 1, n + 1))
    S_new[:n, :n] = S
    S_new[:n, n] = y
    S_new[n, :n] = y
    S_new[n, n] = C * S[i, i] + 1.0 - C
    return S_new


def inc_c2(n, src, dst, S, j, C, K):
    """Alg 4 / Thm 6-7: edge (i, j) with i new (index n), j in V.

    z from Eq. 60; xi_0 = e_j, eta_0 = z; xi_{k+1} = C Q xi_k - C/(d_j+1) (Q_{j,*} xi_k) e_j,
    eta_{k+1} = Q eta_k - 1/(d_j+1) (Q_{j,*} eta_k) e_j; M_{k+1} = xi eta^T + M_k;
    Delta S11 = C/(d_j+1) (M_K + M_K^T); S_new = diag(S + Delta S11, 1 - C).
    """
    Q = transition_matrix(n, src, dst)
    d = int(in_degrees(n, dst)[j])
    ej = np.zeros(n)
    ej[j] = 1.0
    z = ((S[j, j] - (1.0 - C) ** 2) / (2.0 * C * (d + 1)) + (1.0 - C) / C) * ej - S[:, j] / C
    qj = Q[j, :]
    xi = ej.copy()
    eta = z.copy()
    M = np.outer(xi, eta)
    for _ in range(K):
        xi_next = C * (Q @ xi) - C / (d + 1) * float(qj @ xi) * ej
        eta_next = Q @ eta - 1.0 / (d + 1) * float(qj @ eta) * ej
        xi, eta = xi_next, eta_next
        M = np.outer(xi, eta) + M
    dS = C / (d + 1) * (M + M.T)
    S_new = np.zeros((n + 1, n + 1))
    S_new[:n, :n] = S + dS
    S_new[n, n] = 1.0 - C
    return S_new


def inc_c3(S, C):
    """Alg 5: edge (i, j) with both ends new (indices n, n+1).

    S_new = diag(S, [[1 - C, 0], [0, 1 - C^2]]).
    """
    n = S.shape[0]
    S_new = np.zeros((n + 2, n + 2))
    S_new[:n, :n] = S
    S_new[n, n] = 1.0 - C
    S_new[n + 1, n + 1] = 1.0 - C * C
    return S_new


# ----------------------------------------------------------------------------
# Batch updates (§8): net update, similar-sink partition, Table 2, Alg 6
# ----------------------------------------------------------------------------

def net_update(updates):
    """§8: cancel redundant updates by counting each edge, +1 per insertion and
    -1 per deletion; edges with non-zero counts form Delta G_net.

    Returns (net_plus, net_minus) as lists of (i, j) in first-appearance order.
    reading: a net count outside {-1, 0, +1} is an invalid batch (ValueError).
    """
    count = {}
    order = []
    for i, j, op in updates:
        key = (int(i), int(j))
        if key not in count:
            count[key] = 0
            order.append(key)
        count[key] += 1 if op > 0 else -1
    plus, minus = [], []
    for key in order:
        c = count[key]
        if c == 1:
            plus.append(key)
        elif c == -1:
            minus.append(key)
        elif c != 0:
            raise ValueError(f"net count {c} for edge {key}")
    return plus, minus


def partition_similar_sink(net_plus, net_minus, is_old):
    """§8: group edges by their end node ("similar sink edges"), then split each
    insertion block by whether the source is in the old V.

    ``is_old(x)`` says whether node x is in the old V.
    reading (canonical order): deletion blocks by ascending sink, then
    insertion sub-blocks by ascending sink with the old-source sub-block
    before the new-source sub-block; sources keep ascending order.  Returns
    (deletion_blocks, insertion_blocks), each a list of (sink, [sources]).
    The case C0..C3 of a sub-block is decided when it is applied (see
    :func:`block_case`), because an earlier sub-block of the same batch may
    already have created its sink or sources.
    """
    def blocks(edges):
        by_sink = {}
        for i, j in edges:
            by_sink.setdefault(j, []).append(i)
        return by_sink

    dels = [(j, sorted(srcs)) for j, srcs in sorted(blocks(net_minus).items())]
    ins = []
    for j, srcs in sorted(blocks(net_plus).items()):
        old_src = sorted(s for s in srcs if is_old(s))
        new_src = sorted(s for s in srcs if not is_old(s))
        if old_src:
            ins.append((j, old_src))
        if new_src:
            ins.append((j, new_src))
    return dels, ins


def block_case(sources, j, exists):
    """Split a sub-block by the current node set and label each part with its
    case of §8: C0 (i in V, j in V), C1 (i in V, j new), C2 (i new, j in V),
    C3 (i new, j new).  Parts with existing sources come first."""
    have = [i for i in sources if exists(i)]
    new = [i for i in sources if not exists(i)]
    parts = []
    j_in = exists(j)
    if have:
        parts.append((0 if j_in else 1, have))
        j_in = True
    if new:
        parts.append((2 if j_in else 3, new))
    return parts


class BorderedState:
    """Graph + S of the literal §6/§8 algorithms, where S grows as new nodes
    appear.  ``pos`` maps a caller node id to its row in S (new nodes are
    appended in the order in which blocks introduce them)."""

    def __init__(self, n, src, dst, S):
        self.n = n
        self.edges = set(zip(np.asarray(src).tolist(), np.asarray(dst).tolist()))
        self.S = S.copy()
        self.pos = {x: x for x in range(n)}

    def local_edges(self):
        src = np.array([self.pos[a] for a, _ in self.edges], np.int64)
        dst = np.array([self.pos[b] for _, b in self.edges], np.int64)
        return src, dst

    def add_node(self, x):
        self.pos[x] = len(self.pos)


def table2_block(state, case, j, sources, op, C, K):
    """Apply one block of Table 2 to ``state`` (a :class:`BorderedState`).

    C0 insert/delete: Alg 1 with Table 2's u, v, gamma (:func:`inc_usr`).
    C1 (sources old, j new): S_new = [[S, y], [y^T, C/delta^2 S_II + 1 - C]],
        y = C/delta Q S_{*,I}.
    C2 (sources new, j old): Q_hat = Q - delta/(d_j+delta) e_j Q_{j,*};
        M = sum_k C^k Q_hat^k e_j z^T Q_hat^kT with Table 2's z;
        S_new = diag(S + C delta/(d_j+delta) (M + M^T), (1-C) I_delta).
    C3 (all new): S_new = diag(S, (1-C) I_delta, (1-C)(1 + C/delta)).
    """
    n = state.S.shape[0]
    S = state.S
    delta = len(sources)
    src, dst = state.local_edges()
    if case == 0:
        lj = state.pos[j]
        lI = [state.pos[i] for i in sources]
        state.S = inc_usr(n, src, dst, S, lj, lI, op, C, K)
    elif case == 1:
        Q = transition_matrix(n, src, dst)
        lI = [state.pos[i] for i in sources]
        col = np.zeros(n)
        S_II = 0.0
        for a in lI:
            col += S[:, a]
            for b in lI:
                S_II += S[a, b]
        y = (C / delta) * (Q @ col)
        S_new = np.zeros((n + 1, n + 1))
        S_new[:n, :n] = S
        S_new[:n, n] = y
        S_new[n, :n] = y
        S_new[n, n] = C / delta ** 2 * S_II + 1.0 - C
        state.S = S_new
        state.add_node(j)
    elif case == 2:
        Q = transition_matrix(n, src, dst)
        lj = state.pos[j]
        d = int(in_degrees(n, dst)[lj])
        ej = np.zeros(n)
        ej[lj] = 1.0
        z = ((delta * S[lj, lj] - (delta - C) * (1.0 - C)) / (2.0 * C * (d + delta))
             + (1.0 - C) / C) * ej - S[:, lj] / C
        Q_hat = Q - (delta / (d + delta)) * np.outer(ej, Q[lj, :])
        xi = ej.copy()
        eta = z.copy()
        M = np.outer(xi, eta)
        for _ in range(K):
            xi = C * (Q_hat @ xi)
            eta = Q_hat @ eta
            M = np.outer(xi, eta) + M
        S_new = np.zeros((n + delta, n + delta))
        S_new[:n, :n] = S + (C * delta / (d + delta)) * (M + M.T)
        for t in range(delta):
            S_new[n + t, n + t] = 1.0 - C
        state.S = S_new
        for i in sources:
            state.add_node(i)
    else:
        S_new = np.zeros((n + delta + 1, n + delta + 1))
        S_new[:n, :n] = S
        for t in range(delta):
            S_new[n + t, n + t] = 1.0 - C
        S_new[n + delta, n + delta] = (1.0 - C) * (1.0 + C / delta)
        state.S = S_new
        for i in sources:
            state.add_node(i)
        state.add_node(j)
    for i in sources:
        if op == INSERT:
            state.edges.add((i, j))
        else:
            state.edges.discard((i, j))


def inc_bsr(n, src, dst, S, updates, C, K):
    """Alg 6 (Inc-bSR) with the literal Table 2 block formulas.

    Net update by hashing, split by sign, similar-sink partition, all deletion
    blocks, then all insertion sub-blocks, each applied to the S and graph
    left by the previous block.
    reading: "remove all singleton nodes" keeps isolated nodes in place (their
    S row (1-C) e_x stays a valid fixed point), so node ids never shift.
    Returns S indexed by caller ids 0..n_final-1.
    """
    plus, minus = net_update(updates)
    dels, ins = partition_similar_sink(plus, minus, lambda x: x < n)
    state = BorderedState(n, src, dst, S)
    for j, srcs in dels:
        table2_block(state, 0, j, srcs, DELETE, C, K)
    for j, srcs in ins:
        for case, part in block_case(srcs, j, lambda x: x in state.pos):
            table2_block(state, case, j, part, INSERT, C, K)
    n_final = len(state.pos)
    perm = np.empty(n_final, np.int64)
    for x, p in state.pos.items():
        perm[x] = p
    return state.S[np.ix_(perm, perm)], sorted(state.edges)


def inc_bsr_isolated(n, n_final, src, dst, S, updates, C, K):
    """Alg 6 with every new node pre-allocated as an isolated node
    (S_xx = 1 - C) so that each block is a C0 block of Table 2.

    This is the reduction the CUDA path uses; it agrees with :func:`inc_bsr`
    term by term at any K (tested).
    """
    plus, minus = net_update(updates)
    dels, ins = partition_similar_sink(plus, minus, lambda x: x < n)
    Sx = np.zeros((n_final, n_final))
    Sx[:n, :n] = S
    for x in range(n, n_final):
        Sx[x, x] = 1.0 - C
    edges = set(zip(np.asarray(src).tolist(), np.asarray(dst).tolist()))
    exists = set(range(n))
    order = [(DELETE, j, srcs) for j, srcs in dels]
    for j, srcs in ins:
        for _, part in block_case(srcs, j, lambda x: x in exists):
            order.append((INSERT, j, part))
            exists.update(part)
            exists.add(j)
    for op, j, srcs in order:
        s_arr = np.array([a for a, _ in edges], np.int64)
        d_arr = np.array([b for _, b in edges], np.int64)
        Sx = inc_usr(n_final, s_arr, d_arr, Sx, j, srcs, op, C, K)
        for i in srcs:
            if op == INSERT:
                edges.add((i, j))
            else:
                edges.discard((i, j))
    return Sx, sorted(edges)


def sequential_unit_updates(n_final, src, dst, S, updates, C, K):
    """Unit updates applied one at a time in the given order (Alg 1 per edge,
    new nodes pre-allocated as isolated nodes)."""
    edges = set(zip(np.asarray(src).tolist(), np.asarray(dst).tolist()))
    for i, j, op in updates:
        s_arr = np.array([a for a, _ in edges], np.int64)
        d_arr = np.array([b for _, b in edges], np.int64)
        S = inc_usr(n_final, s_arr, d_arr, S, int(j), [int(i)], int(op), C, K)
        if op > 0:
            edges.add((int(i), int(j)))
        else:
            edges.discard((int(i), int(j)))
    return S, sorted(edges)


def alg1_stream_columns(n, src, dst, S0_block, updates, C, K, query):
    """Alg 1 applied to each update of a stream in order, returning only the
    columns ``query`` of the final S (for graphs whose dense S is too large).

    Every update is Alg 1 exactly as in :func:`inc_usr` (w from the old Q and
    the old column(s) of the sources, lambda and gamma by the d_j branch,
    xi_{k+1} = C Q xi_k + C (v^T xi_k) u, eta_{k+1} = Q eta_k + (v^T eta_k) u);
    only the storage of S differs: S_t = S_0 + sum_{u <= t} (M_u + M_u^T) is
    kept as S_0 plus the factors of each M_u = sum_k xi_k eta_k^T, and a
    column of the current S is read as S_0[:, x] + sum_u (Xi_u H_u[x, :]^T
    + H_u Xi_u[x, :]^T).  ``S0_block(cols)`` returns the columns ``cols`` of
    S_0 (n x len(cols)).  Updates are unit updates between existing nodes.
    """
    edges = set(zip(np.asarray(src).tolist(), np.asarray(dst).tolist()))
    need = sorted({int(x) for u in updates for x in u[:2]} | {int(x) for x in query})
    base = S0_block(need)
    pos = {x: c for c, x in enumerate(need)}
    Xi, H = [], []  # per update: n x (K+1) factor matrices

    def column(x):
        col = np.array(base[:, pos[x]], np.float64)
        for A, B in zip(Xi, H):
            col += A @ B[x, :] + B @ A[x, :]
        return col

    for i, j, op in updates:
        i, j, op = int(i), int(j), int(op)
        if i >= n or j >= n:
            raise ValueError("alg1_stream_columns handles existing nodes only")
        s_arr = np.array([a for a, _ in edges], np.int64)
        d_arr = np.array([b for _, b in edges], np.int64)
        Q = transition_matrix(n, s_arr, d_arr, sparse=True)
        d = int(in_degrees(n, d_arr)[j])
        Si, Sj = column(i), column(j)
        w = np.asarray(Q @ Si).ravel()
        u, v = rank_one_factors(Q, d, j, [i], op)
        gamma, _ = gamma_sink_block(w, Sj, Si[i], Sj[j], d, 1, op, C, j)
        A = np.zeros((n, K + 1))
        B = np.zeros((n, K + 1))
        xi = np.zeros(n)
        xi[j] = C
        eta = gamma.copy()
        A[:, 0], B[:, 0] = xi, eta
        for k in range(K):
            xi_next = C * np.asarray(Q @ xi).ravel() + C * float(v @ xi) * u
            eta_next = np.asarray(Q @ eta).ravel() + float(v @ eta) * u
            xi, eta = xi_next, eta_next
            A[:, k + 1], B[:, k + 1] = xi, eta
        Xi.append(A)
        H.append(B)
        if op > 0:
            edges.add((i, j))
        else:
            edges.discard((i, j))
    return np.stack([column(int(x)) for x in query], axis=1)


# ----------------------------------------------------------------------------
# One-shot batch form (rank-2r Sylvester): the definition written out
# ----------------------------------------------------------------------------

def one_shot_batch(n_final, src_old, dst_old, src_new, dst_new, S, C, K):
    """Whole-batch update at truncation K, from the recursion of Eq. 23-25.

    Subtracting Eq. 1 for the old graph from Eq. 1 for the new graph gives
    Delta S = C Q_new Delta S Q_new^T + C T with T = Q_new S Q_new^T - Q S Q^T
    (Eq. 23 with Eq. 25); its series truncated after k = K is
    Delta S_K = sum_{k=0}^{K} C^{k+1} Q_new^k T Q_new^kT.  T is formed here
    directly with dense products (no use of the fixed-point identity Eq. 33).
    ``S`` is the old S padded with isolated new nodes (S_xx = 1 - C).
    """
    Q = transition_matrix(n_final, src_old, dst_old)
    Qn = transition_matrix(n_final, src_new, dst_new)
    T = Qn @ S @ Qn.T - Q @ S @ Q.T
    X = C * T
    dS = X.copy()
    for _ in range(K):
        X = C * (Qn @ X @ Qn.T)
        dS += X
    return S + dS


# ----------------------------------------------------------------------------
# Column-wise update (Alg 7, Inc-SR-All-P)
# ----------------------------------------------------------------------------

def inc_sr_all_p(n, src, dst, S_col_x, x, updates, C, K, K_old=None):
    """Alg 7 (Inc-SR-All-P): column x of S updated through a list of unit
    updates between existing or new nodes, using O(Kn + m) memory.

    For each update the old columns S_{*,i}, S_{*,j} come from PartialSim
    (Procedure 1) on the current graph; the case C0..C3 is chosen by whether
    i, j are nodes yet; only the x-th entries of xi_k, eta_k feed the column
    accumulators m, n.
    reading: Alg 7's "d_j <- 0" after cases C1 and C3 is taken as d_j <- 1
    (j gains the in-neighbour i); deletions of existing edges are handled
    like C0 with Thm 9's u, v, gamma (the algorithm prints only insertions).
    New nodes take the next free id, as the caller names them.
    ``K_old`` (default K, as in Alg 7) is the truncation of PartialSim for
    the old columns; a large K_old gives the converged old columns.
    """
    K_old = K if K_old is None else K_old
    edges = set(zip(np.asarray(src).tolist(), np.asarray(dst).tolist()))
    n_cur = n
    col = np.array(S_col_x, np.float64).copy()

    def arrays():
        return (np.array([a for a, _ in edges], np.int64),
                np.array([b for _, b in edges], np.int64))

    for i, j, op in updates:
        i, j, op = int(i), int(j), int(op)
        s_arr, d_arr = arrays()
        Q = transition_matrix(n_cur, s_arr, d_arr, sparse=True)
        i_in, j_in = i < n_cur, j < n_cur
        if i_in and j_in and x >= n_cur:
            pass  # column x is not a node yet: nothing to update
        elif i_in and j_in:
            Si = partial_sim(Q, i, K_old, C)
            Sj = partial_sim(Q, j, K_old, C)
            d = int(in_degrees(n_cur, d_arr)[j])
            w = Q @ Si
            u, v = rank_one_factors(Q, d, j, [i], op)
            gamma, _ = gamma_sink_block(w, Sj, Si[i], Sj[j], d, 1, op, C, j)
            xi = np.zeros(n_cur)
            xi[j] = C
            eta = gamma.copy()
            m_acc = eta[x] * xi
            n_acc = xi[x] * eta
            for _ in range(K):
                xi = C * (Q @ xi) + C * float(v @ xi) * u
                eta = Q @ eta + float(v @ eta) * u
                m_acc = eta[x] * xi + m_acc
                n_acc = xi[x] * eta + n_acc
            col = col + m_acc + n_acc
        elif i_in and not j_in:  # C1
            Si = partial_sim(Q, i, K_old, C)
            y = C * (Q @ Si)
            if x == j:
                col = np.concatenate([y, [C * Si[i] + 1.0 - C]])
            elif x >= n_cur:
                col = np.concatenate([col, [0.0]])
            else:
                col = np.concatenate([col, [y[x]]])
            n_cur += 1
        elif not i_in and j_in:  # C2
            if x == i:
                col = np.concatenate([np.zeros(n_cur), [1.0 - C]])
            elif x >= n_cur:
                col = np.concatenate([col, [0.0]])
            else:
                Sj = partial_sim(Q, j, K_old, C)
                d = int(in_degrees(n_cur, d_arr)[j])
                ej = np.zeros(n_cur)
                ej[j] = 1.0
                z = ((Sj[j] - (1.0 - C) ** 2) / (2.0 * C * (d + 1)) + (1.0 - C) / C) * ej - Sj / C
                qj = _row(Q, j)
                xi = ej.copy()
                eta = z.copy()
                m_acc = z[x] * ej
                n_acc = ej[x] * z
                for _ in range(K):
                    xi = C * (Q @ xi) - C / (d + 1) * float(qj @ xi) * ej
                    eta = Q @ eta - 1.0 / (d + 1) * float(qj @ eta) * ej
                    m_acc = eta[x] * xi + m_acc
                    n_acc = xi[x] * eta + n_acc
                col = np.concatenate([col + C / (d + 1) * (m_acc + n_acc), [0.0]])
            n_cur += 1
        else:  # C3
            if x == i:
                col = np.concatenate([np.zeros(n_cur), [1.0 - C, 0.0]])
            elif x == j:
                col = np.concatenate([np.zeros(n_cur), [0.0, 1.0 - C * C]])
            else:
                col = np.concatenate([col, [0.0, 0.0]])
            n_cur += 2
        if op > 0:
            edges.add((i, j))
        else:
            edges.discard((i, j))
    return col


def inc_sr_all_p_blocks(n, n_final, src, dst, S_col_x, x, updates, C, K, K_old=None):
    """Alg 7 combined with the batch scheme of §8 (the closing remark of §7):
    column x of S through a batch of updates applied as similar-sink blocks.

    Net update and partition as in Alg 6 (:func:`net_update`,
    :func:`partition_similar_sink`, :func:`block_case`); new nodes are
    pre-allocated as isolated nodes (ids n .. n_final - 1, S column (1-C) e_x),
    so every block is a C0 block of Table 2.  For each block (delta sources I
    into sink j) the old columns S_{*,i} (i in I) and S_{*,j} come from
    PartialSim (Procedure 1) at K_old on the current graph, which needs the
    delta + 1 columns only; w = (1/delta) Q sum_i S_{*,i}, S_II, u, v and gamma
    follow Table 2, and only the x-th entries of xi_k, eta_k feed the column
    accumulators.  ``S_col_x`` is column x of the old S on the n old nodes.
    ``K_old`` defaults to K (Alg 7 as printed).
    """
    K_old = K if K_old is None else K_old
    plus, minus = net_update(updates)
    dels, ins = partition_similar_sink(plus, minus, lambda y: y < n)
    order = [(DELETE, j, srcs) for j, srcs in dels]
    exists = set(range(n))
    for j, srcs in ins:
        for _, part in block_case(srcs, j, lambda y: y in exists):
            order.append((INSERT, j, part))
            exists.update(part)
            exists.add(j)
    col = np.zeros(n_final)
    if x < n:
        col[:n] = np.asarray(S_col_x, np.float64)
    else:
        col[x] = 1.0 - C
    edges = set(zip(np.asarray(src).tolist(), np.asarray(dst).tolist()))
    for op, j, srcs in order:
        s_arr = np.array([a for a, _ in edges], np.int64)
        d_arr = np.array([b for _, b in edges], np.int64)
        Q = transition_matrix(n_final, s_arr, d_arr, sparse=True)
        d = int(in_degrees(n_final, d_arr)[j])
        delta = len(srcs)
        S_cols_I = [partial_sim(Q, i, K_old, C) for i in srcs]
        sI = np.sum(S_cols_I, axis=0)
        Sj = partial_sim(Q, j, K_old, C)
        S_II = float(sum(sI[i] for i in srcs))
        w = np.asarray(Q @ sI).ravel() / delta
        u, v = rank_one_factors(Q, d, j, srcs, op)
        gamma, _ = gamma_sink_block(w, Sj, S_II, Sj[j], d, delta, op, C, j)
        xi = np.zeros(n_final)
        xi[j] = C
        eta = gamma.copy()
        m_acc = eta[x] * xi
        n_acc = xi[x] * eta
        for _ in range(K):
            xi = C * np.asarray(Q @ xi).ravel() + C * float(v @ xi) * u
            eta = np.asarray(Q @ eta).ravel() + float(v @ eta) * u
            m_acc = eta[x] * xi + m_acc
            n_acc = xi[x] * eta + n_acc
        col = col + m_acc + n_acc
        for i in srcs:
            if op > 0:
                edges.add((i, j))
            else:
                edges.discard((i, j))
    return col


# ----------------------------------------------------------------------------
# Gradient of a pair loss with respect to edge weights
# ----------------------------------------------------------------------------

def pair_loss_and_weight_grad(n, src, dst, weight, a, b, target, C, K):
    """Loss L = sum_p (S_K[a_p, b_p] - t_p)^2 and dL/d(edge weight).

    S_K is the truncated series of Eq. 17, S_K = (1-C) sum_{k<=K} C^k Q^k Q^kT,
    with the weighted Q of :func:`transition_matrix` (reading: the paper
    defines neither weights nor gradients; this is the derivative of the same
    K-truncated forward).  The derivative is taken by reverse-mode automatic
    differentiation of these dense float64 CPU operations.
    """
    import torch

    src_t = torch.as_tensor(np.asarray(src, np.int64))
    dst_t = torch.as_tensor(np.asarray(dst, np.int64))
    w = torch.tensor(np.asarray(weight, np.float64), requires_grad=True)
    A = torch.zeros((n, n), dtype=torch.float64).index_put((dst_t, src_t), w, accumulate=True)
    rs = A.sum(dim=1, keepdim=True)
    Q = torch.where(rs > 0, A / torch.where(rs > 0, rs, torch.ones_like(rs)), torch.zeros_like(A))
    P = torch.eye(n, dtype=torch.float64)
    S = torch.zeros((n, n), dtype=torch.float64)
    for k in range(K + 1):
        S = S + (C ** k) * (P @ P.T)
        P = Q @ P
    S = (1.0 - C) * S
    s = S[torch.as_tensor(np.asarray(a, np.int64)), torch.as_tensor(np.asarray(b, np.int64))]
    L = ((s - torch.as_tensor(np.asarray(target, np.float64))) ** 2).sum()
    L.backward()
    return float(L.detach()), w.grad.detach().numpy().copy(), S.detach().numpy()


def pair_loss(n, src, dst, weight, a, b, target, C, K):
    """The same loss as :func:`pair_loss_and_weight_grad`, forward only (for
    finite differences)."""
    Q = transition_matrix(n, src, dst, weight)
    S = simrank_truncated_series(Q, C, K)
    s = S[np.asarray(a), np.asarray(b)]
    return float(np.sum((s - np.asarray(target)) ** 2))
