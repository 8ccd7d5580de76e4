"""Seeded graph and update-stream generators.

All generators return plain int32 / float arrays.  An edge (i, j) means i -> j.
The shapes follow the paper's workloads (§9: power-law in/out degrees, mean
degree 5-24, streams of 80% insertions and 20% deletions); the real datasets
are not available, so these draws stand in for them.
"""
from __future__ import annotations

import numpy as np

UPDATE_INSERT = 1
UPDATE_DELETE = -1


def _key(src, dst, n_key):
    return np.asarray(src, np.int64) * np.int64(n_key) + np.asarray(dst, np.int64)


def er_graph(n: int, m: int, seed: int):
    """Directed Erdos-Renyi G(n, m): m distinct ordered pairs u != v, uniform."""
    if m > n * (n - 1):
        raise ValueError("too many edges for a simple digraph")
    rng = np.random.default_rng(seed)
    keys = np.empty(0, np.int64)
    while keys.size < m:
        need = m - keys.size
        s = rng.integers(0, n, size=2 * need + 16)
        d = rng.integers(0, n, size=2 * need + 16)
        ok = s != d
        k = _key(s[ok], d[ok], n)
        # keep first occurrences in draw order
        keys = np.concatenate([keys, k])
        _, first = np.unique(keys, return_index=True)
        keys = keys[np.sort(first)]
    keys = keys[:m]
    return (keys // n).astype(np.int32), (keys % n).astype(np.int32)


def _power_weights(n: int, m: int, exponent: float, rng):
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (exponent - 1.0))
    w *= m / w.sum()
    return w[rng.permutation(n)]


def chung_lu_digraph(n: int, m: int, gamma_in: float, gamma_out: float, seed: int):
    """Directed Chung-Lu graph with power-law in/out weights.

    w_i ~ (i+1)^(-1/(gamma-1)) scaled so that sum w = m; the in- and out-weight
    sequences get independent seeded permutations.  Sources are drawn
    proportional to w_out, targets proportional to w_in; self-loops and
    duplicates are rejected until m distinct edges exist.
    """
    rng = np.random.default_rng(seed)
    w_out = _power_weights(n, m, gamma_out, rng)
    w_in = _power_weights(n, m, gamma_in, rng)
    p_out = w_out / w_out.sum()
    p_in = w_in / w_in.sum()
    keys = np.empty(0, np.int64)
    rounds = 0
    while keys.size < m:
        need = m - keys.size
        draw = int(need * 1.3) + 64
        s = rng.choice(n, size=draw, p=p_out)
        d = rng.choice(n, size=draw, p=p_in)
        ok = s != d
        keys = np.concatenate([keys, _key(s[ok], d[ok], n)])
        _, first = np.unique(keys, return_index=True)
        keys = keys[np.sort(first)]
        rounds += 1
        if rounds > 200:
            raise RuntimeError("Chung-Lu rejection sampling did not converge")
    keys = keys[:m]
    return (keys // n).astype(np.int32), (keys % n).astype(np.int32)


def random_arborescence(n: int, seed: int):
    """Random rooted tree, edges parent -> child; node 0 is the root."""
    rng = np.random.default_rng(seed)
    parent = np.array([rng.integers(0, v) for v in range(1, n)], dtype=np.int32)
    child = np.arange(1, n, dtype=np.int32)
    return parent, child


def random_forest(sizes, seed: int):
    """Random rooted trees of the given sizes on consecutive ids (the first
    node of each tree is its root), edges parent -> child."""
    ps, cs = [], []
    off = 0
    for t, sz in enumerate(sizes):
        p, c = random_arborescence(int(sz), seed * 1000 + t)
        ps.append(p + off)
        cs.append(c + off)
        off += int(sz)
    return np.concatenate(ps).astype(np.int32), np.concatenate(cs).astype(np.int32)


def tree_with_extra_edges(n: int, extra: int, seed: int):
    """A random rooted tree on n nodes (edges parent -> child) and `extra`
    further edges that are neither tree edges, duplicates nor self-loops:
    source uniform, target drawn with probability proportional to
    (1 + number of extra edges it already has), so some nodes collect many
    in-neighbours.  Returns (tree_src, tree_dst, extra_src, extra_dst)."""
    ps, cs = random_arborescence(n, seed)
    rng = np.random.default_rng(seed + 7)
    have = set(zip(ps.tolist(), cs.tolist()))
    w = np.ones(n)
    es, ed = [], []
    while len(es) < extra:
        i = int(rng.integers(0, n))
        j = _Sampler(w, rng)()
        if i == j or (i, j) in have:
            continue
        have.add((i, j))
        es.append(i)
        ed.append(j)
        w[j] += 1.0
    return ps, cs, np.array(es, np.int32), np.array(ed, np.int32)


def block_graph(sizes, deg: int, cross: int, seed: int):
    """Directed Chung-Lu blocks (exponent 2.1, mean degree `deg`) on
    consecutive ids, plus `cross` edges between distinct blocks (uniform
    endpoints).  Returns (block_src, block_dst, cross_src, cross_dst)."""
    bs, bd = [], []
    off = 0
    starts = []
    for t, sz in enumerate(sizes):
        s, d = chung_lu_digraph(int(sz), deg * int(sz), 2.1, 2.1, seed * 1000 + t)
        bs.append(s + off)
        bd.append(d + off)
        starts.append(off)
        off += int(sz)
    n = off
    block_of = np.zeros(n, np.int64)
    for t, st in enumerate(starts):
        block_of[st:st + int(sizes[t])] = t
    rng = np.random.default_rng(seed + 11)
    have = set()
    xs, xd = [], []
    while len(xs) < cross:
        i, j = int(rng.integers(0, n)), int(rng.integers(0, n))
        if block_of[i] == block_of[j] or (i, j) in have:
            continue
        have.add((i, j))
        xs.append(i)
        xd.append(j)
    return (np.concatenate(bs).astype(np.int32), np.concatenate(bd).astype(np.int32),
            np.array(xs, np.int32), np.array(xd, np.int32))


def edge_weights(m: int, seed: int, low: float = 0.1, high: float = 1.0):
    """Edge weights uniform in (low, high]."""
    rng = np.random.default_rng(seed)
    u = rng.random(m)  # [0, 1)
    return (high - (high - low) * u).astype(np.float32)


class _Sampler:
    """Draws ids with probability proportional to `weights` (inverse CDF)."""

    def __init__(self, weights, rng):
        c = np.cumsum(np.asarray(weights, np.float64))
        self.cdf = c / c[-1]
        self.rng = rng

    def __call__(self):
        return int(min(np.searchsorted(self.cdf, self.rng.random(), side="right"), self.cdf.size - 1))


class EdgeSet:
    """Mutable simple digraph used to draw valid sequential updates."""

    def __init__(self, n: int, src, dst):
        self.n = int(n)
        self.edges = list(zip(np.asarray(src).tolist(), np.asarray(dst).tolist()))
        self.pos = {e: t for t, e in enumerate(self.edges)}
        self.out_deg = np.bincount(np.asarray(src, np.int64), minlength=n).astype(np.int64)
        self.in_deg = np.bincount(np.asarray(dst, np.int64), minlength=n).astype(np.int64)

    def has(self, i, j):
        return (i, j) in self.pos

    def add_node(self):
        self.n += 1
        self.out_deg = np.append(self.out_deg, 0)
        self.in_deg = np.append(self.in_deg, 0)
        return self.n - 1

    def insert(self, i, j):
        assert (i, j) not in self.pos and i != j
        self.pos[(i, j)] = len(self.edges)
        self.edges.append((i, j))
        self.out_deg[i] += 1
        self.in_deg[j] += 1

    def delete(self, i, j):
        t = self.pos.pop((i, j))
        last = self.edges.pop()
        if t < len(self.edges):
            self.edges[t] = last
            self.pos[last] = t
        self.out_deg[i] -= 1
        self.in_deg[j] -= 1


def update_stream(n: int, src, dst, count: int, seed: int, frac_insert: float = 0.8,
                  edge_set: EdgeSet | None = None):
    """Sequentially valid stream of unit updates between existing nodes.

    Insertions draw the source proportional to (out-degree + 1) and the
    target proportional to (in-degree + 1), both taken from the degrees at
    the start of the stream, and redraw while the edge exists or is a
    self-loop.  Deletions pick a uniformly random existing edge.  Returns an
    int32 array of shape (count, 3): (src, dst, op) with op = +1 / -1.
    Pass ``edge_set`` to continue a stream from an earlier one.
    """
    rng = np.random.default_rng(seed)
    g = edge_set if edge_set is not None else EdgeSet(n, src, dst)
    draw_src = _Sampler(g.out_deg[: g.n] + 1.0, rng)
    draw_dst = _Sampler(g.in_deg[: g.n] + 1.0, rng)
    out = np.empty((count, 3), np.int32)
    for t in range(count):
        if rng.random() < frac_insert or not g.edges:
            while True:
                i = draw_src()
                j = draw_dst()
                if i != j and not g.has(i, j):
                    break
            g.insert(i, j)
            out[t] = (i, j, UPDATE_INSERT)
        else:
            i, j = g.edges[int(rng.integers(0, len(g.edges)))]
            g.delete(i, j)
            out[t] = (i, j, UPDATE_DELETE)
    return out


def keyed_update_stream(n: int, src, dst, count: int, seed: int, frac_insert: float = 0.8):
    """Same distribution as :func:`update_stream`, for graphs too large for a
    Python edge set: membership tests use the sorted int64 keys src * n + dst.

    Insertions draw the source proportional to (out-degree + 1) and the
    target proportional to (in-degree + 1) of the initial graph; deletions
    pick a uniformly random edge among those present (initial edges not yet
    deleted and edges inserted earlier in the stream).  Returns an int32
    array of shape (count, 3).
    """
    rng = np.random.default_rng(seed)
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    keys = np.sort(src * n + dst)
    draw_src = _Sampler(np.bincount(src, minlength=n) + 1.0, rng)
    draw_dst = _Sampler(np.bincount(dst, minlength=n) + 1.0, rng)
    added, removed = set(), set()

    def present(k):
        if k in added:
            return True
        if k in removed:
            return False
        p = np.searchsorted(keys, k)
        return p < keys.size and keys[p] == k

    out = np.empty((count, 3), np.int32)
    for t in range(count):
        if rng.random() < frac_insert:
            while True:
                i, j = draw_src(), draw_dst()
                k = i * n + j
                if i != j and not present(k):
                    break
            added.add(k)
            removed.discard(k)
            out[t] = (i, j, UPDATE_INSERT)
        else:
            while True:
                if added and rng.random() < len(added) / (len(added) + keys.size):
                    k = sorted(added)[int(rng.integers(0, len(added)))]
                else:
                    k = int(keys[int(rng.integers(0, keys.size))])
                if present(k):
                    break
            added.discard(k)
            removed.add(k)
            out[t] = (k // n, k % n, UPDATE_DELETE)
    return out


def batch_with_new_nodes(n: int, src, dst, b: int, seed: int, frac_new: float = 0.10,
                         frac_insert: float = 0.8, reuse_target: float = 0.25,
                         edge_set: EdgeSet | None = None):
    """One batch of b edge updates of which ``frac_new`` attach new nodes.

    The new-node edges are insertions, split in equal thirds into
    source-new (i new, j old), target-new (i old, j new) and both-new.  A
    fraction ``reuse_target`` of the edges with a new target reuse a new
    target already created in this batch, so some new sinks receive several
    edges.  New node ids are n_cur, n_cur+1, ... in order of first use.  The
    remaining edges are updates between existing nodes (``frac_insert``
    insertions, the rest deletions of edges that existed before the batch),
    drawn as in :func:`update_stream`; the batch is returned in a random
    order, so a deletion never targets an edge the batch inserts.
    Returns (updates int32 (b,3), number of new nodes).
    """
    rng = np.random.default_rng(seed)
    g = edge_set if edge_set is not None else EdgeSet(n, src, dst)
    n_old = g.n
    n_new_edges = int(round(b * frac_new))
    kinds = np.array([0, 1, 2] * (n_new_edges // 3 + 1))[:n_new_edges]
    rng.shuffle(kinds)
    draw_src = _Sampler(g.out_deg[:n_old] + 1.0, rng)
    draw_dst = _Sampler(g.in_deg[:n_old] + 1.0, rng)
    ups = []
    new_targets = []
    fresh = set()  # edges this batch inserts
    for kind in kinds:
        if kind == 0:  # source new, target old
            i = g.add_node()
            j = draw_dst()
        elif kind == 1:  # source old, target new
            i = draw_src()
            if new_targets and rng.random() < reuse_target:
                j = int(new_targets[int(rng.integers(0, len(new_targets)))])
                if g.has(i, j):
                    j = g.add_node()
                    new_targets.append(j)
            else:
                j = g.add_node()
                new_targets.append(j)
        else:  # both new
            i = g.add_node()
            if new_targets and rng.random() < reuse_target:
                j = int(new_targets[int(rng.integers(0, len(new_targets)))])
            else:
                j = g.add_node()
                new_targets.append(j)
        g.insert(i, j)
        fresh.add((i, j))
        ups.append((i, j, UPDATE_INSERT))
    for _ in range(b - n_new_edges):
        if rng.random() < frac_insert or not g.edges:
            while True:
                i = draw_src()
                j = draw_dst()
                if i != j and not g.has(i, j):
                    break
            g.insert(i, j)
            fresh.add((i, j))
            ups.append((i, j, UPDATE_INSERT))
        else:
            while True:
                i, j = g.edges[int(rng.integers(0, len(g.edges)))]
                if i < n_old and j < n_old and (i, j) not in fresh:
                    break
            g.delete(i, j)
            ups.append((i, j, UPDATE_DELETE))
    order = rng.permutation(len(ups))
    out = np.array([ups[t] for t in order], np.int32).reshape(-1, 3)
    return out, g.n - n_old


def query_pairs(n: int, count: int, seed: int, t_low: float = 0.0, t_high: float = 0.3):
    """Random node pairs (a, b), a != b, with targets uniform in [t_low, t_high]."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, n, size=count)
    b = rng.integers(0, n - 1, size=count)
    b = np.where(b >= a, b + 1, b)
    t = rng.uniform(t_low, t_high, size=count)
    return a.astype(np.int32), b.astype(np.int32), t.astype(np.float64)
