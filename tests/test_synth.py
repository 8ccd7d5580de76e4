"""The seeded input generators produce valid update sequences: every
insertion adds an absent edge and every deletion removes a present one, in
the order the updates are returned (a batch is shuffled, so a deletion must
never target an edge the same batch inserts)."""
import numpy as np
import pytest

from synth import EdgeSet, batch_with_new_nodes, chung_lu_digraph, update_stream


def _replay(n_edges_src, n_edges_dst, ups):
    live = set(zip(np.asarray(n_edges_src).tolist(), np.asarray(n_edges_dst).tolist()))
    for i, j, op in np.asarray(ups).tolist():
        assert i != j
        if op > 0:
            assert (i, j) not in live, (i, j)
            live.add((i, j))
        else:
            assert (i, j) in live, (i, j)
            live.discard((i, j))
    return live


@pytest.mark.parametrize("b", [64, 1024])
def test_batches_replay_in_their_shuffled_order(b):
    n, m = 3000, 24000
    s, d = chung_lu_digraph(n, m, 2.2, 2.2, 5)
    es = EdgeSet(n, s, d)
    live = set(zip(s.tolist(), d.tolist()))
    for t in range(4):
        ups, n_new = batch_with_new_nodes(n, s, d, b, 100 + t, edge_set=es)
        assert len(ups) == b and n_new > 0
        src = [a for a, _ in live]
        dst = [c for _, c in live]
        live = _replay(src, dst, ups)
    assert live == set(es.edges)


def test_update_stream_replays():
    n, m = 2000, 16000
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 6)
    ups = update_stream(n, s, d, 500, 7)
    _replay(s, d, ups)
