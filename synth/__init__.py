"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package only draws random graphs, update streams and query pairs.  It
holds none of the SimRank arithmetic: no transition matrix, no similarity,
no update formula.  Both sides of every parity test take their inputs from
here and nowhere else.
"""
from .graphs import (  # noqa: F401
    er_graph,
    chung_lu_digraph,
    random_arborescence,
    random_forest,
    tree_with_extra_edges,
    block_graph,
    update_stream,
    keyed_update_stream,
    batch_with_new_nodes,
    edge_weights,
    query_pairs,
    EdgeSet,
)
