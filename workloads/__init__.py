"""Seeded synthetic inputs shared by the tests, the bench and the oracle timing.

This package builds graphs and query sets only.  It holds none of the search
method's arithmetic (no relaxation, no pruning, no potential): both the CUDA
path and the CPU oracle consume what it produces, and neither side imports the
other.

The graph shapes stand in for the paper's workloads (Sec. 6, "Setup" and the
graph table): road networks and k-NN graphs are large-diameter, low-degree,
planar-ish graphs with coordinates (jittered grids with deletions and short
shortcuts here); social networks are power-law graphs (RMAT here), with
integer weights drawn uniformly at random as the paper does for graphs that
come without weights.
"""

from .graphs import CSRGraph, grid_graph, road_like_graph, rmat_graph, csr_from_undirected, one_way_graph
from .queries import (
    random_pairs,
    near_mid_far_pairs,
    star_pairs,
    clique_pairs,
    config_workload,
)

__all__ = [
    "CSRGraph",
    "grid_graph",
    "road_like_graph",
    "rmat_graph",
    "csr_from_undirected",
    "one_way_graph",
    "random_pairs",
    "near_mid_far_pairs",
    "star_pairs",
    "clique_pairs",
    "config_workload",
]
