"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the bench.

This package builds graphs, vertex partitions and query pairs.  It holds none of the
distance-query method's arithmetic (no shortest-path computation of any kind): the
graphs are plain undirected edge lists turned into symmetric CSR arrays, the partitions
are geometric or index-based splits, and the queries are uniform random vertex pairs.

Workloads (stand-ins for the paper's unnamed 256k-vertex planar test graph, Sec. 5):
  grid4        W x H 4-neighbour grid, integer weights uniform in [1, wmax]
  grid_holes   4-neighbour grid with a fraction of the vertices removed at random
  grid_diag    4-neighbour grid plus one random diagonal per cell (still planar)
  delaunay     Delaunay triangulation of uniform points in the unit square
"""

from .graphs import (  # noqa: F401
    Graph,
    csr_from_edges,
    grid4,
    grid_holes,
    grid_diag,
    delaunay,
    edges_from_csr,
)
from .partition import grid_blocks, rcb, kdtree  # noqa: F401
from .queries import random_pairs  # noqa: F401
from .configs import workload, WORKLOADS  # noqa: F401
