"""Named workloads with fixed seeds (seed = 1234 + workload index).

  grid64          64x64 4-neighbour grid, w ~ U{1..100}, 16 blocks of 16x16, 10,000 pairs
  delaunay1m      Delaunay of 2^20 uniform points, w = round(1e6 * length), RCB into 1,024
                  components of 1,024 vertices, 10,000,000 pairs
  batch512        512 instances: even index grid with 10% of vertices removed, odd index
                  Delaunay; n log-uniform in [1,000, 65,536]; w ~ U{1..1000}; kd-tree
                  components with a leaf cap log-uniform in [128, 2,048]; 100,000 pairs each
  delaunay256k    Delaunay of 2^18 points, f32 w = length * lognormal(0, 0.25), RCB into 256
                  components of 1,024, 1,000,000 pairs
  grid1024diag    1024x1024 grid with one random diagonal per cell, w ~ U{1..1000},
                  32x32-block components

Scaled-down variants (for parity tests at oracle-friendly sizes) take the same recipe with
smaller sizes: `delaunay(npts, levels)`, `grid(W, bw)`.
"""

from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import graphs, partition, queries


@dataclass
class Workload:
    name: str
    graph: graphs.Graph
    part: np.ndarray
    k: int
    pairs: Optional[np.ndarray]
    seed: int


def grid64(q: int = 10_000, seed: int = 1235) -> Workload:
    g = graphs.grid4(64, 64, wmax=100, seed=seed)
    part, k = partition.grid_blocks(64, 64, 16, 16)
    return Workload("grid64", g, part, k, queries.random_pairs(g.n, q, seed + 1), seed)


def grid_blocks_workload(W: int, H: int, bw: int, bh: int, wmax: int, q: int, seed: int) -> Workload:
    g = graphs.grid4(W, H, wmax=wmax, seed=seed)
    part, k = partition.grid_blocks(W, H, bw, bh)
    return Workload(f"grid{W}x{H}_b{bw}x{bh}", g, part, k, queries.random_pairs(g.n, q, seed + 1), seed)


def delaunay_rcb(npts: int, levels: int, q: int, seed: int) -> Workload:
    g = graphs.delaunay(npts, seed=seed)
    part, k = partition.rcb(g.xy, levels)
    return Workload(f"delaunay{npts}_rcb{levels}", g, part, k, queries.random_pairs(g.n, q, seed + 1), seed)


def delaunay1m(q: int = 10_000_000, seed: int = 1236) -> Workload:
    w = delaunay_rcb(1 << 20, 10, q, seed)
    w.name = "delaunay1m"
    return w


def batch_instances(count: int = 512, seed: int = 1237, q_per: int = 100_000,
                    n_lo: int = 1000, n_hi: int = 65536, leaf_lo: int = 128, leaf_hi: int = 2048,
                    only: Optional[int] = None) -> list:
    """Instances of the batching workload (kd-tree components, uneven sizes).  With
    `only`, just instance number `only` (same sizes and seeds as in the full list)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        leaf = int(round(math.exp(rng.uniform(math.log(leaf_lo), math.log(leaf_hi)))))
        if only is not None and i != only:
            continue
        s = seed * 1000 + i
        if i % 2 == 0:
            g = graphs.grid_holes(n, 0.1, wmax=1000, seed=s)
        else:
            g = graphs.delaunay(n, seed=s)
            # reweight: uniform integer weights in [1, 1000], one per undirected edge
            u, v, _ = graphs.edges_from_csr(g)
            wr = np.random.default_rng(s + 1).integers(1, 1001, size=u.shape[0]).astype(np.int32)
            rp, col, ww = graphs.csr_from_edges(g.n, u, v, wr)
            g = graphs.Graph(g.n, rp, col, ww.astype(np.int32), g.xy, dict(g.meta, reweighted=True))
        part, k = partition.kdtree(g.xy, leaf)
        pairs = queries.random_pairs(g.n, q_per, s + 2)
        out.append(Workload(f"batch{i}", g, part, k, pairs, s))
    return out


def delaunay256k(q: int = 1_000_000, seed: int = 1238) -> Workload:
    g = graphs.delaunay(1 << 18, seed=seed, weight="f32_lognormal")
    part, k = partition.rcb(g.xy, 8)
    return Workload("delaunay256k", g, part, k, queries.random_pairs(g.n, q, seed + 1), seed)


def grid1024diag(q: int = 0, seed: int = 1239) -> Workload:
    g = graphs.grid_diag(1024, 1024, wmax=1000, seed=seed)
    part, k = partition.grid_blocks(1024, 1024, 32, 32)
    pairs = queries.random_pairs(g.n, q, seed + 1) if q else None
    return Workload("grid1024diag", g, part, k, pairs, seed)


WORKLOADS = {
    "grid64": grid64,
    "delaunay1m": delaunay1m,
    "delaunay256k": delaunay256k,
    "grid1024diag": grid1024diag,
}


def workload(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)
