"""Graph generators: undirected edge lists -> symmetric CSR (row_ptr int64, col int32, w).

Every generator draws one weight per undirected edge and writes it in both directions,
so the CSR is symmetric as the query structure requires (the paper's graphs are
undirected: Sec. 2 defines dist(v, w) over paths of G without orientation).
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[m]
    w: np.ndarray  # int32[m] or float32[m]
    xy: Optional[np.ndarray] = None  # float64[n, 2] vertex coordinates, if geometric
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.col.shape[0])


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray) -> tuple:
    """Symmetric CSR from an undirected edge list (each edge given once).

    Adjacency lists are sorted by neighbour id; each undirected edge appears as
    (u -> v, w) and (v -> u, w)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w)
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    counts = np.bincount(src, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, dst.astype(np.int32), ww


def edges_from_csr(g: Graph) -> tuple:
    """Undirected edge list (u < v) of a symmetric CSR graph (parallel edges kept)."""
    deg = np.diff(g.row_ptr)
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    dst = g.col.astype(np.int64)
    keep = src < dst
    return src[keep], dst[keep], g.w[keep]


def _grid_edges(W: int, H: int):
    idx = np.arange(W * H, dtype=np.int64).reshape(H, W)
    hu, hv = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    vu, vv = idx[:-1, :].ravel(), idx[1:, :].ravel()
    return np.concatenate([hu, vu]), np.concatenate([hv, vv])


def grid4(W: int, H: int, wmax: int = 100, seed: int = 0, wmin: int = 1) -> Graph:
    """W x H 4-neighbour grid; vertex id = y*W + x; weights uniform in [wmin, wmax]."""
    rng = np.random.default_rng(seed)
    u, v = _grid_edges(W, H)
    w = rng.integers(wmin, wmax + 1, size=u.shape[0], dtype=np.int64).astype(np.int32)
    row_ptr, col, ww = csr_from_edges(W * H, u, v, w)
    ys, xs = np.divmod(np.arange(W * H), W)
    xy = np.stack([xs, ys], axis=1).astype(np.float64)
    return Graph(W * H, row_ptr, col, ww.astype(np.int32), xy, {"kind": "grid4", "W": W, "H": H})


def grid_diag(W: int, H: int, wmax: int = 1000, seed: int = 0) -> Graph:
    """4-neighbour grid plus, in each cell, one diagonal chosen uniformly between the
    two (down-right or down-left); the result stays planar."""
    rng = np.random.default_rng(seed)
    u, v = _grid_edges(W, H)
    idx = np.arange(W * H, dtype=np.int64).reshape(H, W)
    a = idx[:-1, :-1].ravel()  # top-left corner of each cell
    choose = rng.integers(0, 2, size=a.shape[0])
    # choose 0: (x,y)-(x+1,y+1); choose 1: (x+1,y)-(x,y+1)
    du = np.where(choose == 0, a, a + 1)
    dv = np.where(choose == 0, a + W + 1, a + W)
    u = np.concatenate([u, du])
    v = np.concatenate([v, dv])
    w = rng.integers(1, wmax + 1, size=u.shape[0], dtype=np.int64).astype(np.int32)
    row_ptr, col, ww = csr_from_edges(W * H, u, v, w)
    ys, xs = np.divmod(np.arange(W * H), W)
    xy = np.stack([xs, ys], axis=1).astype(np.float64)
    return Graph(W * H, row_ptr, col, ww.astype(np.int32), xy, {"kind": "grid_diag", "W": W, "H": H})


def grid_holes(n_target: int, frac_removed: float = 0.1, wmax: int = 1000, seed: int = 0) -> Graph:
    """4-neighbour grid with ceil(n_target / (1 - frac)) cells, then frac of the vertices
    removed uniformly at random; the survivors are renumbered densely (row-major order).
    The grid is as square as possible."""
    rng = np.random.default_rng(seed)
    cells = int(np.ceil(n_target / (1.0 - frac_removed)))
    W = int(np.ceil(np.sqrt(cells)))
    H = int(np.ceil(cells / W))
    total = W * H
    n_rm = int(round(frac_removed * total))
    removed = np.zeros(total, dtype=bool)
    removed[rng.choice(total, size=n_rm, replace=False)] = True
    newid = np.full(total, -1, dtype=np.int64)
    keep_ids = np.nonzero(~removed)[0]
    newid[keep_ids] = np.arange(keep_ids.shape[0])
    u, v = _grid_edges(W, H)
    ok = (~removed[u]) & (~removed[v])
    u, v = newid[u[ok]], newid[v[ok]]
    w = rng.integers(1, wmax + 1, size=u.shape[0], dtype=np.int64).astype(np.int32)
    n = int(keep_ids.shape[0])
    row_ptr, col, ww = csr_from_edges(n, u, v, w)
    ys, xs = np.divmod(keep_ids, W)
    xy = np.stack([xs, ys], axis=1).astype(np.float64)
    return Graph(n, row_ptr, col, ww.astype(np.int32), xy, {"kind": "grid_holes", "W": W, "H": H})


def delaunay_points(npts: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.random((npts, 2))


def delaunay_edges(xy: np.ndarray):
    """Undirected edge set (u < v) of the Delaunay triangulation of the points."""
    from scipy.spatial import Delaunay

    tri = Delaunay(xy)
    s = tri.simplices.astype(np.int64)
    e = np.concatenate([s[:, [0, 1]], s[:, [1, 2]], s[:, [0, 2]]])
    e.sort(axis=1)
    key = e[:, 0] * xy.shape[0] + e[:, 1]
    key = np.unique(key)
    return key // xy.shape[0], key % xy.shape[0]


def delaunay(npts: int, seed: int = 0, weight: str = "int_1e6", lognormal_sigma: float = 0.25,
             scale: float = 1.0) -> Graph:
    """Delaunay triangulation of npts uniform points in the unit square.

    weight = "int_1e6": w = round(1e6 * Euclidean length) as int32, clamped to >= 1.
    weight = "int": w = round(scale * Euclidean length) as int32, clamped to >= 1.
    weight = "f32_lognormal": w = scale * length * exp(N(0, sigma^2)) as float32
    (the lognormal factor is drawn once per undirected edge)."""
    xy = delaunay_points(npts, seed)
    u, v = delaunay_edges(xy)
    length = np.sqrt(((xy[u] - xy[v]) ** 2).sum(axis=1))
    meta = {"kind": "delaunay", "npts": npts}
    if weight in ("int_1e6", "int"):
        w = np.rint((1e6 if weight == "int_1e6" else scale) * length)
        meta["clamped_to_1"] = int((w < 1).sum())
        w = np.maximum(w, 1).astype(np.int32)
    elif weight == "f32_lognormal":
        rng = np.random.default_rng(seed + 7919)
        w = (scale * length * np.exp(rng.normal(0.0, lognormal_sigma, size=length.shape[0]))).astype(np.float32)
    else:
        raise ValueError(weight)
    row_ptr, col, ww = csr_from_edges(npts, u, v, w)
    return Graph(npts, row_ptr, col, ww, xy, meta)
