"""Vertex partitions (k-partitions in the sense of Sec. 2): part[v] in [0, k).

The paper partitions with METIS (Sec. 4); these are deterministic geometric stand-ins
that give components of a fixed size with uneven boundaries.
"""

from __future__ import annotations

import numpy as np


def grid_blocks(W: int, H: int, bw: int, bh: int) -> tuple:
    """Square-block partition of a W x H grid (vertex id = y*W + x); returns (part, k)."""
    ys, xs = np.divmod(np.arange(W * H, dtype=np.int64), W)
    nbx = (W + bw - 1) // bw
    nby = (H + bh - 1) // bh
    part = (ys // bh) * nbx + (xs // bw)
    return part.astype(np.int32), int(nbx * nby)


def _split(xy: np.ndarray, ids: np.ndarray):
    """Median split of ids along the longer side of their bounding box; stable on ties."""
    pts = xy[ids]
    span = pts.max(axis=0) - pts.min(axis=0)
    axis = 0 if span[0] >= span[1] else 1
    order = np.lexsort((ids, pts[:, axis]))  # coordinate, then vertex id
    half = ids.shape[0] // 2
    return ids[order[:half]], ids[order[half:]]


def rcb(xy: np.ndarray, levels: int) -> tuple:
    """Recursive coordinate bisection, `levels` levels deep: 2**levels components whose
    sizes differ by at most one.  Component ids follow the leaves of the bisection tree
    from left to right.  Returns (part, k)."""
    n = xy.shape[0]
    nodes = [np.arange(n, dtype=np.int64)]
    for _ in range(levels):
        nxt = []
        for ids in nodes:
            a, b = _split(xy, ids)
            nxt.append(a)
            nxt.append(b)
        nodes = nxt
    part = np.empty(n, dtype=np.int32)
    for c, ids in enumerate(nodes):
        part[ids] = c
    return part, len(nodes)


def kdtree(xy: np.ndarray, leaf_cap: int) -> tuple:
    """kd-tree partition: split at the median along the longer bounding-box side while a
    node holds more than leaf_cap vertices.  Returns (part, k); leaves numbered in
    depth-first order."""
    n = xy.shape[0]
    part = np.empty(n, dtype=np.int32)
    stack = [np.arange(n, dtype=np.int64)]
    leaves = []
    while stack:
        ids = stack.pop()
        if ids.shape[0] <= leaf_cap:
            leaves.append(ids)
            continue
        a, b = _split(xy, ids)
        stack.append(b)
        stack.append(a)
    for c, ids in enumerate(leaves):
        part[ids] = c
    return part, len(leaves)
