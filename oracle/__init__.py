"""Oracle for the distance-query method: plain CPU shortest-path definitions.

TEST INFRASTRUCTURE ONLY.  Only the test suite, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg import this package.  The CUDA path never imports, links or
calls it, and shares no code with it.

What it computes (the paper's Sec. 2): dist(v, w) = minimum over v-w paths of the sum of
edge weights in the undirected graph G; dist_H for an induced subgraph H.  The method's
Lemma 3 says the query structure returns exactly dist(v1, v2), so these definitions are
the parity target.  The C functions live in `spq_oracle.c` (Dijkstra with a binary heap,
plain Floyd-Warshall); `brute_force_dist` below is pure Python for graphs of <= 8 vertices.

Every function here is pinned by `tests/test_oracle_pins.py` against things other than
itself: brute-force path enumeration, Bellman-Ford written in the test, scipy's
independent csgraph routines, the closed form |dx| + |dy| on uniform grids, symmetry,
the triangle inequality and d(v, v) = 0.
"""

from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np

INF_I64 = np.iinfo(np.int64).max
_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile spq_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    src = os.path.join(_HERE, "spq_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        lib.oracle_sssp_i64.argtypes = [i32, P, P, P, i32, P]
        lib.oracle_subgraph_sssp_i64.argtypes = [i32, P, P, P, P, i32, i32, P]
        lib.oracle_multi_sssp_i64.argtypes = [i32, P, P, P, i64, P, P, i32]
        lib.oracle_pairs_i64.argtypes = [i32, P, P, P, i64, P, P, i32]
        lib.oracle_sssp_f64.argtypes = [i32, P, P, P, i32, P]
        lib.oracle_pairs_f64.argtypes = [i32, P, P, P, i64, P, P, P, P, i32]
        lib.oracle_fw_i64.argtypes = [i32, P]
        for f in (lib.oracle_sssp_i64, lib.oracle_subgraph_sssp_i64, lib.oracle_multi_sssp_i64,
                  lib.oracle_pairs_i64, lib.oracle_sssp_f64, lib.oracle_pairs_f64, lib.oracle_fw_i64):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(row_ptr, col, w, wdtype):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=wdtype)
    return rp, c, ww


def sssp(row_ptr, col, w, src: int) -> np.ndarray:
    """int64[n] distances from src (INF_I64 if unreachable); integer weights."""
    rp, c, ww = _csr(row_ptr, col, w, np.int64)
    n = rp.shape[0] - 1
    out = np.empty(n, dtype=np.int64)
    if _load().oracle_sssp_i64(n, _p(rp), _p(c), _p(ww), int(src), _p(out)):
        raise ValueError("oracle_sssp_i64: bad input")
    return out


def subgraph_sssp(row_ptr, col, w, mask, mask_val: int, src: int) -> np.ndarray:
    """dist_H(src, .) where H is induced by {v : mask[v] == mask_val} (Sec. 2)."""
    rp, c, ww = _csr(row_ptr, col, w, np.int64)
    n = rp.shape[0] - 1
    mk = np.ascontiguousarray(mask, dtype=np.int32)
    out = np.empty(n, dtype=np.int64)
    if _load().oracle_subgraph_sssp_i64(n, _p(rp), _p(c), _p(ww), _p(mk), int(mask_val), int(src), _p(out)):
        raise ValueError("oracle_subgraph_sssp_i64: bad input")
    return out


def multi_sssp(row_ptr, col, w, srcs, nthreads: int = 0) -> np.ndarray:
    """int64[len(srcs), n]: one Dijkstra row per source (OpenMP over sources)."""
    rp, c, ww = _csr(row_ptr, col, w, np.int64)
    n = rp.shape[0] - 1
    s = np.ascontiguousarray(srcs, dtype=np.int32)
    out = np.empty((s.shape[0], n), dtype=np.int64)
    if _load().oracle_multi_sssp_i64(n, _p(rp), _p(c), _p(ww), s.shape[0], _p(s), _p(out), int(nthreads)):
        raise ValueError("oracle_multi_sssp_i64: bad input")
    return out


def pairs_dist(row_ptr, col, w, pairs, nthreads: int = 0) -> np.ndarray:
    """int64[q]: dist(v, w) per pair by early-exit Dijkstra (OpenMP over pairs)."""
    rp, c, ww = _csr(row_ptr, col, w, np.int64)
    n = rp.shape[0] - 1
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.empty(pr.shape[0], dtype=np.int64)
    if _load().oracle_pairs_i64(n, _p(rp), _p(c), _p(ww), pr.shape[0], _p(pr), _p(out), int(nthreads)):
        raise ValueError("oracle_pairs_i64: bad input")
    return out


def sssp_f64(row_ptr, col, w, src: int) -> np.ndarray:
    rp, c, ww = _csr(row_ptr, col, w, np.float64)
    n = rp.shape[0] - 1
    out = np.empty(n, dtype=np.float64)
    if _load().oracle_sssp_f64(n, _p(rp), _p(c), _p(ww), int(src), _p(out)):
        raise ValueError("oracle_sssp_f64: bad input")
    return out


def pairs_dist_f64(row_ptr, col, w, pairs, g=None, nthreads: int = 0):
    """float64[q] distances; with g (float64[q]) also returns the per-CSR-slot gradient of
    sum_i g[i] * dist_i accumulated along each pair's Dijkstra path."""
    rp, c, ww = _csr(row_ptr, col, w, np.float64)
    n = rp.shape[0] - 1
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.empty(pr.shape[0], dtype=np.float64)
    grad = None
    gp = None
    if g is not None:
        gp = np.ascontiguousarray(g, dtype=np.float64)
        grad = np.zeros(ww.shape[0], dtype=np.float64)
    rc = _load().oracle_pairs_f64(n, _p(rp), _p(c), _p(ww), pr.shape[0], _p(pr), _p(out),
                                  _p(gp) if gp is not None else None,
                                  _p(grad) if grad is not None else None, int(nthreads))
    if rc:
        raise ValueError("oracle_pairs_f64: bad input")
    return (out, grad) if g is not None else out


def dense_from_csr(n: int, row_ptr, col, w) -> np.ndarray:
    """Dense int64 n x n matrix of Sec. 4: wt(i, j) (smallest parallel edge) or INF_I64."""
    d = np.full((n, n), INF_I64, dtype=np.int64)
    rp = np.asarray(row_ptr)
    for u in range(n):
        for e in range(int(rp[u]), int(rp[u + 1])):
            v = int(col[e])
            if u != v:
                d[u, v] = min(d[u, v], int(w[e]))
    return d


def floyd_warshall(d: np.ndarray) -> np.ndarray:
    """Plain Floyd-Warshall (in a copy) on a dense int64 matrix with INF_I64 entries."""
    out = np.ascontiguousarray(d, dtype=np.int64).copy()
    n = out.shape[0]
    if _load().oracle_fw_i64(n, _p(out)):
        raise ValueError("oracle_fw_i64: bad input")
    return out


def brute_force_dist(n: int, edges, src: int, dst: int):
    """Minimum over all simple src-dst paths of the sum of edge weights (Sec. 2's
    definition, enumerated literally).  edges: iterable of undirected (u, v, w).
    Returns None if dst is unreachable.  Only for n <= 8."""
    if n > 8:
        raise ValueError("brute force is for n <= 8")
    if src == dst:
        return 0
    wt = {}
    for u, v, w in edges:
        if u == v:
            continue
        for a, b in ((u, v), (v, u)):
            wt[(a, b)] = min(wt.get((a, b), w), w)
    best = None
    others = [x for x in range(n) if x not in (src, dst)]
    for r in range(len(others) + 1):
        for mid in itertools.permutations(others, r):
            path = (src,) + mid + (dst,)
            total = 0
            ok = True
            for a, b in zip(path[:-1], path[1:]):
                if (a, b) not in wt:
                    ok = False
                    break
                total += wt[(a, b)]
            if ok and (best is None or total < best):
                best = total
    return best
