"""Pins of the oracle to things other than itself (CPU only).

The oracle computes dist(v, w) of the paper's Sec. 2 (minimum path length in the
undirected graph) by Dijkstra, and plain Floyd-Warshall on the dense matrix of Sec. 4.
Each test below checks it against an independent source of truth:
  - brute-force enumeration of simple paths (the definition, literally) on n <= 7;
  - Bellman-Ford written here in numpy (a different algorithm) on n <= 200;
  - scipy.sparse.csgraph's Dijkstra and Floyd-Warshall (an independent library);
  - closed forms on grids with uniform weights: c * (|dx| + |dy|);
  - metric invariants: d(v, v) = 0, symmetry, triangle inequality;
  - the golden fixtures (brute-force distance matrices of hand-made graphs for the
    cases the paper singles out: a shortest path between two vertices of one component
    that leaves the component, Sec. 3).
A plausible slip in the oracle (a dropped relaxation, one edge direction missing, the
wrong parallel edge kept, an early exit one vertex too soon, an off-by-one row_ptr bound)
fails at least one of them.
"""

import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))

import gen  # noqa: E402
import oracle  # noqa: E402
from make_golden import FIXTURES, load  # noqa: E402

INF = oracle.INF_I64


def random_graph(n, m, seed, wlo=0, whi=20, self_loops=True, parallel=True):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    if not self_loops:
        keep = u != v
        u, v = u[keep], v[keep]
    if not parallel:
        a, b = np.minimum(u, v), np.maximum(u, v)
        key = np.unique(a * n + b)
        u, v = key // n, key % n
    w = rng.integers(wlo, whi + 1, size=u.shape[0])
    rp, col, ww = gen.csr_from_edges(n, u, v, w)
    return rp, col, ww.astype(np.int64), list(zip(u.tolist(), v.tolist(), w.tolist()))


def to_i64(a):
    """float distances (inf = unreachable) -> int64 with INF."""
    out = np.full(a.shape, INF, dtype=np.int64)
    fin = np.isfinite(a)
    out[fin] = a[fin].astype(np.int64)
    return out


def bellman_ford(n, edges, src):
    """Bellman-Ford on the undirected edge list (both directions), numpy relaxations."""
    d = np.full(n, INF, dtype=np.int64)
    d[src] = 0
    if not edges:
        return d
    e = np.array(edges, dtype=np.int64)
    a = np.concatenate([e[:, 0], e[:, 1]])
    b = np.concatenate([e[:, 1], e[:, 0]])
    w = np.concatenate([e[:, 2], e[:, 2]])
    for _ in range(n):
        da = d[a]
        ok = da != INF
        cand = np.where(ok, da + w, INF)
        nd = d.copy()
        np.minimum.at(nd, b, cand)
        if np.array_equal(nd, d):
            break
        d = nd
    return d


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 8))
    m = int(rng.integers(0, 14))
    rp, col, w, edges = random_graph(n, m, seed)
    for s in range(n):
        row = oracle.sssp(rp, col, w, s)
        for t in range(n):
            bf = oracle.brute_force_dist(n, edges, s, t)
            assert row[t] == (INF if bf is None else bf), (seed, s, t)
    pairs = np.array([(s, t) for s in range(n) for t in range(n)], dtype=np.int32)
    got = oracle.pairs_dist(rp, col, w, pairs, nthreads=2)
    for (s, t), g in zip(pairs, got):
        bf = oracle.brute_force_dist(n, edges, int(s), int(t))
        assert g == (INF if bf is None else bf)


@pytest.mark.parametrize("seed", range(8))
def test_bellman_ford(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 200))
    m = int(rng.integers(n // 2, 3 * n))
    rp, col, w, edges = random_graph(n, m, 100 + seed, wlo=0, whi=50)
    for s in rng.integers(0, n, size=5):
        assert np.array_equal(oracle.sssp(rp, col, w, int(s)), bellman_ford(n, edges, int(s)))


@pytest.mark.parametrize("seed", range(4))
def test_scipy_dijkstra(seed):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra

    n = 1500
    rp, col, w, _ = random_graph(n, 4000, 200 + seed, wlo=1, whi=1000, self_loops=False, parallel=False)
    A = csr_matrix((w.astype(np.float64), col, rp), shape=(n, n))
    srcs = np.arange(0, n, 97)
    ref = dijkstra(A, directed=True, indices=srcs)
    got = oracle.multi_sssp(rp, col, w, srcs, nthreads=4)
    ref_i = to_i64(ref)
    assert np.array_equal(got, ref_i)
    rr = np.random.default_rng(seed)
    pairs = np.stack([rr.choice(srcs, 200), rr.integers(0, n, 200)], 1)
    pd = oracle.pairs_dist(rp, col, w, pairs.astype(np.int32), nthreads=4)
    exp = [ref_i[list(srcs).index(s), t] for s, t in pairs]
    assert np.array_equal(pd, np.array(exp))


@pytest.mark.parametrize("c", [1, 7])
def test_grid_closed_form(c):
    W, H = 23, 17
    g = gen.grid4(W, H, wmax=c, wmin=c, seed=0)
    for s in [0, 5, W * H - 1, 7 * W + 11]:
        row = oracle.sssp(g.row_ptr, g.col, g.w, s)
        sy, sx = divmod(s, W)
        ys, xs = np.divmod(np.arange(W * H), W)
        assert np.array_equal(row, c * (np.abs(xs - sx) + np.abs(ys - sy)))


def test_metric_invariants():
    g = gen.delaunay(3000, seed=3)
    rng = np.random.default_rng(3)
    srcs = rng.integers(0, g.n, size=12)
    rows = oracle.multi_sssp(g.row_ptr, g.col, g.w, srcs, nthreads=4)
    assert all(rows[i, s] == 0 for i, s in enumerate(srcs))
    for i, s in enumerate(srcs):
        for j, t in enumerate(srcs):
            assert rows[i, t] == rows[j, s]  # symmetry
            for k_, x in enumerate(srcs):
                assert rows[i, x] <= rows[i, t] + rows[j, x]  # triangle via t


@pytest.mark.parametrize("seed", range(6))
def test_fw_matches_dijkstra_and_scipy(seed):
    from scipy.sparse.csgraph import floyd_warshall as sp_fw

    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2, 120))
    rp, col, w, _ = random_graph(n, int(rng.integers(0, 3 * n)), 300 + seed, wlo=1, whi=30)
    dense = oracle.dense_from_csr(n, rp, col, w)
    fw = oracle.floyd_warshall(dense)
    rows = oracle.multi_sssp(rp, col, w, np.arange(n), nthreads=2)
    assert np.array_equal(fw, rows)
    sp_in = np.where(dense == INF, np.inf, dense).astype(np.float64)
    ref = sp_fw(sp_in, directed=True)
    assert np.array_equal(fw, to_i64(ref))


def test_subgraph_sssp_equals_extracted_subgraph():
    w_ = gen.configs.grid_blocks_workload(24, 24, 8, 8, 50, 10, seed=9)
    g, part = w_.graph, w_.part
    for c in [0, 4, 8]:
        ids = np.nonzero(part == c)[0]
        relabel = -np.ones(g.n, dtype=np.int64)
        relabel[ids] = np.arange(ids.shape[0])
        src_all = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        keep = (part[src_all] == c) & (part[g.col] == c) & (src_all < g.col)
        rp, col, ww = gen.csr_from_edges(ids.shape[0], relabel[src_all[keep]], relabel[g.col[keep]], g.w[keep])
        for s in ids[:5]:
            sub = oracle.subgraph_sssp(g.row_ptr, g.col, g.w, part, c, int(s))
            ref = oracle.sssp(rp, col, ww, int(relabel[s]))
            assert np.array_equal(sub[ids], ref)
            assert np.all(sub[part != c] == INF)


@pytest.mark.parametrize("name", sorted(FIXTURES))
def test_golden_fixtures(name):
    n, k, part, edges, dist = load(name)
    u = np.array([e[0] for e in edges])
    v = np.array([e[1] for e in edges])
    w = np.array([e[2] for e in edges])
    rp, col, ww = gen.csr_from_edges(n, u, v, w)
    exp = np.array(dist, dtype=np.int64)
    exp[exp < 0] = INF
    rows = oracle.multi_sssp(rp, col, ww, np.arange(n))
    assert np.array_equal(rows, exp)


def test_golden_detour_leaves_component():
    """dist_C(0, 1) inside component 0 is larger than dist_G(0, 1) (Sec. 3's remark)."""
    n, k, part, edges, dist = load("detour_two_components.txt")
    rp, col, ww = gen.csr_from_edges(n, np.array([e[0] for e in edges]), np.array([e[1] for e in edges]),
                                     np.array([e[2] for e in edges]))
    sub = oracle.subgraph_sssp(rp, col, ww, np.array(part), 0, 0)
    assert sub[1] == 100 and dist[0][1] == 3


def test_f64_matches_scipy_and_int():
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra

    g = gen.delaunay(2000, seed=11, weight="f32_lognormal")
    A = csr_matrix((g.w.astype(np.float64), g.col, g.row_ptr), shape=(g.n, g.n))
    for s in [0, 17, 1999]:
        ref = dijkstra(A, indices=s)
        got = oracle.sssp_f64(g.row_ptr, g.col, g.w, s)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    gi = gen.grid4(10, 10, wmax=9, seed=4)
    pairs = np.array([[0, 99], [5, 50], [33, 33]], dtype=np.int32)
    assert np.array_equal(oracle.pairs_dist_f64(gi.row_ptr, gi.col, gi.w, pairs),
                          oracle.pairs_dist(gi.row_ptr, gi.col, gi.w, pairs).astype(np.float64))


def test_f64_path_gradient_tree_and_fd():
    """On a tree every path is unique: the gradient of dist(v, w) is 1 on each path edge
    (both CSR slots summed), 0 elsewhere.  On a random tie-free Delaunay graph it matches
    central finite differences of the oracle's own distances."""
    # path graph 0-1-2-3-4 plus a pendant 5 on 2
    u = np.array([0, 1, 2, 3, 2])
    v = np.array([1, 2, 3, 4, 5])
    w = np.array([1.5, 2.0, 0.5, 1.0, 3.0])
    rp, col, ww = gen.csr_from_edges(6, u, v, w)
    pairs = np.array([[0, 4], [5, 1]], dtype=np.int32)
    d, grad = oracle.pairs_dist_f64(rp, col, ww, pairs, g=np.array([1.0, 2.0]))
    assert np.allclose(d, [5.0, 5.0])
    src = np.repeat(np.arange(6), np.diff(rp))
    und = {}
    for e in range(col.shape[0]):
        key = (min(src[e], col[e]), max(src[e], col[e]))
        und[key] = und.get(key, 0.0) + grad[e]
    assert und == {(0, 1): 1.0, (1, 2): 3.0, (2, 3): 1.0, (3, 4): 1.0, (2, 5): 2.0}

    g = gen.delaunay(400, seed=21, weight="f32_lognormal", scale=20.0)
    rng = np.random.default_rng(21)
    pairs = rng.integers(0, g.n, size=(30, 2)).astype(np.int32)
    up = rng.normal(size=30)
    base = g.w.astype(np.float64)
    _, grad = oracle.pairs_dist_f64(g.row_ptr, g.col, base, pairs, g=up)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    checked = 0
    for e in rng.choice(g.col.shape[0], size=40, replace=False):
        a, b = src[e], g.col[e]
        rev = np.nonzero((src == b) & (g.col == a))[0]
        slots = np.concatenate([[e], rev])
        analytic = grad[slots].sum()
        h = 1e-3 * base[e]
        fd = []
        for hh in (h, h / 2):
            wp, wm = base.copy(), base.copy()
            wp[slots] += hh
            wm[slots] -= hh
            fp = up @ oracle.pairs_dist_f64(g.row_ptr, g.col, wp, pairs)
            fm = up @ oracle.pairs_dist_f64(g.row_ptr, g.col, wm, pairs)
            fd.append((fp - fm) / (2 * hh))
        if abs(fd[0] - fd[1]) > 1e-6 * (1 + abs(fd[0])):
            continue  # not locally linear at this step (a path switch): skip this edge
        checked += 1
        assert abs(analytic - fd[0]) <= 1e-6 * (1 + abs(fd[0])), (e, analytic, fd)
    assert checked >= 30


def test_bad_input_rejected():
    rp, col, w, _ = random_graph(5, 6, 1, wlo=1, whi=3)
    w2 = w.copy()
    w2[0] = -1
    with pytest.raises(ValueError):
        oracle.sssp(rp, col, w2, 0)
    with pytest.raises(ValueError):
        oracle.pairs_dist(rp, col, w, np.array([[0, 5]], dtype=np.int32))
