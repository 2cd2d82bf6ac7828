"""Shortest-path retrieval (needs a GPU).

Several shortest paths can tie, so what is checked is what any correct answer shares:
the path starts at v1 and ends at v2, consecutive vertices are adjacent, and the sum of
the weights along it (the lightest slot between two consecutive vertices) equals the
oracle's distance exactly (integer weights) or within float rounding (FP32 weights).
On trees the path is unique and compared vertex by vertex with the path read off a
breadth-first search from v1.  Unreachable pairs report length -1; v1 = v2 gives [v1].
"""

import numpy as np
import pytest

from _util import opts, spq, torch_dev

import gen
import oracle

pytestmark = pytest.mark.gpu


def _paths(g, part, k, pairs, max_len, **kw):
    m = spq()
    torch, dev = torch_dev()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    h = m.spq_build(g.n, T(g.row_ptr), T(g.col), T(g.w), T(part), k, opts=opts(**kw) if kw else None)
    dp = T(pairs)
    dist, saved = m.spq_query_saved(h, dp)
    verts, lens = m.spq_query_paths(h, dp, saved, max_len)
    torch.cuda.synchronize()
    m.spq_query_status(h)
    out = dist.cpu().numpy(), verts.cpu().numpy(), lens.cpu().numpy()
    h.free()
    return out


def _edge_weight(g):
    """(u, v) -> lightest slot weight from u to v."""
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    w = {}
    for u, v, x in zip(src.tolist(), g.col.tolist(), g.w.tolist()):
        if (u, v) not in w or x < w[(u, v)]:
            w[(u, v)] = x
    return w


def _check_paths(g, pairs, verts, lens, ref, exact):
    ew = _edge_weight(g)
    reach = ref != oracle.INF_I64 if exact else np.isfinite(ref)
    assert np.array_equal(lens == -1, ~reach)
    for i in np.nonzero(reach)[0]:
        v1, v2 = int(pairs[i, 0]), int(pairs[i, 1])
        L = int(lens[i])
        assert 1 <= L <= verts.shape[1], (i, L)
        p = verts[i, :L].tolist()
        assert p[0] == v1 and p[-1] == v2, (i, p[:3], p[-3:])
        tot = 0
        for a, b in zip(p[:-1], p[1:]):
            assert (a, b) in ew, (i, a, b)
            tot += ew[(a, b)]
        if exact:
            assert tot == ref[i], (i, tot, ref[i])
        else:
            assert abs(tot - ref[i]) <= 1e-5 * ref[i] + 1e-6, (i, tot, ref[i])


@pytest.mark.parametrize("order", [1, 2, 3])
def test_integer_paths_are_shortest(order):
    w = gen.configs.delaunay_rcb(6000, 3, 1500, seed=111)
    g = w.graph
    pairs = w.pairs.copy()
    pairs[:20, 1] = pairs[:20, 0]  # v1 = v2
    dist, verts, lens = _paths(g, w.part, w.k, pairs, 512, order=order)
    ref = oracle.pairs_dist(g.row_ptr, g.col, g.w, pairs)
    assert np.array_equal(dist.astype(np.int64), ref)
    assert np.all(lens[:20] == 1) and np.array_equal(verts[:20, 0], pairs[:20, 0])
    _check_paths(g, pairs, verts, lens, ref, exact=True)


def test_grid_with_holes_has_unreachable_pairs():
    # 35% of the sites removed: many small clusters, ~10% of random pairs unreachable
    g = gen.grid_holes(4000, 0.35, wmax=1000, seed=113)
    part, k = gen.kdtree(g.xy, 256)
    pairs = gen.random_pairs(g.n, 3000, 114)
    ref = oracle.pairs_dist(g.row_ptr, g.col, g.w, pairs)
    assert (ref == oracle.INF_I64).sum() > 100
    _, verts, lens = _paths(g, part, k, pairs, 1024)
    _check_paths(g, pairs, verts, lens, ref, exact=True)


def test_float_paths_are_shortest():
    g = gen.delaunay(5000, seed=115, weight="f32_lognormal", scale=float(np.sqrt(5000)))
    part, k = gen.rcb(g.xy, 3)
    pairs = gen.random_pairs(g.n, 1500, 116)
    _, verts, lens = _paths(g, part, k, pairs, 512)
    ref = oracle.pairs_dist_f64(g.row_ptr, g.col, g.w.astype(np.float64), pairs)
    gw = gen.Graph(g.n, g.row_ptr, g.col, g.w.astype(np.float64))
    _check_paths(gw, pairs, verts, lens, ref, exact=False)


def test_tree_paths_are_the_unique_path_and_truncate():
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order, minimum_spanning_tree

    d = gen.delaunay(3000, seed=117)
    rng = np.random.default_rng(117)
    u, v, _ = gen.edges_from_csr(d)
    t = minimum_spanning_tree(csr_matrix((rng.random(u.shape[0]) + 0.1, (u, v)), shape=(d.n, d.n))).tocoo()
    rp, col, ww = gen.csr_from_edges(d.n, t.row, t.col, rng.integers(1, 50, size=t.row.shape[0]))
    tree = gen.Graph(d.n, rp, col, ww.astype(np.int32), d.xy)
    part, k = gen.rcb(d.xy, 3)
    pairs = rng.integers(0, d.n, size=(400, 2)).astype(np.int32)
    A = csr_matrix((np.ones(col.shape[0]), col, rp), shape=(d.n, d.n))
    full = _paths(tree, part, k, pairs, d.n)
    short = _paths(tree, part, k, pairs, 8)
    for i, (v1, v2) in enumerate(pairs.tolist()):
        _, pred = breadth_first_order(A, v1, directed=True, return_predecessors=True)
        p = [v2]
        while p[-1] != v1:
            p.append(int(pred[p[-1]]))
        p = p[::-1]
        assert full[2][i] == len(p) and full[1][i, :len(p)].tolist() == p, i
        assert short[2][i] == len(p) and short[1][i, :min(8, len(p))].tolist() == p[:8], i


def test_empty_and_argument_errors():
    m = spq()
    torch, dev = torch_dev()
    w = gen.configs.grid64(q=10)
    g = w.graph
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    h = m.spq_build(g.n, T(g.row_ptr), T(g.col), T(g.w), T(w.part), w.k)
    e = torch.empty((0, 2), dtype=torch.int32, device=dev)
    verts, lens = m.spq_query_paths(h, e, e, 16)
    assert verts.shape == (0, 16) and lens.shape == (0,)
    dp = T(w.pairs)
    _, saved = m.spq_query_saved(h, dp)
    _, lens = m.spq_query_paths(h, dp, saved, 0)  # lengths only
    ref = oracle.pairs_dist(g.row_ptr, g.col, g.w, w.pairs)
    assert np.all(lens.cpu().numpy() >= 1) and np.all(ref < oracle.INF_I64)
    with pytest.raises(m.SpqError):
        m.spq_query_paths(h, dp, saved, -1)
    h.free()
