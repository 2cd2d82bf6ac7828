"""Edge-weight gradients of query distances (needs a GPU).

Float32 Delaunay graphs with lognormal weights (tie-free), coordinates scaled by sqrt(n) so
that weights are O(1) and a step of 1e-3 * w_e does not switch shortest paths.  The
backward is checked against
  - the CPU reference gradient: the oracle's Dijkstra predecessor paths, each slot on a
    pair's path credited with the pair's upstream gradient;
  - FP64 central finite differences of sum_i g_i * dist_i on 64 random edges, kept only
    where the differences at h and h/2 agree (locally linear), within rel 1e-4;
  - exact path counts on a tree with integer weights (unique paths).
"""

import numpy as np
import pytest

from _util import spq, torch_dev

import gen
import oracle

pytestmark = pytest.mark.gpu


def _undirected(g, grad):
    """Sum the two CSR slots of each undirected edge: dict (u, v) -> value (u < v)."""
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    a = np.minimum(src, g.col)
    b = np.maximum(src, g.col)
    key = a.astype(np.int64) * g.n + b
    uniq, inv = np.unique(key, return_inverse=True)
    out = np.zeros(uniq.shape[0])
    np.add.at(out, inv, grad)
    return uniq, out, inv


def _setup(npts, levels, q, seed):
    g = gen.delaunay(npts, seed=seed, weight="f32_lognormal", scale=float(np.sqrt(npts)))
    part, k = gen.rcb(g.xy, levels)
    rng = np.random.default_rng(seed)
    pairs = rng.integers(0, g.n, size=(q, 2)).astype(np.int32)
    up = rng.normal(size=q)
    return g, part, k, pairs, up


def _gpu_grad(g, part, k, pairs, up):
    m = spq()
    torch, dev = torch_dev()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    h = m.spq_build(g.n, T(g.row_ptr), T(g.col), T(g.w), T(part), k)
    dp = T(pairs)
    dist, saved = m.spq_query_saved(h, dp)
    gw = torch.zeros(g.col.shape[0], dtype=torch.float32, device=dev)
    m.spq_query_backward(h, dp, saved, T(up.astype(np.float32)), gw)
    torch.cuda.synchronize()
    m.spq_query_status(h)
    out = dist.cpu().numpy().astype(np.float64), saved.cpu().numpy(), gw.cpu().numpy().astype(np.float64)
    h.free()
    return out


def test_forward_and_backward_match_the_dijkstra_reference():
    g, part, k, pairs, up = _setup(6000, 3, 4000, seed=91)
    dist, saved, grad = _gpu_grad(g, part, k, pairs, up)
    ref_d, ref_g = oracle.pairs_dist_f64(g.row_ptr, g.col, g.w.astype(np.float64), pairs, g=up)
    np.testing.assert_allclose(dist, ref_d, rtol=2e-5, atol=0)
    assert np.all(saved[pairs[:, 0] == pairs[:, 1]] == -2)
    _, gu, _ = _undirected(g, grad)
    _, ru, _ = _undirected(g, ref_g)
    scale = np.abs(up).sum()
    np.testing.assert_allclose(gu, ru, rtol=1e-4, atol=1e-6 * scale)


def test_backward_matches_central_finite_differences():
    g, part, k, pairs, up = _setup(3000, 3, 800, seed=93)
    _, _, grad = _gpu_grad(g, part, k, pairs, up)
    keys, gu, inv = _undirected(g, grad)
    base = g.w.astype(np.float64)
    rng = np.random.default_rng(93)
    used = np.nonzero(gu != 0)[0]
    cand = np.concatenate([rng.choice(used, size=56, replace=False),
                           rng.choice(np.nonzero(gu == 0)[0], size=8, replace=False)])
    checked = 0
    for ei in cand:
        slots = np.nonzero(inv == ei)[0]
        h = 1e-3 * base[slots[0]]
        fd = []
        for hh in (h, h / 2):
            wp, wm = base.copy(), base.copy()
            wp[slots] += hh
            wm[slots] -= hh
            fp = up @ oracle.pairs_dist_f64(g.row_ptr, g.col, wp, pairs)
            fm = up @ oracle.pairs_dist_f64(g.row_ptr, g.col, wm, pairs)
            fd.append((fp - fm) / (2 * hh))
        if abs(fd[0] - fd[1]) > 1e-6 * (1 + abs(fd[0])):
            continue  # a path switches inside the step: not locally linear here
        checked += 1
        assert abs(gu[ei] - fd[0]) <= 1e-4 * (1 + abs(fd[0])), (ei, gu[ei], fd)
    assert checked >= 50


def test_autograd_function():
    m = spq()
    torch, dev = torch_dev()
    g, part, k, pairs, up = _setup(2000, 2, 500, seed=95)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    w = T(g.w).requires_grad_(True)
    dist = m.ShortestPathDistance.apply(w, T(g.row_ptr), T(g.col), T(part), k, T(pairs))
    (dist * T(up.astype(np.float32))).sum().backward()
    _, _, ref = _gpu_grad(g, part, k, pairs, up)
    np.testing.assert_allclose(w.grad.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)


def test_integer_tree_gradients_are_exact_path_counts():
    # a random spanning tree of a Delaunay triangulation: every path is unique
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree

    d = gen.delaunay(1500, seed=97)
    rng = np.random.default_rng(97)
    u, v, _ = gen.edges_from_csr(d)
    A = csr_matrix((rng.random(u.shape[0]) + 0.1, (u, v)), shape=(d.n, d.n))
    t = minimum_spanning_tree(A).tocoo()
    wts = rng.integers(1, 50, size=t.row.shape[0]).astype(np.int32)
    rp, col, ww = gen.csr_from_edges(d.n, t.row, t.col, wts)
    tree = gen.Graph(d.n, rp, col, ww.astype(np.int32), d.xy)
    part, k = gen.rcb(d.xy, 3)
    pairs = rng.integers(0, d.n, size=(600, 2)).astype(np.int32)
    up = rng.normal(size=600)
    _, _, grad = _gpu_grad(tree, part, k, pairs, up)
    _, ref = oracle.pairs_dist_f64(tree.row_ptr, tree.col, tree.w.astype(np.float64), pairs, g=up)
    _, gu, _ = _undirected(tree, grad)
    _, ru, _ = _undirected(tree, ref)
    np.testing.assert_allclose(gu, ru, rtol=1e-5, atol=1e-4)
