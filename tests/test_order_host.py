"""Host logic of the component order along the boundary-graph matrix (no GPU).

Floyd-Warshall is correct for any order of its intermediate vertices; the order only
decides how many tile updates are provably no-ops (an all-infinite pivot panel).  These
tests check that every method returns a permutation, and that the symbolic cost the
library minimises equals a brute-force evaluation of its definition: when component p
supplies the pivots, the finite rows are those of components joined to p through
already-eliminated components, plus their uneliminated neighbours.
"""

import ctypes

import numpy as np
import pytest

import gen


@pytest.fixture(scope="module")
def lib():
    from paper_1503_07192_gb300 import _lib, build_ext

    build_ext.build()
    return _lib.load()


def csr(k, edges):
    adj = [set() for _ in range(k)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    ptr = np.zeros(k + 1, np.int64)
    for c in range(k):
        ptr[c + 1] = ptr[c] + len(adj[c])
    flat = np.array([x for c in range(k) for x in sorted(adj[c])], np.int32)
    return ptr, flat, adj


def order_of(lib, k, ptr, flat, w, method):
    out = np.empty(k, np.int32)
    cost = (ctypes.c_double * 3)()
    pick = lib.spq_component_order_host(k, ptr.ctypes.data, flat.ctypes.data if flat.size else None,
                                        w.ctypes.data, method, out.ctypes.data, cost)
    return pick, out, list(cost)


def brute_cost(k, adj, w, order):
    elim = set()
    total = 0.0
    for p in order:
        elim.add(p)
        # components reachable from p through eliminated components, plus their neighbours
        seen = {p}
        stack = [p]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if y in elim and y not in seen:
                    seen.add(y)
                    stack.append(y)
        reach = set(seen)
        for x in seen:
            reach |= {y for y in adj[x] if y not in elim}
        r = sum(w[x] for x in reach)
        total += w[p] * r * r * 0.5
    return total


def random_planar_components(k, seed):
    rng = np.random.default_rng(seed)
    xy = rng.random((k, 2))
    if k >= 3:
        u, v = gen.graphs.delaunay_edges(xy)
        edges = list(zip(u.tolist(), v.tolist()))
    else:
        edges = [(0, 1)] if k == 2 else []
    return edges, rng.integers(1, 50, size=k).astype(np.int32)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("k", [1, 2, 7, 30])
def test_orders_are_permutations_and_costs_match_bruteforce(lib, k, seed):
    edges, w = random_planar_components(k, seed)
    ptr, flat, adj = csr(k, edges)
    for method in range(3):
        pick, order, cost = order_of(lib, k, ptr, flat, w, method)
        assert pick == method
        assert sorted(order.tolist()) == list(range(k))
        assert cost[method] == pytest.approx(brute_cost(k, adj, w, order.tolist()), rel=1e-12)
    pick, order, cost = order_of(lib, k, ptr, flat, w, 3)
    assert cost[pick] == min(cost)


def test_grid_of_components(lib):
    """32 x 32 grid of components: a nested-dissection order costs a fraction of the
    row-major id order."""
    side = 32
    idx = np.arange(side * side).reshape(side, side)
    edges = [(int(a), int(b)) for a, b in zip(idx[:, :-1].ravel(), idx[:, 1:].ravel())]
    edges += [(int(a), int(b)) for a, b in zip(idx[:-1, :].ravel(), idx[1:, :].ravel())]
    k = side * side
    ptr, flat, adj = csr(k, edges)
    w = np.full(k, 124, np.int32)
    _, _, cost = order_of(lib, k, ptr, flat, w, 3)
    n = float(w.sum())
    assert cost[0] / n ** 3 > 0.15
    assert min(cost[1], cost[2]) / n ** 3 < 0.05
