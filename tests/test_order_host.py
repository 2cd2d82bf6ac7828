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


def bg_structure(w):
    """Boundary slots of a workload (component-grouped, ascending vertex id inside each
    component as the library numbers them), the component adjacency and, per slot, the
    other components its vertex touches."""
    g, part, k = w.graph, w.part, w.k
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    cross = part[src] != part[g.col]
    bnd = np.zeros(g.n, bool)
    bnd[src[cross]] = True
    slots = []
    slot_off = np.zeros(k + 1, np.int64)
    for c in range(k):
        ids = np.nonzero((part == c) & bnd)[0]
        slots.extend(ids.tolist())
        slot_off[c + 1] = slot_off[c] + ids.size
    slot_of = {v: i for i, v in enumerate(slots)}
    nbrs = [set() for _ in slots]
    edges = set()
    for a, b in zip(src[cross], g.col[cross]):
        nbrs[slot_of[int(a)]].add(int(part[b]))
        edges.add((int(part[a]), int(part[b])))
    ptr, flat, adj = csr(k, list(edges))
    snb_ptr = np.zeros(len(slots) + 1, np.int64)
    for i, s in enumerate(nbrs):
        snb_ptr[i + 1] = snb_ptr[i] + len(s)
    snb = np.array([c for s in nbrs for c in sorted(s)], np.int32)
    return slots, slot_off, ptr, flat, snb_ptr, snb, slot_of


def vertex_cost(w, slots, slot_off, order):
    """Symbolic vertex-level Floyd-Warshall cost (sum over pivots of finite rows^2 / 2)
    on the boundary graph with its clique edges."""
    g, part = w.graph, w.part
    k = w.k
    comp_of_slot = np.repeat(np.arange(k), np.diff(slot_off))
    members = [list(range(slot_off[c], slot_off[c + 1])) for c in range(k)]
    slot_of = {v: i for i, v in enumerate(slots)}
    inter = [set() for _ in slots]
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    for a, b in zip(src, g.col):
        if part[a] != part[b]:
            inter[slot_of[int(a)]].add(slot_of[int(b)])
    elim = np.zeros(len(slots), bool)
    total = 0.0
    for p in order:
        elim[p] = True
        seen = {p}
        stack = [p]
        reach = set()
        while stack:
            x = stack.pop()
            for y in list(inter[x]) + members[comp_of_slot[x]]:
                if elim[y]:
                    if y not in seen:
                        seen.add(y)
                        stack.append(y)
                else:
                    reach.add(y)
        total += (len(seen) + len(reach)) ** 2 * 0.5
    return total


@pytest.mark.parametrize("rule", [1, 2])
def test_vertex_order_is_a_permutation_and_cheaper(lib, rule):
    w = gen.configs.delaunay_rcb(1500, 3, 10, seed=3)
    slots, slot_off, ptr, flat, snb_ptr, snb, _ = bg_structure(w)
    out = np.empty(len(slots), np.int32)
    rc = lib.spq_boundary_order_host(w.k, ptr.ctypes.data, flat.ctypes.data, slot_off.ctypes.data,
                                     snb_ptr.ctypes.data, snb.ctypes.data, rule, out.ctypes.data)
    assert rc == 0
    assert sorted(out.tolist()) == list(range(len(slots)))
    comp_order = []
    nb = np.diff(slot_off).astype(np.int32)
    _, corder, _ = order_of(lib, w.k, ptr, flat, nb, rule)
    for c in corder:
        comp_order.extend(range(slot_off[c], slot_off[c + 1]))
    ident = list(range(len(slots)))
    c_id = vertex_cost(w, slots, slot_off, ident)
    c_comp = vertex_cost(w, slots, slot_off, comp_order)
    c_vert = vertex_cost(w, slots, slot_off, out.tolist())
    assert c_vert < c_comp < c_id, (c_vert, c_comp, c_id)


@pytest.mark.parametrize("depth", [0, 3, 4, 5])
def test_layout_runs_cover_every_block_row_once(lib, depth):
    """The elimination form's layout (the runs of rounds a build issues side by side):
    every slot gets its own matrix row; the runs' block-row ranges partition the matrix
    (every round done once); a run waits for the two runs of its halves, listed before it;
    the padding stays within one partial tile per aligned start (the build's memory bound);
    and there are at most 2^(depth + 1) - 1 runs."""
    w = gen.configs.delaunay_rcb(1 << 17, 7, 10, seed=5)
    slots, slot_off, ptr, flat, snb_ptr, snb, _ = bg_structure(w)
    ns = len(slots)
    assert ns >= 2 * 16 * 128 * 4  # room for at least two levels of pieces of 16 tiles
    bgpos = np.empty(ns, np.int32)
    npad = ctypes.c_longlong()
    cap = 2 ** 6
    tasks = np.full((cap, 5), -7, np.int32)
    nt = lib.spq_boundary_layout_host(w.k, ptr.ctypes.data, flat.ctypes.data, slot_off.ctypes.data,
                                      snb_ptr.ctypes.data, snb.ctypes.data, 1, depth, bgpos.ctypes.data,
                                      ctypes.byref(npad), tasks.ctypes.data, cap)
    assert nt >= 0
    npad = npad.value
    assert len(set(bgpos.tolist())) == ns and bgpos.min() >= 0 and bgpos.max() < npad
    if depth == 0:
        assert nt == 0 and npad == ns
        return
    assert 1 < nt <= 2 ** (depth + 1) - 1
    assert npad - ns <= (nt - 1) * 127
    R = (npad + 127) // 128
    cover = np.zeros(R, np.int32)
    for t in range(nt):
        lo, hi, shared_from, d0, d1 = tasks[t].tolist()
        assert 0 <= lo <= hi <= R and shared_from == hi
        cover[lo:hi] += 1
        assert (d0 == -1) == (d1 == -1), t
        if d0 >= 0:
            assert d0 < t and d1 < t and d0 != d1
            # the halves' rows come before the separator's
            assert tasks[d0][1] <= lo and tasks[d1][1] <= lo
    assert (cover == 1).all(), np.nonzero(cover != 1)[0][:10]
    leaves = sum(1 for t in range(nt) if tasks[t][3] < 0)
    assert leaves <= 2 ** depth and nt == 2 * leaves - 1
