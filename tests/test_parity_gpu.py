"""CUDA path vs the oracle, through the C ABI (needs a GPU).

Integer-weight results must be bit-identical to the oracle's dist(v, w) (the paper's
Lemma 3 says the method is exact).  Besides the final distances, the intermediate
tables are checked against the definitions they stand for:
  - APSP(C) = dist_C, Dijkstra restricted to the subgraph induced by C (Sec. 2);
  - the boundary-graph matrix = dist_G between boundary vertices (Lemma 1).
Sizes span several 128-wide tiles with ragged tails; edge cases: one component (no
boundary), every vertex its own component, empty and disconnected components,
unreachable pairs, v == w, parallel edges, self-loops, zero weights.
"""

import numpy as np
import pytest

from _util import (all_pairs, assert_pairs_exact, build, graph_from_edges, opts, oracle_i32, query,
                   random_graph, spq, torch_dev)

import gen
import oracle
from make_golden import FIXTURES, load

pytestmark = pytest.mark.gpu

ARITHS = [1, 2]  # SPQ_ARITH_I32, SPQ_ARITH_F32
ORDERS = [0, 1, 2, 3]  # SPQ_ORDER_AUTO, _ID, _DISSECTION, _VERTEX_DISSECTION
BGS = [0, 1, 2]  # SPQ_BG_AUTO, _FW, _ELIM


@pytest.mark.parametrize("name", sorted(FIXTURES))
@pytest.mark.parametrize("arith", ARITHS)
def test_golden_fixtures(name, arith):
    n, k, part, edges, dist = load(name)
    g = graph_from_edges(n, edges)
    h = build(g, np.array(part, np.int32), k, arith=arith)
    got = query(h, all_pairs(n)).reshape(n, n).astype(np.int64)
    exp = np.array(dist, dtype=np.int64)
    exp[exp < 0] = spq().SPQ_INF_I32
    assert np.array_equal(got, exp)
    h.free()


def _check_tables(h, g, part, k):
    """APSP(C) against dist_C, the boundary-graph matrix against Lemma 1."""
    meta = h.meta()
    comp, local, nb, bg_off = meta["comp"], meta["local"], meta["nb"], meta["bg_off"]
    assert np.array_equal(comp, part)
    for c in range(k):
        ids = np.nonzero(part == c)[0]
        # local order: boundary vertices first, each class by ascending id (Sec. 4, Fig. 1)
        order = ids[np.argsort(local[ids])]
        nbc = nb[c]
        assert np.all(np.diff(order[:nbc]) > 0) and np.all(np.diff(order[nbc:]) > 0)
        A = h.apsp(c)
        for li, v in enumerate(order):
            ref = oracle_i32(oracle.subgraph_sssp(g.row_ptr, g.col, g.w, part, c, int(v)))
            assert np.array_equal(A[li].astype(np.int64), ref[order]), (c, v)
    B = h.bg()
    nbg = B.shape[0]
    bvert = np.empty(nbg, np.int64)
    for c in range(k):
        ids = np.nonzero((part == c) & (local < nb[c]))[0]
        bvert[bg_off[c] + local[ids]] = ids
    rows = oracle_i32(oracle.multi_sssp(g.row_ptr, g.col, g.w, bvert))
    assert np.array_equal(B.astype(np.int64), rows[:, bvert])


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bg", BGS)
def test_grid64_all_queries_and_tables(arith, order, bg):
    w = gen.configs.grid64()
    h = build(w.graph, w.part, w.k, arith=arith, order=order, bg=bg)
    assert h.profile()["bg_method"] == (2 if bg == 2 or (bg == 0 and h.profile()["order_method"] != 0) else 1)
    st = h.stats()
    assert st["n_bg"] == 732
    assert_pairs_exact(h, w.graph, w.pairs)
    _check_tables(h, w.graph, w.part, w.k)
    h.free()


def test_modes_agree_on_delaunay():
    w = gen.configs.delaunay_rcb(6000, 3, 3000, seed=31)
    outs = []
    for arith in ARITHS:
        for order in ORDERS:
            for skip in (0, 1):
                for bg in (1, 2):
                    h = build(w.graph, w.part, w.k, arith=arith, order=order, skip=skip, bg=bg)
                    outs.append(query(h, w.pairs))
                    h.free()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    h = build(w.graph, w.part, w.k)
    assert_pairs_exact(h, w.graph, w.pairs)
    h.free()


@pytest.mark.parametrize("n", [5, 128, 300, 517])
def test_single_component_is_plain_apsp(n):
    """k = 1: no boundary vertex, the query is APSP(G) (= plain Floyd-Warshall)."""
    g = random_graph(n, 3 * n, seed=n, wmax=40)
    part = np.zeros(n, np.int32)
    h = build(g, part, 1)
    assert h.stats()["n_bg"] == 0
    got = query(h, all_pairs(n)).reshape(n, n).astype(np.int64)
    fw = oracle.floyd_warshall(oracle.dense_from_csr(n, g.row_ptr, g.col, g.w))
    assert np.array_equal(got, oracle_i32(fw))
    h.free()


@pytest.mark.parametrize("n", [1, 2, 60, 200])
def test_every_vertex_its_own_component(n):
    """k = n: every vertex with an edge is a boundary vertex and BG is G itself."""
    g = random_graph(n, 2 * n, seed=100 + n, wmax=30)
    part = np.arange(n, dtype=np.int32)
    h = build(g, part, n)
    got = query(h, all_pairs(n)).reshape(n, n).astype(np.int64)
    fw = oracle.floyd_warshall(oracle.dense_from_csr(n, g.row_ptr, g.col, g.w))
    assert np.array_equal(got, oracle_i32(fw))
    h.free()


def test_uneven_empty_and_disconnected_components():
    g = gen.delaunay(4000, seed=41)
    rng = np.random.default_rng(41)
    part, k = gen.kdtree(g.xy, 300)  # leaves of 150..300 vertices
    # merge two far-apart leaves into one (disconnected) component, leave an id empty,
    # and split one leaf into a tiny piece of 3 vertices
    part = part.copy()
    part[part == k - 1] = 0
    tiny = np.nonzero(part == 5)[0][:3]
    part[tiny] = k  # new id k; id k-1 is now empty
    k += 1
    h = build(g, part, k)
    pairs = rng.integers(0, g.n, size=(20000, 2)).astype(np.int32)
    pairs[:50, 1] = pairs[:50, 0]  # v == w
    assert_pairs_exact(h, g, pairs)
    _check_tables(h, g, part, k)
    h.free()


def test_ragged_uneven_random_graph_tables():
    """Random sparse graph, components of 1..700 vertices: several tiles and ragged
    tails in both the component blocks and the boundary-graph matrix."""
    n = 1900
    g = random_graph(n, 4 * n, seed=7, wmax=1000, wmin=0)  # zero weights allowed
    rng = np.random.default_rng(7)
    cuts = np.sort(rng.choice(np.arange(1, n), size=6, replace=False))
    part = np.searchsorted(cuts, np.arange(n), side="right").astype(np.int32)
    part = rng.permutation(7)[part].astype(np.int32)
    h = build(g, part, 7)
    assert_pairs_exact(h, g, rng.integers(0, n, size=(30000, 2)).astype(np.int32))
    _check_tables(h, g, part, 7)
    h.free()


def test_unreachable_pairs_report_inf():
    a = gen.grid4(20, 20, wmax=9, seed=1)
    # two copies side by side, no edge between them
    u, v, w = gen.edges_from_csr(a)
    u2 = np.concatenate([u, u + a.n])
    v2 = np.concatenate([v, v + a.n])
    w2 = np.concatenate([w, w])
    rp, col, ww = gen.csr_from_edges(2 * a.n, u2, v2, w2)
    g = gen.Graph(2 * a.n, rp, col, ww.astype(np.int32))
    part = (np.arange(g.n) // 100).astype(np.int32)
    h = build(g, part, 8)
    pairs = np.array([[0, a.n], [5, 799], [399, 400], [3, 3]], np.int32)
    got = query(h, pairs)
    inf = spq().SPQ_INF_I32
    assert got[0] == inf and got[1] == inf and got[2] == inf and got[3] == 0
    assert_pairs_exact(h, g, np.random.default_rng(2).integers(0, g.n, (5000, 2)).astype(np.int32))
    h.free()


def test_host_buffers_match_device_buffers():
    w = gen.configs.grid_blocks_workload(40, 30, 10, 10, 100, 4000, seed=13)
    hd = build(w.graph, w.part, w.k, on_device=True)
    hh = build(w.graph, w.part, w.k, on_device=False)
    a = query(hd, w.pairs, on_device=True)
    b = query(hh, w.pairs, on_device=False)
    c = query(hd, w.pairs, on_device=False)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert query(hd, np.zeros((0, 2), np.int32), on_device=False).shape == (0,)
    hd.free()
    hh.free()


def test_invalid_inputs_are_rejected():
    m = spq()
    g = gen.grid4(8, 8, wmax=5, seed=3)
    part = (np.arange(64) // 16).astype(np.int32)
    # asymmetric weight
    bad = g.w.copy()
    bad[0] += 1
    with pytest.raises(m.SpqError) as e:
        build(gen.Graph(g.n, g.row_ptr, g.col, bad), part, 4)
    assert e.value.status == m.SPQ_EINVAL
    # negative weight (both directions, so the graph stays symmetric)
    neg = g.w.copy()
    neg[:] = -1
    with pytest.raises(m.SpqError):
        build(gen.Graph(g.n, g.row_ptr, g.col, neg), part, 4)
    # part out of range
    with pytest.raises(m.SpqError):
        build(g, np.full(64, 4, np.int32), 4)
    # column id out of range
    col = g.col.copy()
    col[3] = 64
    with pytest.raises(m.SpqError):
        build(gen.Graph(g.n, g.row_ptr, col, g.w), part, 4)
    # a missing reverse slot
    one_way = gen.Graph(3, np.array([0, 1, 1, 1], np.int64), np.array([1], np.int32), np.array([1], np.int32))
    with pytest.raises(m.SpqError):
        build(one_way, np.zeros(3, np.int32), 1)
    h = build(g, part, 4)
    # out-of-range pair: host path returns EINVAL, device path marks the handle
    with pytest.raises(m.SpqError):
        query(h, np.array([[0, 64]], np.int32), on_device=False)
    with pytest.raises(m.SpqError):
        query(h, np.array([[-1, 3]], np.int32), on_device=True)
    # the handle stays usable
    assert query(h, np.array([[0, 63]], np.int32))[0] == oracle.pairs_dist(
        g.row_ptr, g.col, g.w, np.array([[0, 63]], np.int32))[0]
    h.free()


def test_f32_weights_within_rounding():
    """SPQ_F32 graphs: float32 sums; compared with the FP64 oracle.  A distance is a
    sum of at most H edge weights, each addition rounding by at most 2^-24 relative,
    so |gpu - exact| <= H * 2^-24 * exact; H < 200 hops here, so rtol = 2e-5."""
    g = gen.delaunay(5000, seed=51, weight="f32_lognormal", scale=100.0)
    part, k = gen.rcb(g.xy, 3)
    rng = np.random.default_rng(51)
    pairs = rng.integers(0, g.n, size=(20000, 2)).astype(np.int32)
    h = build(g, part, k)
    got = query(h, pairs).astype(np.float64)
    ref = oracle.pairs_dist_f64(g.row_ptr, g.col, g.w.astype(np.float64), pairs)
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=0)
    h.free()


def test_delaunay16k_sampled_and_full_rows():
    w = gen.configs.delaunay_rcb(1 << 14, 4, 20000, seed=61)
    h = build(w.graph, w.part, w.k)
    assert_pairs_exact(h, w.graph, w.pairs)
    g = w.graph
    srcs = np.array([0, 4097, 16383])
    rows = oracle_i32(oracle.multi_sssp(g.row_ptr, g.col, g.w, srcs))
    for i, s in enumerate(srcs):
        pairs = np.stack([np.full(g.n, s), np.arange(g.n)], 1).astype(np.int32)
        assert np.array_equal(query(h, pairs).astype(np.int64), rows[i])
    h.free()


def _build_with(w, grouped, query_kernel=0):
    return build(w.graph, w.part, w.k, query_grouped=grouped, query_kernel=query_kernel)


def test_grouped_and_input_order_queries_agree():
    """The grouped query form (pairs sorted by component pair, blocks staged in shared
    memory) and the one-warp-per-pair form give the same bit-exact answers, including
    long runs of one component pair (split across 64-pair tiles), reversed pairs,
    same-component pairs and v == w."""
    w = gen.configs.grid_blocks_workload(64, 48, 16, 16, 100, 20000, seed=17)
    g = w.graph
    rng = np.random.default_rng(17)
    same_pair = np.tile(np.array([[5, 3000]], np.int32), (5000, 1))
    one_block = np.stack([rng.integers(0, 256, 3000), 2048 + rng.integers(0, 256, 3000)], 1).astype(np.int32)
    same_comp = np.stack([rng.integers(0, 16, 2000) * 64 + rng.integers(0, 16, 2000),
                          rng.integers(0, 16, 2000) * 64 + rng.integers(0, 16, 2000)], 1).astype(np.int32)
    pairs = np.concatenate([w.pairs, same_pair, one_block, one_block[:, ::-1], same_comp,
                            np.repeat(np.arange(0, g.n, 97)[:, None], 2, 1).astype(np.int32)])
    pairs = pairs[rng.permutation(pairs.shape[0])]
    hg = _build_with(w, 1)
    hc = _build_with(w, 1, query_kernel=1)  # grouped, every block by the gathering kernel
    hu = _build_with(w, 0)
    a = query(hg, pairs)
    b = query(hu, pairs)
    c = query(hc, pairs)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert_pairs_exact(hg, g, pairs[:20000])
    hg.free()
    hu.free()
    hc.free()


def test_grouped_and_input_order_queries_agree_float_weights():
    """With float weights too both forms answer a pair from its lower-numbered
    component's side, so their sums round alike: bit-identical answers, and the same
    answer for a pair of two components given in either orientation."""
    g = gen.delaunay(8000, seed=23, weight="f32_lognormal", scale=float(np.sqrt(8000)))
    part, k = gen.rcb(g.xy, 3)
    rng = np.random.default_rng(23)
    pairs = rng.integers(0, g.n, size=(30000, 2)).astype(np.int32)
    pairs = np.concatenate([pairs, pairs[:, ::-1]])
    hg = build(g, part, k, query_grouped=1)
    hu = build(g, part, k, query_grouped=0)
    hc = build(g, part, k, query_grouped=1, query_kernel=1)
    a = query(hg, pairs)
    b = query(hu, pairs)
    assert a.dtype == np.float32 and np.array_equal(a, b) and np.array_equal(a, query(hc, pairs))
    hc.free()
    diff = part[pairs[:30000, 0]] != part[pairs[:30000, 1]]  # (same-component pairs keep their own order)
    assert np.array_equal(a[:30000][diff], a[30000:][diff])
    hg.free()
    hu.free()


def test_grouped_query_autotuner_records_its_choice():
    """The first grouped launch of a size class times both kernel configurations on its
    inputs (the answers are the same operations in both) without waiting for them; a
    later launch of the class, once the timing is complete, reads it and keeps the
    faster.  After that the class is in the table, and the chosen configuration answers
    the same."""
    m = spq()
    torch, dev = torch_dev()
    w = gen.configs.grid_blocks_workload(48, 48, 12, 12, 60, 30000, seed=29)
    h = build(w.graph, w.part, w.k, query_kernel=1)  # the gathering kernel is the tuned one
    pairs = torch.from_numpy(w.pairs).to(dev)
    a = m.spq_query(h, pairs)
    torch.cuda.synchronize()
    b = m.spq_query(h, pairs)  # reads the completed measurement
    c = m.spq_query(h, pairs)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)
    q, k, nbg = w.pairs.shape[0], w.k, int(h.meta()["nb"].sum())
    # (few boundary slots: no alignment padding, the matrix order is nbg rounded up to 4)
    N = -(-nbg // 4) * 4
    cls = 16 * (min(max(int(np.floor(np.log2(q / (k * (k + 1) / 2)))), -6), 9) + 6) + min(int(np.log2(N / k)), 15)
    table = m.spq_query_tuning()
    assert table and set(table.values()) <= {-1, 0, 1}
    assert table.get((0, cls)) in (0, 1), (cls, table)
    assert_pairs_exact(h, w.graph, w.pairs[:3000])
    h.free()


def test_first_query_of_a_size_class_does_not_wait_for_the_device():
    """The autotuner's measurement on the first launch of a size class is queued, not
    waited for: the call returns while its kernels still run (its host time is well
    below their device time)."""
    import time

    m = spq()
    torch, dev = torch_dev()
    # 4 components of 8,192 vertices (about 330 boundary slots each) and 1M pairs: a size
    # class no other test uses, and tens of milliseconds of device work; the gathering
    # kernel (the tuned one)
    w = gen.configs.delaunay_rcb(1 << 15, 2, 1_000_000, seed=31)
    h = build(w.graph, w.part, w.k, query_kernel=1)
    pairs = torch.from_numpy(w.pairs).to(dev)
    m.spq_query(h, pairs[:5000])  # another size class: loads both kernel configurations
    torch.cuda.synchronize()
    before = m.spq_query_tuning()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    t0 = time.perf_counter()
    out = m.spq_query(h, pairs)
    host_ms = (time.perf_counter() - t0) * 1e3
    e1.record(s)
    torch.cuda.synchronize()
    dev_ms = e0.elapsed_time(e1)
    after = m.spq_query_tuning()
    mine = {key: v for key, v in after.items() if key not in before}
    if not mine:
        pytest.skip("this size class was measured earlier in the process")
    assert list(mine.values()) == [-1], mine  # measured, not read yet
    assert host_ms < 0.5 * dev_ms, (host_ms, dev_ms)
    again = m.spq_query(h, pairs)
    torch.cuda.synchronize()
    assert torch.equal(out, again)
    assert m.spq_query_tuning()[next(iter(mine))] in (0, 1)  # read by the second launch
    assert_pairs_exact(h, w.graph, w.pairs[:2000])
    h.free()


def test_grouped_queries_mark_invalid_pairs():
    m = spq()
    w = gen.configs.grid_blocks_workload(32, 32, 8, 8, 50, 10000, seed=19)
    h = build(w.graph, w.part, w.k)
    pairs = w.pairs.copy()
    bad = np.array([3, 777, 9999])
    pairs[bad, 1] = w.graph.n + 5
    torch, dev = __import__("_util").torch_dev()
    d = m.spq_query(h, torch.from_numpy(pairs).to(dev))
    torch.cuda.synchronize()
    with pytest.raises(m.SpqError):
        m.spq_query_status(h)
    got = d.cpu().numpy().astype(np.int64)
    assert np.all(got[bad] == -1)
    ok = np.setdiff1d(np.arange(pairs.shape[0]), bad)
    ref = oracle_i32(oracle.pairs_dist(w.graph.row_ptr, w.graph.col, w.graph.w, pairs[ok]))
    assert np.array_equal(got[ok], ref)
    m.spq_query_status(h)  # the mark was cleared
    h.free()


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("order", [1, 3])
def test_elimination_matrix_equals_floyd_warshall(arith, order):
    """The boundary-graph matrix from elimination + back-substitution is the one
    Floyd-Warshall gives, entry for entry (60 row blocks, a ragged last block), also
    when the panels are processed in many launches of 1 MiB each, and it holds Lemma 1's
    distances."""
    w = gen.configs.delaunay_rcb(1 << 16, 6, 20000, seed=57)
    ref = build(w.graph, w.part, w.k, arith=arith, order=order, bg=1)
    B0 = ref.bg()
    ref.free()
    for panel_mib in (0, 1):
        h = build(w.graph, w.part, w.k, arith=arith, order=order, bg=2, panel_mib=panel_mib)
        assert h.profile()["bg_method"] == 2
        assert np.array_equal(h.bg(), B0)
        assert_pairs_exact(h, w.graph, w.pairs)
        h.free()
    n_bg = B0.shape[0]
    assert n_bg > 59 * 128
    # a few boundary rows against multi-source Dijkstra (Lemma 1)
    h = build(w.graph, w.part, w.k, arith=arith, order=order, bg=2)
    meta = h.meta()
    comp, local, nb, bg_off = meta["comp"], meta["local"], meta["nb"], meta["bg_off"]
    bvert = np.empty(n_bg, np.int64)
    for c in range(w.k):
        ids = np.nonzero((comp == c) & (local < nb[c]))[0]
        bvert[bg_off[c] + local[ids]] = ids
    rows = np.random.default_rng(57).choice(n_bg, size=40, replace=False)
    ref_rows = oracle_i32(oracle.multi_sssp(w.graph.row_ptr, w.graph.col, w.graph.w, bvert[rows]))
    assert np.array_equal(B0[rows].astype(np.int64), ref_rows[:, bvert])
    h.free()


@pytest.mark.parametrize("arith", ARITHS)
def test_concurrent_elimination_runs_match_floyd_warshall(arith):
    """2^17 points (about 16k boundary vertices): the dissection's top bisections are
    aligned to tiles and their elimination rounds run on concurrent streams, sharing the
    separators' tiles; the matrix must still equal Floyd-Warshall's entry for entry."""
    w = gen.configs.delaunay_rcb(1 << 17, 7, 20000, seed=61)
    ref = build(w.graph, w.part, w.k, arith=arith, bg=1)
    B0 = ref.bg()
    ref.free()
    h = build(w.graph, w.part, w.k, arith=arith, bg=2)
    assert h.profile()["bg_method"] == 2
    assert np.array_equal(h.bg(), B0)
    assert_pairs_exact(h, w.graph, w.pairs)
    h.free()


def _two_islands(weight):
    """Two far-apart Delaunay triangulations as one graph: a boundary graph in two parts
    with no path between them."""
    a = gen.delaunay(9000, seed=47, weight=weight, scale=float(np.sqrt(9000)))
    u, v, w = gen.edges_from_csr(a)
    rp, col, ww = gen.csr_from_edges(2 * a.n, np.concatenate([u, u + a.n]), np.concatenate([v, v + a.n]),
                                     np.concatenate([w, w]))
    xy = np.concatenate([a.xy, a.xy + np.array([3.0, 0.0])])
    g = gen.Graph(2 * a.n, rp, col, ww.astype(a.w.dtype), xy)
    part, k = gen.rcb(g.xy, 5)
    return g, part, k


@pytest.mark.parametrize("weight,arith", [("f32_lognormal", 0), ("int_1e6", 1)])
def test_elimination_of_a_disconnected_boundary_graph(weight, arith):
    """Row blocks with no finite entry right of the diagonal (the last blocks of the first
    island) in the forms that keep float32 values or int32 arithmetic: their tiles to the
    right must come out infinite, as Floyd-Warshall leaves them."""
    g, part, k = _two_islands(weight)
    hf = build(g, part, k, arith=arith, bg=1)
    he = build(g, part, k, arith=arith, bg=2)
    assert he.profile()["bg_method"] == 2
    Bf, Be = hf.bg(), he.bg()
    fin_f = np.isfinite(Bf) if Bf.dtype == np.float32 else Bf < 0x20000000
    fin_e = np.isfinite(Be) if Be.dtype == np.float32 else Be < 0x20000000
    assert np.array_equal(fin_f, fin_e) and not fin_e.all()
    if Be.dtype == np.float32:
        np.testing.assert_allclose(Be[fin_e], Bf[fin_f], rtol=1e-5)
    else:
        assert np.array_equal(Be, Bf)
    rng = np.random.default_rng(47)
    pairs = rng.integers(0, g.n, size=(4000, 2)).astype(np.int32)
    if Be.dtype != np.float32:
        assert_pairs_exact(he, g, pairs)
    hf.free()
    he.free()


def _mixed_components(weight, seed):
    """Delaunay kd-tree components of assorted sizes: most of several tiles, one merged
    from two far-apart leaves (disconnected), a few below one tile, and one merged from
    many leaves above the 4,096 vertices the dissection kernel orders (Floyd-Warshall)."""
    g = gen.delaunay(24000, seed=seed, weight=weight, scale=float(np.sqrt(24000)))
    part, k = gen.kdtree(g.xy, 1400)
    part = part.copy()
    part[part == k - 1] = 0                 # two far-apart leaves: a disconnected component
    part[np.isin(part, [1, 2, 3, 4, 5, 6])] = 1  # one large component
    rng = np.random.default_rng(seed)
    small = np.nonzero(part == 7)[0]
    part[small[:90]] = k - 1                # a component below one tile
    sizes = np.bincount(part, minlength=k)
    assert sizes.max() > 4096 and (sizes[sizes > 0] < 128).any() and (sizes > 128).sum() > 5
    return g, part, k, rng


@pytest.mark.parametrize("arith", [0, 1])
def test_component_elimination_equals_floyd_warshall(arith):
    """APSP(C) by elimination + back-substitution in a level-structure dissection order
    of each component equals the blocked Floyd-Warshall tables bit for bit (integer
    weights, float32 or int32 arithmetic), and the distances are the oracle's."""
    g, part, k, rng = _mixed_components("int_1e6", 53)
    hf = build(g, part, k, arith=arith, comp=1)
    he = build(g, part, k, arith=arith, comp=2)
    for c in range(k):
        assert np.array_equal(hf.apsp(c), he.apsp(c)), c
    assert np.array_equal(hf.bg(), he.bg())
    # updates: the same Floyd-Warshall count for the component above the ordering limit
    # in both builds; the others by elimination well below Floyd-Warshall's
    sizes = np.bincount(part, minlength=k)
    R = (np.ceil(sizes / 4) * 4 + 127) // 128
    fw_each = R * (1 + (R - 1) + R * (R - 1) / 2) * 128.0 ** 3
    big = fw_each[sizes > 4096].sum() + fw_each[(sizes > 0) & (np.ceil(sizes / 4) * 4 <= 128)].sum()
    su, sf = he.stats()["comp_updates"], hf.stats()["comp_updates"]
    assert sf == pytest.approx(fw_each.sum())
    assert 0 < su - big < 0.6 * (sf - big)
    # rows of the disconnected component and of the one below a tile against Dijkstra
    # inside the component
    local = he.meta()["local"]
    for c in (0, k - 1):
        ids = np.nonzero(part == c)[0]
        order = ids[np.argsort(local[ids])]
        A = he.apsp(c)
        for li in rng.choice(ids.size, 12, replace=False):
            ref = oracle_i32(oracle.subgraph_sssp(g.row_ptr, g.col, g.w, part, c, int(order[li])))
            assert np.array_equal(A[li].astype(np.int64), ref[order]), (c, li)
    pairs = rng.integers(0, g.n, size=(20000, 2)).astype(np.int32)
    assert_pairs_exact(he, g, pairs)
    hf.free()
    he.free()


def test_component_elimination_float_weights():
    g, part, k, rng = _mixed_components("f32_lognormal", 59)
    hf = build(g, part, k, comp=1)
    he = build(g, part, k, comp=2)
    for c in range(k):
        a, b = hf.apsp(c), he.apsp(c)
        assert np.array_equal(np.isinf(a), np.isinf(b)), c
        np.testing.assert_allclose(b[np.isfinite(b)], a[np.isfinite(a)], rtol=1e-5)
    pairs = rng.integers(0, g.n, size=(5000, 2)).astype(np.int32)
    exact = oracle.pairs_dist_f64(g.row_ptr, g.col, g.w.astype(np.float64), pairs)
    np.testing.assert_allclose(query(he, pairs), exact, rtol=2e-5)
    hf.free()
    he.free()


def test_elimination_profile_counts():
    m = spq()
    torch, dev = torch_dev()
    w = gen.configs.delaunay_rcb(1 << 15, 5, 10, seed=59)
    g = w.graph
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    upd = {}
    for bg in (1, 2):
        o = opts(bg=bg)
        o.profile_kernels = 1
        h = m.spq_build(g.n, t(g.row_ptr), t(g.col), t(g.w), t(w.part), w.k, opts=o)
        pf, st = h.profile(), h.stats()
        assert pf["bg_method"] == bg and len(pf) == 15
        upd[bg] = st["bg_updates"]
        if bg == 2:
            nR = -(-st["n_bg"] // 128)
            assert pf["bs_items"] >= nR * (nR + 1) // 2  # (alignment padding may add block rows)
            assert 0 < pf["bs_updates"] < st["bg_updates"] and pf["bs_ms"] > 0 and pf["bs_launches"] == 1
        h.free()
    assert upd[2] < upd[1]  # dissection order: fewer updates than Floyd-Warshall


def test_table_memory_is_pooled_and_released():
    """spq_free keeps the tables' memory in the library's pool for the next build;
    spq_release_cached_memory gives it back to the device."""
    m = spq()
    torch, dev = torch_dev()
    w = gen.configs.delaunay_rcb(1 << 16, 6, 10, seed=63)
    m.spq_release_cached_memory()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    h = build(w.graph, w.part, w.k)
    fp = h.stats()["footprint_bytes"]
    h.free()
    free1 = torch.cuda.mem_get_info(dev)[0]
    assert free1 < free0 - fp // 2  # kept in the pool
    h = build(w.graph, w.part, w.k)  # served from the pool
    assert_pairs_exact(h, w.graph, w.pairs)
    h.free()
    m.spq_release_cached_memory()
    free2 = torch.cuda.mem_get_info(dev)[0]
    assert free2 > free0 - fp // 4


def test_shorter_opts_struct_is_accepted():
    """A caller compiled against an earlier spq_opts (ending before bg_method, or before
    comp_method) gets the defaults for the newer fields; a struct_size shorter than the
    first version is rejected, and so is an unknown comp_method."""
    m = spq()
    torch, dev = torch_dev()
    w = gen.configs.grid64(q=2000)
    g = w.graph
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    o = m.spq_opts_default()
    o.bg_method = 1  # must be ignored: outside the declared size
    o.struct_size = m.SpqOpts.bg_method.offset
    h = m.spq_build(g.n, t(g.row_ptr), t(g.col), t(g.w), t(w.part), w.k, opts=o)
    assert h.profile()["bg_method"] == (2 if h.profile()["order_method"] != 0 else 1)
    assert_pairs_exact(h, g, w.pairs)
    h.free()
    o.struct_size = m.SpqOpts.bg_method.offset - 4
    with pytest.raises(m.SpqError):
        m.spq_build(g.n, t(g.row_ptr), t(g.col), t(g.w), t(w.part), w.k, opts=o)
    # a struct ending before comp_method: the component tables take the default form
    # (elimination), whatever the caller's memory beyond the declared size holds
    o = m.spq_opts_default()
    o.comp_method = 1
    hf = m.spq_build(g.n, t(g.row_ptr), t(g.col), t(g.w), t(w.part), w.k, opts=o)
    o.struct_size = m.SpqOpts.comp_method.offset
    he = m.spq_build(g.n, t(g.row_ptr), t(g.col), t(g.w), t(w.part), w.k, opts=o)
    assert he.stats()["comp_updates"] < hf.stats()["comp_updates"]
    for c in range(w.k):
        assert np.array_equal(he.apsp(c), hf.apsp(c))
    hf.free()
    he.free()
    o = m.spq_opts_default()
    o.comp_method = 3
    with pytest.raises(m.SpqError):
        m.spq_build(g.n, t(g.row_ptr), t(g.col), t(g.w), t(w.part), w.k, opts=o)


def test_wide_blocks_take_the_gathering_kernel_in_the_same_launch():
    """Grouped queries read component blocks from the block copy up to 2,048 padded
    columns; wider blocks (components with more boundary vertices) are gathered from the
    boundary matrix by the other kernel of the same launch.  A 2,200 x 3 grid cut into
    its three rows (every vertex a boundary vertex: 2,200-wide blocks) plus a narrow
    4 x 40 strip of two components joined to it: all answers against the oracle."""
    W = 2200
    u, v = [], []
    for y in range(3):
        for x in range(W):
            i = y * W + x
            if x + 1 < W:
                u.append(i), v.append(i + 1)
            if y + 1 < 3:
                u.append(i), v.append(i + W)
    base = 3 * W
    for y in range(40):
        for x in range(4):
            i = base + y * 4 + x
            if x + 1 < 4:
                u.append(i), v.append(i + 1)
            if y + 1 < 40:
                u.append(i), v.append(i + 4)
    u.append(base), v.append(0)  # the strip hangs off the grid's corner
    n = base + 160
    rng = np.random.default_rng(101)
    w = rng.integers(1, 50, size=len(u)).astype(np.int32)
    rp, col, ww = gen.csr_from_edges(n, np.array(u), np.array(v), w)
    g = gen.Graph(n, rp, col, ww.astype(np.int32))
    part = np.empty(n, np.int32)
    part[:base] = np.arange(base) // W
    part[base:] = 3 + (np.arange(160) // 80)
    h = build(g, part, 5)
    assert h.meta()["nb"].max() > 2048
    pairs = rng.integers(0, n, size=(30000, 2)).astype(np.int32)
    assert_pairs_exact(h, g, pairs)
    hu = build(g, part, 5, query_grouped=0)
    assert np.array_equal(query(h, pairs), query(hu, pairs))
    h.free()
    hu.free()


def test_query_kernel_option_and_shorter_struct():
    """A caller's spq_opts that ends before query_kernel gets the default (the staged
    grouped kernel); query_kernel = 1 gathers every block with the earlier kernel and
    answers the same; values other than 0 and 1 are rejected."""
    m = spq()
    torch, dev = torch_dev()
    w = gen.configs.grid64(q=8000)
    g = w.graph
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    o = m.spq_opts_default()
    o.query_kernel = 1
    h1 = m.spq_build(g.n, t(g.row_ptr), t(g.col), t(g.w), t(w.part), w.k, opts=o)
    o.struct_size = m.SpqOpts.query_kernel.offset  # (the 1 above lies outside the declared size)
    h0 = m.spq_build(g.n, t(g.row_ptr), t(g.col), t(g.w), t(w.part), w.k, opts=o)
    assert np.array_equal(query(h0, w.pairs), query(h1, w.pairs))
    assert_pairs_exact(h0, g, w.pairs)
    h0.free()
    h1.free()
    o = m.spq_opts_default()
    o.query_kernel = 2
    with pytest.raises(m.SpqError):
        m.spq_build(g.n, t(g.row_ptr), t(g.col), t(g.w), t(w.part), w.k, opts=o)
