"""The float32 -> int32 switch of the default arithmetic (needs a GPU).

For int32 graphs the default SPQ_ARITH_AUTO computes the tables in float32, which is
exact while every stored value is below 2^24 (a float32 sum of two exact integers below
2^24 is exact, and a sum at or above 2^24 never rounds below 2^24).  The build checks
every final entry and, when one is at or above 2^24, builds again in int32 arithmetic.
These graphs have distances on both sides of 2^24 (and below 2^29, the int32 sentinel):
the answers must still be the oracle's, bit for bit (Lemma 3), the component tables
dist_C (Sec. 2) and the boundary matrix Lemma 1's distances, and the handle must report
the arithmetic it ended with.  A graph whose largest distance is just below 2^24 keeps
float32 arithmetic and is exact.
"""

import numpy as np
import pytest

from _util import assert_pairs_exact, build, oracle_i32, spq, torch_dev

import gen
import oracle
from test_parity_gpu import _check_tables

pytestmark = pytest.mark.gpu

TWO24 = 1 << 24
ARITH_I32, ARITH_F32 = 1, 2


def _grid(wmin, wmax, seed):
    g = gen.grid4(64, 64, wmax=wmax, wmin=wmin, seed=seed)
    part, k = gen.grid_blocks(64, 64, 16, 16)
    return g, part, k, gen.random_pairs(g.n, 10_000, seed + 1)


def _delaunay_long(seed):
    # w = round(2e8 * length) on the unit square: the longest distances are about 3e8,
    # above 2^24 by a factor of 18 and below 2^29
    g = gen.delaunay(1 << 14, seed=seed, weight="int", scale=2e8)
    part, k = gen.rcb(g.xy, 4)
    return g, part, k, gen.random_pairs(g.n, 10_000, seed + 1)


CASES = {
    # component tables below 2^24 (16x16 blocks: at most 30 edges of 2.5e5), the
    # boundary matrix and the answers above it (up to 126 edges)
    "grid_bg_above": lambda: _grid(150_000, 250_000, 71),
    # component tables above 2^24 already (30 edges of up to 1.2e6)
    "grid_comp_above": lambda: _grid(800_000, 1_200_000, 73),
    "delaunay_2e8": lambda: _delaunay_long(75),
}


def _max_finite(g, sources):
    rows = oracle.multi_sssp(g.row_ptr, g.col, g.w, np.asarray(sources))
    fin = rows[rows != oracle.INF_I64]
    return int(fin.max())


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("bg,comp", [(1, 1), (2, 2), (2, 1), (1, 2)])
def test_auto_arith_rebuilds_in_int32_and_stays_exact(case, bg, comp):
    g, part, k, pairs = CASES[case]()
    assert int(g.w.max()) < spq().SPQ_INF_I32
    mx = _max_finite(g, [0, g.n // 2, g.n - 1])
    assert TWO24 < mx < spq().SPQ_INF_I32, mx
    h = build(g, part, k, arith=0, bg=bg, comp=comp)
    assert h.stats()["arith"] == ARITH_I32
    assert h.profile()["bg_method"] == bg
    assert_pairs_exact(h, g, pairs)
    _check_tables(h, g, part, k)
    h.free()


@pytest.mark.parametrize("bg,comp", [(1, 1), (2, 2)])
def test_auto_arith_just_below_2_24_stays_float32(bg, comp):
    # at most 126 edges of 130,000: 16,380,000 < 2^24 = 16,777,216
    g, part, k, pairs = _grid(100_000, 130_000, 77)
    assert 126 * int(g.w.max()) < TWO24
    h = build(g, part, k, arith=0, bg=bg, comp=comp)
    assert h.stats()["arith"] == ARITH_F32
    assert_pairs_exact(h, g, pairs)
    _check_tables(h, g, part, k)
    h.free()


def test_forced_float32_falls_back_too():
    """SPQ_ARITH_F32 asks for float32 but must fall back the same way."""
    g, part, k, pairs = CASES["grid_bg_above"]()
    h = build(g, part, k, arith=2)
    assert h.stats()["arith"] == ARITH_I32
    assert_pairs_exact(h, g, pairs)
    h.free()


def test_batch_auto_arith_rebuilds_in_int32():
    """spq_build_many: one instance with long distances sends the whole batch to int32
    arithmetic; every instance stays exact.  A batch whose distances all stay below
    2^24 keeps float32."""
    m = spq()
    torch, dev = torch_dev()
    short = gen.configs.grid_blocks_workload(48, 40, 12, 10, 1000, 3000, seed=81)
    g1, p1, k1, q1 = _grid(150_000, 250_000, 83)
    g2, p2, k2, q2 = _delaunay_long(85)

    def run(items):
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        keep = [(t(g.row_ptr), t(g.col), t(g.w), t(p)) for g, p, _, _ in items]
        graphs = [(g.n, *keep[i][:3], keep[i][3], k) for i, (g, _, k, _) in enumerate(items)]
        hs = m.spq_build_many(graphs)
        for h, (g, p, k, q) in zip(hs, items):
            assert_pairs_exact(h, g, q)
        return hs

    hs = run([(short.graph, short.part, short.k, short.pairs), (g1, p1, k1, q1), (g2, p2, k2, q2)])
    assert all(h.stats()["arith"] == ARITH_I32 for h in hs)
    _check_tables(hs[1], g1, p1, k1)
    for h in hs:
        h.free()
    hs = run([(short.graph, short.part, short.k, short.pairs)] * 2)
    assert all(h.stats()["arith"] == ARITH_F32 for h in hs)
    for h in hs:
        h.free()


def test_int32_weight_at_the_sentinel_is_rejected():
    """An int32 weight at or above SPQ_INF_I32 would read as 'unreachable' (and sums of
    such weights could overflow int32): the build rejects it."""
    m = spq()
    g = gen.grid4(8, 8, wmax=5, seed=3)
    part = (np.arange(64) // 16).astype(np.int32)
    big = g.w.copy()
    big[:] = m.SPQ_INF_I32  # both directions: the graph stays symmetric
    with pytest.raises(m.SpqError) as e:
        build(gen.Graph(g.n, g.row_ptr, g.col, big), part, 4)
    assert e.value.status == m.SPQ_EINVAL
    big[:] = m.SPQ_INF_I32 - 1  # the largest accepted weight
    h = build(gen.Graph(g.n, g.row_ptr, g.col, big), part, 4)
    got = h.meta()
    assert got["comp"].shape == (64,)
    h.free()


def test_answers_above_2_24_from_tables_below_it():
    """Every table entry below 2^24 (the build keeps float32-exact arithmetic) while some
    answers exceed it: two chains of 80 vertices (one component each, odd weights of
    200,001, so that a float sum rounded in the binade above 2^24 would be off by one)
    joined end to end, plus an isolated third chain (unreachable pairs).  The grouped
    queries compute in the float encoding and recompute the answers at or above 2^24 in
    int32: all must be the oracle's."""
    L, W = 80, 200_001
    u, v = [], []
    for c in range(3):
        for i in range(L - 1):
            u.append(c * L + i), v.append(c * L + i + 1)
    u.append(L - 1), v.append(L)  # chains 0 and 1 joined; chain 2 isolated
    n = 3 * L
    rp, col, ww = gen.csr_from_edges(n, np.array(u), np.array(v), np.full(len(u), W, np.int32))
    g = gen.Graph(n, rp, col, ww.astype(np.int32))
    part = (np.arange(n) // L).astype(np.int32)
    assert (L - 1) * W < TWO24 < (2 * L - 1) * W
    h = build(g, part, 3)
    assert h.stats()["arith"] == ARITH_F32
    pairs = np.stack(np.meshgrid(np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 2).astype(np.int32)
    assert_pairs_exact(h, g, pairs)
    h.free()
