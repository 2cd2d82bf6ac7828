"""Parity at the benchmark's full size (needs a GPU; about two minutes).

Workload: Delaunay triangulation of 2^20 uniform points, w = round(1e6 * length),
recursive coordinate bisection into 1,024 components of 1,024 vertices, 10,000,000
query pairs; built and queried with the options the benchmark times.  The oracle
cannot answer all 10M pairs in seconds, so the check is on:
  - a seeded sample of 1,500 of the pairs, each against Dijkstra (bit-exact);
  - two complete rows: (s, w) for every vertex w, against one Dijkstra from s each;
  - properties that hold at any size, on all 10M answers or large samples: every
    answer finite (the triangulation is connected), 0 exactly when v == w, symmetry
    d(v, w) = d(w, v), and the triangle inequality through random midpoints.
"""

import numpy as np
import pytest

from _util import oracle_i32, spq, torch_dev

import gen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def built():
    torch, dev = torch_dev()
    m = spq()
    w = gen.configs.delaunay1m()
    g = w.graph
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    o = m.spq_opts_default()
    o.profile_kernels = 1
    h = m.spq_build(g.n, T(g.row_ptr), T(g.col), T(g.w), T(w.part), w.k, opts=o)
    d_pairs = T(w.pairs)
    d = m.spq_query(h, d_pairs)
    torch.cuda.synchronize()
    m.spq_query_status(h)
    yield w, h, d.cpu().numpy().astype(np.int64)
    h.free()


def _q(h, pairs):
    torch, dev = torch_dev()
    m = spq()
    d = m.spq_query(h, torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).to(dev))
    torch.cuda.synchronize()
    return d.cpu().numpy().astype(np.int64)


def test_sampled_pairs_exact(built):
    w, h, d = built
    g = w.graph
    rng = np.random.default_rng(2024)
    idx = rng.choice(w.pairs.shape[0], size=1500, replace=False)
    ref = oracle_i32(oracle.pairs_dist(g.row_ptr, g.col, g.w, w.pairs[idx]))
    bad = np.nonzero(d[idx] != ref)[0]
    assert bad.size == 0, (bad.size, w.pairs[idx[bad[0]]], d[idx[bad[0]]], ref[bad[0]])
    st = h.stats()
    assert st["n_bg"] == 133231


def test_full_rows_exact(built):
    w, h, _ = built
    g = w.graph
    for s in (0, 777_777):
        pairs = np.stack([np.full(g.n, s), np.arange(g.n)], 1).astype(np.int32)
        got = _q(h, pairs)
        ref = oracle_i32(oracle.sssp(g.row_ptr, g.col, g.w, s))
        assert np.array_equal(got, ref), s


def test_properties_at_full_size(built):
    w, h, d = built
    m = spq()
    same = w.pairs[:, 0] == w.pairs[:, 1]
    assert np.all(d < m.SPQ_INF_I32)
    assert np.all((d == 0) == same)
    rng = np.random.default_rng(5)
    idx = rng.choice(w.pairs.shape[0], size=200_000, replace=False)
    rev = _q(h, w.pairs[idx][:, ::-1])
    assert np.array_equal(rev, d[idx])
    mid = rng.integers(0, w.graph.n, size=idx.shape[0]).astype(np.int32)
    a = _q(h, np.stack([w.pairs[idx, 0], mid], 1))
    b = _q(h, np.stack([mid, w.pairs[idx, 1]], 1))
    assert np.all(d[idx] <= a + b)
