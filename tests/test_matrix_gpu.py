"""Many-to-many distances, spq_query_matrix (needs a GPU).

Every entry must equal spq_query on the same pair (bit-identical for integer weights, the
same table entries are minimised; for float weights bit-identical where spq_query takes
the same orientation, else within rounding) and the oracle's Dijkstra distances.  Cases: sources
and targets spread over many components, sources concentrated in one component and
targets covering whole components (the reuse the two-stage split exists for), duplicates,
v1 = v2, unreachable pairs, host buffers, float weights, out-of-range ids.
"""

import numpy as np
import pytest

from _util import build, oracle_i32, spq, torch_dev

import gen
import oracle

pytestmark = pytest.mark.gpu


def _pairs_of(src, tgt):
    s, t = np.meshgrid(src, tgt, indexing="ij")
    return np.stack([s.ravel(), t.ravel()], 1).astype(np.int32)


def _check_against_query(h, src, tgt):
    m = spq()
    torch, dev = torch_dev()
    D = m.spq_query_matrix(h, torch.from_numpy(src).to(dev), torch.from_numpy(tgt).to(dev))
    torch.cuda.synchronize()
    m.spq_query_status(h)
    ref = m.spq_query(h, torch.from_numpy(_pairs_of(src, tgt)).to(dev)).reshape(len(src), len(tgt))
    assert torch.equal(D, ref)
    return D.cpu().numpy()


def test_matrix_equals_pairwise_queries_and_oracle():
    w = gen.configs.delaunay_rcb(20000, 4, 10, seed=81)
    g = w.graph
    rng = np.random.default_rng(81)
    h = build(g, w.part, w.k)
    src = rng.integers(0, g.n, size=37).astype(np.int32)
    src[5] = src[4]  # duplicate source
    tgt = rng.integers(0, g.n, size=1500).astype(np.int32)
    tgt[:3] = src[:3]  # v1 = v2 entries
    D = _check_against_query(h, src, tgt)
    rows = oracle.multi_sssp(g.row_ptr, g.col, g.w, src[:6].astype(np.int64))
    assert np.array_equal(D[:6].astype(np.int64), oracle_i32(rows[:, tgt]))
    assert np.all(D[0, 0] == 0)
    h.free()


def test_matrix_reuse_regime_whole_components():
    """Eight sources in one component against every vertex of four components."""
    w = gen.configs.delaunay_rcb(30000, 4, 10, seed=83)
    g = w.graph
    h = build(g, w.part, w.k)
    src = np.nonzero(w.part == 3)[0][:8].astype(np.int32)
    tgt = np.nonzero(np.isin(w.part, [0, 3, 7, 12]))[0].astype(np.int32)
    D = _check_against_query(h, src, tgt)
    rows = oracle.multi_sssp(g.row_ptr, g.col, g.w, src.astype(np.int64))
    assert np.array_equal(D.astype(np.int64), oracle_i32(rows[:, tgt]))
    h.free()


def test_matrix_unreachable_host_buffers_and_errors():
    m = spq()
    a = gen.grid4(16, 16, wmax=9, seed=2)
    u, v, wt = gen.edges_from_csr(a)
    rp, col, ww = gen.csr_from_edges(2 * a.n, np.concatenate([u, u + a.n]), np.concatenate([v, v + a.n]),
                                     np.concatenate([wt, wt]))
    g = gen.Graph(2 * a.n, rp, col, ww.astype(np.int32))
    part = (np.arange(g.n) // 64).astype(np.int32)
    h = build(g, part, int(part.max()) + 1)
    src = np.array([0, 5, a.n + 3], np.int32)
    tgt = np.array([1, a.n + 7, 200, a.n + 200, 5], np.int32)
    D = m.spq_query_matrix(h, src, tgt)  # host buffers: synchronous
    ref = oracle_i32(oracle.multi_sssp(g.row_ptr, g.col, g.w, src.astype(np.int64))[:, tgt])
    assert np.array_equal(D.astype(np.int64), ref)
    assert D[0, 1] == m.SPQ_INF_I32 and D[2, 0] == m.SPQ_INF_I32
    with pytest.raises(m.SpqError):
        m.spq_query_matrix(h, np.array([0, g.n], np.int32), tgt)
    assert m.spq_query_matrix(h, np.zeros(0, np.int32), tgt).shape == (0, len(tgt))
    h.free()


def test_matrix_float_weights():
    m = spq()
    torch, dev = torch_dev()
    g = gen.delaunay(6000, seed=85, weight="f32_lognormal", scale=float(np.sqrt(6000)))
    part, k = gen.rcb(g.xy, 3)
    h = build(g, part, k)
    rng = np.random.default_rng(85)
    src = rng.integers(0, g.n, size=20).astype(np.int32)
    tgt = rng.integers(0, g.n, size=700).astype(np.int32)
    D = m.spq_query_matrix(h, torch.from_numpy(src).to(dev), torch.from_numpy(tgt).to(dev)).cpu().numpy()
    ref = m.spq_query(h, torch.from_numpy(_pairs_of(src, tgt)).to(dev)).cpu().numpy().reshape(20, 700)
    # spq_query answers a pair from its lower-numbered component's side, the matrix from the
    # source's: the same terms summed in another order, equal up to float rounding
    np.testing.assert_allclose(D, ref, rtol=1e-6, atol=0)
    comp_ok = part[src][:, None] <= part[tgt][None, :]
    assert np.array_equal(D[comp_ok], ref[comp_ok])
    exact = oracle.pairs_dist_f64(g.row_ptr, g.col, g.w.astype(np.float64), _pairs_of(src[:3], tgt))
    np.testing.assert_allclose(D[:3].ravel(), exact, rtol=2e-5)
    h.free()
