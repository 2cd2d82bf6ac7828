"""Parity at the full size of the batching and serving workloads (needs a GPU; slow).

grid1024diag: 1024 x 1024 grid with one random diagonal per cell (planar), integer
weights U{1..1000}, 32 x 32-block components (1,024 of them), |BG| = 123,132.  Queried
with 2M random pairs (the grouped form); 1,500 of them are checked against Dijkstra bit
for bit, and one complete row (all 2^20 targets of one source) against one Dijkstra.

batch512: the 512 instances of the batching workload at their full recipe (half grids
with 10% of the vertices removed, half Delaunay, n log-uniform in [1,000, 65,536],
weights U{1..1000}, kd-tree components with leaf caps log-uniform in [128, 2,048]),
built with one spq_build_many and queried with their 100,000 pairs each through
spq_query_many, as the benchmark does.  Per instance 1,000 sampled pairs against
Dijkstra (Lemma 3: exact); for three instances whose boundary graph takes the batched
elimination (|BG| >= 4,096) sampled rows of the boundary matrix against multi-source
Dijkstra (Lemma 1) and sampled rows of APSP(C) against Dijkstra inside C (Sec. 2).
"""

import numpy as np
import pytest

from _util import oracle_i32, spq, torch_dev

import gen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _dev(a):
    torch, dev = torch_dev()
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def test_grid1024diag_sampled_pairs_and_a_full_row():
    m = spq()
    torch, _ = torch_dev()
    w = gen.configs.grid1024diag()
    g = w.graph
    h = m.spq_build(g.n, _dev(g.row_ptr), _dev(g.col), _dev(g.w), _dev(w.part), w.k)
    assert h.stats()["n_bg"] == 123_132
    pairs = gen.random_pairs(g.n, 2_000_000, 4242)
    d = m.spq_query(h, _dev(pairs))
    torch.cuda.synchronize()
    m.spq_query_status(h)
    d = d.cpu().numpy().astype(np.int64)
    idx = np.random.default_rng(4243).choice(pairs.shape[0], size=1500, replace=False)
    ref = oracle_i32(oracle.pairs_dist(g.row_ptr, g.col, g.w, pairs[idx]))
    bad = np.nonzero(d[idx] != ref)[0]
    assert bad.size == 0, (bad.size, pairs[idx[bad[0]]], d[idx[bad[0]]], ref[bad[0]])
    s = 524_287
    row_pairs = np.stack([np.full(g.n, s), np.arange(g.n)], 1).astype(np.int32)
    got = m.spq_query(h, _dev(row_pairs))
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy().astype(np.int64), oracle_i32(oracle.sssp(g.row_ptr, g.col, g.w, s)))
    h.free()


def _slots(meta, k):
    """Vertex of every boundary slot (slot = bg_off[c] + local index)."""
    comp, local, nb, bg_off = meta["comp"], meta["local"], meta["nb"], meta["bg_off"]
    bvert = np.empty(int(nb.sum()), np.int64)
    for c in range(k):
        ids = np.nonzero((comp == c) & (local < nb[c]))[0]
        bvert[bg_off[c] + local[ids]] = ids
    return bvert


def test_batch512_full_recipe_against_the_oracle():
    m = spq()
    torch, _ = torch_dev()
    ins = gen.configs.batch_instances()
    assert len(ins) == 512
    hs = m.spq_build_many([(x.graph.n, _dev(x.graph.row_ptr), _dev(x.graph.col), _dev(x.graph.w), _dev(x.part), x.k)
                           for x in ins])
    outs = m.spq_query_many(hs, [_dev(x.pairs) for x in ins])
    torch.cuda.synchronize()
    for h in hs:
        m.spq_query_status(h)
    rng = np.random.default_rng(512)
    big = []
    for i, (x, h, o) in enumerate(zip(ins, hs, outs)):
        g = x.graph
        idx = rng.choice(x.pairs.shape[0], size=1000, replace=False)
        got = o.cpu().numpy().astype(np.int64)[idx]
        ref = oracle_i32(oracle.pairs_dist(g.row_ptr, g.col, g.w, x.pairs[idx]))
        bad = np.nonzero(got != ref)[0]
        assert bad.size == 0, (i, bad.size, x.pairs[idx[bad[0]]], got[bad[0]], ref[bad[0]])
        if h.stats()["n_bg"] >= 4096:
            big.append(i)
    assert len(big) >= 3
    for i in (big[0], big[len(big) // 2], big[-1]):
        x, h = ins[i], hs[i]
        g = x.graph
        meta = h.meta()
        bvert = _slots(meta, x.k)
        B = h.bg()
        rows = rng.choice(bvert.shape[0], size=min(200, bvert.shape[0]), replace=False)
        ref_rows = oracle_i32(oracle.multi_sssp(g.row_ptr, g.col, g.w, bvert[rows]))
        assert np.array_equal(B[rows].astype(np.int64), ref_rows[:, bvert]), i
        local = meta["local"]
        for c in rng.choice(x.k, size=min(4, x.k), replace=False):
            ids = np.nonzero(x.part == c)[0]
            if ids.size == 0:
                continue
            order = ids[np.argsort(local[ids])]
            A = h.apsp(int(c))
            for li in rng.choice(ids.size, size=min(8, ids.size), replace=False):
                ref = oracle_i32(oracle.subgraph_sssp(g.row_ptr, g.col, g.w, x.part, int(c), int(order[li])))
                assert np.array_equal(A[li].astype(np.int64), ref[order]), (i, c, li)
    for h in hs:
        h.free()
