"""spq_build_many / spq_query_many (the batching pattern) against single builds and the
oracle (needs a GPU).

A batch of instances of uneven size and kind (grids with 10% of the vertices removed,
Delaunay triangulations, kd-tree partitions of several leaf sizes, an instance with a
single component, one with fewer components than the nested dissection needs) must
give, for every instance, the same tables and the same bit-exact distances as building
that instance alone, and the oracle's distances.
"""

import numpy as np
import pytest

from _util import assert_pairs_exact, build, oracle_i32, query, spq, torch_dev

import gen
import oracle

pytestmark = pytest.mark.gpu


def _instances():
    ins = gen.configs.batch_instances(count=10, seed=77, q_per=3000, n_lo=300, n_hi=5000, leaf_lo=40, leaf_hi=600)
    g = gen.grid4(12, 10, wmax=30, seed=5)
    ins.append(gen.configs.Workload("one_comp", g, np.zeros(g.n, np.int32), 1,
                                    gen.random_pairs(g.n, 2000, 6), 5))
    g2 = gen.grid4(20, 9, wmax=30, seed=8)
    p2, k2 = gen.grid_blocks(20, 9, 10, 9)
    ins.append(gen.configs.Workload("two_comp", g2, p2, k2, gen.random_pairs(g2.n, 2000, 9), 8))
    return ins


def _tuples(ins, on_device):
    torch, dev = torch_dev()
    T = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)) if on_device else (lambda a: a)  # noqa: E731
    return [(w.graph.n, T(w.graph.row_ptr), T(w.graph.col), T(w.graph.w), T(w.part), w.k) for w in ins]


@pytest.mark.parametrize("on_device", [True, False])
def test_batch_matches_single_builds_and_oracle(on_device):
    m = spq()
    ins = _instances()
    hs = m.spq_build_many(_tuples(ins, on_device))
    pairs = [w.pairs for w in ins]
    if on_device:
        torch, dev = torch_dev()
        outs = [o.cpu().numpy() for o in m.spq_query_many(hs, [torch.from_numpy(p).to(dev) for p in pairs])]
        torch.cuda.synchronize()
    else:
        outs = m.spq_query_many(hs, pairs)
    for w, h, o in zip(ins, hs, outs):
        single = build(w.graph, w.part, w.k)
        assert np.array_equal(o, query(single, w.pairs)), w.name
        ref = oracle_i32(oracle.pairs_dist(w.graph.row_ptr, w.graph.col, w.graph.w, w.pairs))
        assert np.array_equal(o.astype(np.int64), ref), w.name
        ms, mb = single.meta(), h.meta()
        for key in ("comp", "local", "csize", "nb", "bg_off"):
            assert np.array_equal(ms[key], mb[key]), (w.name, key)
        assert np.array_equal(single.bg(), h.bg()), w.name
        for c in range(min(w.k, 3)):
            assert np.array_equal(single.apsp(c), h.apsp(c)), (w.name, c)
        single.free()
    # free in an arbitrary order; the remaining handles stay usable
    order = np.random.default_rng(3).permutation(len(hs))
    for j, i in enumerate(order):
        if j == len(order) // 2:
            rest = [int(x) for x in order[j:]]
            for r in rest:
                assert_pairs_exact(hs[r], ins[r].graph, ins[r].pairs[:500], on_device=True)
        hs[i].free()


def test_batch_rejects_an_invalid_instance():
    m = spq()
    ins = _instances()[:4]
    tup = _tuples(ins, False)
    bad = ins[2].graph.w.copy()
    bad[0] += 1  # asymmetric
    n, rp, col, _, part, k = tup[2]
    tup[2] = (n, rp, col, bad, part, k)
    with pytest.raises(m.SpqError) as e:
        m.spq_build_many(tup)
    assert e.value.status == m.SPQ_EINVAL


def _check_batch(ins, hs, on_device=False):
    m = spq()
    outs = m.spq_query_many(hs, [w.pairs for w in ins])
    for w, h, o in zip(ins, hs, outs):
        single = build(w.graph, w.part, w.k)
        assert np.array_equal(o, query(single, w.pairs)), w.name
        ref = oracle_i32(oracle.pairs_dist(w.graph.row_ptr, w.graph.col, w.graph.w, w.pairs))
        assert np.array_equal(o.astype(np.int64), ref), w.name
        assert np.array_equal(single.bg(), h.bg()), w.name
        single.free()


def test_batch_elimination_form_for_every_instance():
    """bg_method = elimination for the whole batch: every instance's boundary graph by
    elimination + back-substitution (the forward rounds of all instances in shared
    launches, one back-substitution over all of them), the same tables and distances as
    single builds."""
    m = spq()
    ins = _instances()
    o = m.spq_opts_default()
    o.bg_method = m.SPQ_BG_ELIM
    hs = m.spq_build_many(_tuples(ins, True), opts=o)
    for w, h in zip(ins, hs):
        if h.meta()["nb"].sum() > 0:
            assert h.profile()["bg_method"] == m.SPQ_BG_ELIM, w.name
    _check_batch(ins, hs)
    for h in hs:
        h.free()


def test_batch_takes_elimination_for_large_boundary_graphs():
    """By default, instances of at least 4,096 boundary vertices take the elimination form
    (in a vertex nested-dissection order) while the others share the batched
    Floyd-Warshall rounds on a second stream; both kinds in one batch, also in int32
    arithmetic and with the back-substitution's A panels split over several launches."""
    m = spq()
    big = gen.configs.delaunay_rcb(40000, 8, 2500, seed=79)
    big.name = "big"
    ins = [big] + _instances()[:5]
    for arith, panel_mib in ((m.SPQ_ARITH_AUTO, 0), (m.SPQ_ARITH_I32, 0), (m.SPQ_ARITH_AUTO, 1)):
        o = m.spq_opts_default()
        o.arith = arith
        o.bg_panel_mib = panel_mib
        hs = m.spq_build_many(_tuples(ins, True), opts=o)
        nbg = [int(h.meta()["nb"].sum()) for h in hs]
        assert nbg[0] >= 4096 and max(nbg[1:]) < 4096
        methods = [h.profile()["bg_method"] for h in hs]
        assert methods[0] == m.SPQ_BG_ELIM and all(x == m.SPQ_BG_FW for x, n in zip(methods[1:], nbg[1:]) if n > 0)
        _check_batch(ins, hs)
        for h in hs:
            h.free()


def test_query_plan_replays_the_batch():
    """spq_query_plan: the batch captured into a CUDA graph answers like spq_query_many,
    and a replay answers the pairs the buffers hold at that time (pairs rewritten in
    place, grouped and per-pair query forms, an empty request)."""
    m = spq()
    torch, dev = torch_dev()
    ins = _instances()[:6]
    hs = m.spq_build_many(_tuples(ins, True))
    rng = np.random.default_rng(31)
    sizes = [5000, 100, 0, 9000, 4096, 7]
    bufs = [torch.from_numpy(rng.integers(0, w.graph.n, size=(q, 2)).astype(np.int32)).to(dev)
            for w, q in zip(ins, sizes)]
    plan = m.spq_query_plan(hs, bufs)
    torch.cuda.synchronize()
    ref = m.spq_query_many(hs, bufs)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(plan.outs, ref))
    for rep in range(2):
        for w, b in zip(ins, bufs):  # new pairs, same buffers
            b.copy_(torch.from_numpy(rng.integers(0, w.graph.n, size=tuple(b.shape)).astype(np.int32)))
        outs = plan.run()
        torch.cuda.synchronize()
        for h, w, b, o in zip(hs, ins, bufs, outs):
            if b.shape[0] == 0:
                continue
            p = b.cpu().numpy()
            assert np.array_equal(o.cpu().numpy(), m.spq_query(h, p)), w.name
            ref = oracle_i32(oracle.pairs_dist(w.graph.row_ptr, w.graph.col, w.graph.w, p[:200]))
            assert np.array_equal(o.cpu().numpy()[:200].astype(np.int64), ref)
    with pytest.raises(ValueError):
        m.spq_query_plan(hs[:1], [bufs[0].cpu().numpy()])
    plan.free()
    for h in hs:
        h.free()
