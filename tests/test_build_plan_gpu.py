"""spq_build_plan_* (the batching pattern's captured build) against fresh builds and the
oracle (needs a GPU).

A build plan keeps the structure-only steps of Algorithm 1 and replays the
weight-dependent launches from a CUDA graph.  After each run with new weights, every
instance must hold the same tables and answer with the same bit-exact distances as a
fresh spq_build_many of the re-weighted graphs, and the oracle's distances.  Bad weights
are refused before any table changes; distances beyond 2^24 send an int32 plan's run
through the exact int32 arithmetic.
"""

import numpy as np
import pytest

from _util import oracle_i32, opts, query, spq, torch_dev

import gen
import oracle

pytestmark = pytest.mark.gpu


def _instances():
    return gen.configs.batch_instances(count=6, seed=91, q_per=1500, n_lo=400, n_hi=4000, leaf_lo=40, leaf_hi=400)


def _reweight(g, seed, lo, hi, f32=False):
    """Symmetric new weights: one value per unordered vertex pair, in the CSR's slot order."""
    u = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    v = g.col.astype(np.int64)
    key = np.minimum(u, v) * g.n + np.maximum(u, v)
    uniq, inv = np.unique(key, return_inverse=True)
    rng = np.random.default_rng(seed)
    if f32:
        vals = rng.uniform(lo, hi, uniq.shape[0]).astype(np.float32)
    else:
        vals = rng.integers(lo, hi + 1, uniq.shape[0]).astype(np.int32)
    return vals[inv.reshape(-1)]


def _tuples(ins, ws=None):
    return [(w.graph.n, w.graph.row_ptr, w.graph.col, w.graph.w if ws is None else ws[i], w.part, w.k)
            for i, w in enumerate(ins)]


def _check_against_fresh(m, ins, ws, hs, o=None, n_pairs=600):
    fresh = m.spq_build_many(_tuples(ins, ws), opts=o)
    for i, (w, h, f) in enumerate(zip(ins, hs, fresh)):
        pairs = w.pairs[:n_pairs]
        got = query(h, pairs)
        assert np.array_equal(got, query(f, pairs)), w.name
        assert np.array_equal(h.bg(), f.bg()), w.name
        for c in range(min(w.k, 3)):
            assert np.array_equal(h.apsp(c), f.apsp(c)), (w.name, c)
        if ws[i].dtype == np.int32:
            ref = oracle_i32(oracle.pairs_dist(w.graph.row_ptr, w.graph.col, ws[i], pairs))
            assert np.array_equal(got.astype(np.int64), ref), w.name
    for f in fresh:
        f.free()


@pytest.mark.parametrize("bg,comp", [(0, 0), (2, 0), (1, 1)])
def test_plan_reweights_like_fresh_builds(bg, comp):
    m = spq()
    o = opts(bg=bg, comp=comp)
    ins = _instances()
    plan = m.spq_build_plan(_tuples(ins), opts=o)
    try:
        _check_against_fresh(m, ins, [w.graph.w for w in ins], plan.handles, o)
        torch, dev = torch_dev()
        for r in range(2):
            ws = [_reweight(w.graph, 100 * r + i, 1, 1000) for i, w in enumerate(ins)]
            # host weights on the first run, device weights on the second
            arg = ws if r == 0 else [torch.from_numpy(x).to(dev) for x in ws]
            plan.run(arg)
            assert all(h.stats()["arith"] == m.SPQ_ARITH_F32 for h in plan.handles)
            _check_against_fresh(m, ins, ws, plan.handles, o)
    finally:
        plan.free()


def test_plan_float_weights_match_fresh_builds():
    m = spq()
    ins = _instances()[:4]
    ws0 = [_reweight(w.graph, 7 + i, 0.5, 20.0, f32=True) for i, w in enumerate(ins)]
    plan = m.spq_build_plan(_tuples(ins, ws0))
    try:
        ws = [_reweight(w.graph, 70 + i, 0.5, 20.0, f32=True) for i, w in enumerate(ins)]
        plan.run(ws)
        fresh = m.spq_build_many(_tuples(ins, ws))
        for w, h, f in zip(ins, plan.handles, fresh):
            assert np.array_equal(query(h, w.pairs[:500]), query(f, w.pairs[:500])), w.name
            assert np.array_equal(h.bg(), f.bg()), w.name
            f.free()
    finally:
        plan.free()


def test_plan_refuses_bad_weights_and_keeps_its_tables():
    m = spq()
    ins = _instances()[:3]
    plan = m.spq_build_plan(_tuples(ins))
    try:
        before = [query(h, w.pairs[:400]) for w, h in zip(ins, plan.handles)]
        ws = [w.graph.w.copy() for w in ins]
        ws[1][0] = -3
        with pytest.raises(m.SpqError) as ei:
            plan.run(ws)
        assert ei.value.status == m.SPQ_EINVAL
        ws = [w.graph.w.copy() for w in ins]
        ws[2][0] += 1  # one slot of an undirected edge changed: asymmetric
        with pytest.raises(m.SpqError):
            plan.run(ws)
        for w, h, b in zip(ins, plan.handles, before):
            assert np.array_equal(query(h, w.pairs[:400]), b), w.name
        # spq_free leaves a plan's handle alone (the binding's and the C entry point)
        m.spq_free(plan.handles[0])
        m._lib.load().spq_free(plan.handles[0].ptr)
        assert np.array_equal(query(plan.handles[0], ins[0].pairs[:400]), before[0])
    finally:
        plan.free()


def test_plan_run_switches_to_int32_for_long_distances_and_back():
    m = spq()
    ins = _instances()[:3]
    plan = m.spq_build_plan(_tuples(ins))
    try:
        assert all(h.stats()["arith"] == m.SPQ_ARITH_F32 for h in plan.handles)
        # weights whose sums pass 2^24 on long paths (still below 2^29)
        big = [_reweight(w.graph, 300 + i, 400_000, 500_000) for i, w in enumerate(ins)]
        plan.run(big)
        assert all(h.stats()["arith"] == m.SPQ_ARITH_I32 for h in plan.handles)
        _check_against_fresh(m, ins, big, plan.handles)
        small = [_reweight(w.graph, 400 + i, 1, 1000) for i, w in enumerate(ins)]
        plan.run(small)
        assert all(h.stats()["arith"] == m.SPQ_ARITH_F32 for h in plan.handles)
        _check_against_fresh(m, ins, small, plan.handles)
    finally:
        plan.free()
