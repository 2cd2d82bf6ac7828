"""The back-substitution's bounded dependency waits run out cleanly (needs a GPU).

In the persistent back-substitution a CTA waits for flags that other CTAs of the same
launch set when they finish the tiles it reads; every such wait is bounded.  A test hook
shortens the bound to 1 ms and has the launch release none of its tiles, so the first
tile that depends on another waits until the bound runs out.  Nothing faults and nothing
hangs: the launch stops, the build returns SPQ_ETIMEOUT and frees what it allocated, and
the next build in the same process is exact again.  This covers the component stage
(elimination of the component tables), the boundary-graph stage and the batched build.
"""

import numpy as np
import pytest

from _util import assert_pairs_exact, build, spq, torch_dev

import gen

pytestmark = pytest.mark.gpu


def test_backsub_wait_runs_out_and_the_device_stays_usable():
    m = spq()
    lib = m._lib.load()
    torch, dev = torch_dev()
    w = gen.configs.delaunay_rcb(1 << 15, 5, 5000, seed=91)
    w2 = gen.configs.delaunay_rcb(1 << 14, 4, 2000, seed=93)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    launches0 = lib.spq_kernel_launches()
    try:
        lib.spq_test_backsub_wait(1_000_000, 1)
        # component tables by elimination (its back-substitution waits first)
        with pytest.raises(m.SpqError) as e:
            build(w.graph, w.part, w.k, comp=2, bg=1)
        assert e.value.status == m.SPQ_ETIMEOUT
        # component tables by Floyd-Warshall, boundary graph by elimination
        with pytest.raises(m.SpqError) as e:
            build(w.graph, w.part, w.k, comp=1, bg=2)
        assert e.value.status == m.SPQ_ETIMEOUT
        # a batch (its component tables take the elimination form)
        graphs = [(x.graph.n, t(x.graph.row_ptr), t(x.graph.col), t(x.graph.w), t(x.part), x.k) for x in (w, w2)]
        with pytest.raises(m.SpqError) as e:
            m.spq_build_many(graphs)
        assert e.value.status == m.SPQ_ETIMEOUT
    finally:
        lib.spq_test_backsub_wait(0, 0)
    assert lib.spq_kernel_launches() > launches0
    torch.cuda.synchronize()  # the context is healthy: no sticky error
    for kw in (dict(), dict(comp=1, bg=2)):
        h = build(w.graph, w.part, w.k, **kw)
        assert_pairs_exact(h, w.graph, w.pairs)
        h.free()
    hs = m.spq_build_many([(x.graph.n, t(x.graph.row_ptr), t(x.graph.col), t(x.graph.w), t(x.part), x.k)
                           for x in (w, w2)])
    for h, x in zip(hs, (w, w2)):
        assert_pairs_exact(h, x.graph, x.pairs)
        h.free()


def test_a_generous_bound_does_not_change_the_result():
    """The hook's bound alone (flags released as usual) changes nothing."""
    m = spq()
    lib = m._lib.load()
    w = gen.configs.delaunay_rcb(1 << 14, 4, 3000, seed=95)
    try:
        lib.spq_test_backsub_wait(500_000_000, 0)
        h = build(w.graph, w.part, w.k)
        assert_pairs_exact(h, w.graph, w.pairs)
        h.free()
    finally:
        lib.spq_test_backsub_wait(0, 0)
