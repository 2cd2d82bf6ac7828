"""The build's autotuner (needs a GPU): the depth of concurrent elimination runs.

The first builds of a size class try depths 3, 4 and 5 of the boundary graph's
dissection (one per build, timed by the build's stage events); later builds take the
fastest.  Whatever the depth, the boundary-graph matrix (read back in slot order) and the
answers must be the same, bit for bit, and equal to the oracle's.
"""

import numpy as np
import pytest

from _util import oracle_i32, query, spq, torch_dev

import gen
import oracle

pytestmark = pytest.mark.gpu


def test_depth_candidates_are_tried_then_the_fastest_is_kept():
    m = spq()
    torch, dev = torch_dev()
    w = gen.configs.delaunay_rcb(1 << 16, 6, 3000, seed=4711)
    g = w.graph
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    args = (g.n, T(g.row_ptr), T(g.col), T(g.w), T(w.part), w.k)
    ref = oracle_i32(oracle.pairs_dist(g.row_ptr, g.col, g.w, w.pairs[:400]))
    first_bg = first_ans = None
    cls = None
    for it in range(4):
        h = m.spq_build(*args)
        st = h.stats()
        assert st["n_bg"] >= 4096
        cls = int(st["n_bg"]).bit_length()
        ans = query(h, w.pairs)
        bg = h.bg()
        if first_bg is None:
            first_bg, first_ans = bg, ans
        else:
            assert np.array_equal(bg, first_bg), it
            assert np.array_equal(ans, first_ans), it
        assert np.array_equal(ans[:400].astype(np.int64), ref), it
        h.free()
    tun = {c: v for (_, c), v in m.spq_build_tuning().items()}
    assert cls in tun, tun
    t = tun[cls]
    assert t["depth"] in (3, 4, 5), t
    assert all(x > 0 for x in t["ms"]), t
    assert t["ms"][t["depth"] - 3] == min(t["ms"]), t
