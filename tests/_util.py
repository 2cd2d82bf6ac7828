"""Helpers shared by the GPU parity tests (CUDA path vs the oracle)."""

import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))

import gen  # noqa: E402
import oracle  # noqa: E402

INF = None  # filled lazily (SPQ_INF_I32)


def spq():
    import paper_1503_07192_gb300 as m

    m.build()
    return m


def torch_dev():
    import torch

    return torch, torch.device("cuda:0")


def opts(arith=0, order=0, skip=1, query_grouped=1, bg=0, panel_mib=0, comp=0, query_kernel=0):
    m = spq()
    o = m.spq_opts_default()
    o.arith, o.order, o.skip_inf_tiles, o.query_grouped = arith, order, skip, query_grouped
    o.bg_method, o.bg_panel_mib, o.comp_method, o.query_kernel = bg, panel_mib, comp, query_kernel
    return o


def build(g, part, k, on_device=True, **kw):
    m = spq()
    o = opts(**kw) if kw else None
    if on_device:
        torch, dev = torch_dev()
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        return m.spq_build(g.n, t(g.row_ptr), t(g.col), t(g.w), t(part), k, opts=o)
    return m.spq_build(g.n, g.row_ptr, g.col, g.w, part, k, opts=o)


def query(h, pairs, on_device=True):
    m = spq()
    if on_device:
        torch, dev = torch_dev()
        d = m.spq_query(h, torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).to(dev))
        torch.cuda.synchronize()
        m.spq_query_status(h)
        return d.cpu().numpy()
    return m.spq_query(h, np.ascontiguousarray(pairs, dtype=np.int32))


def oracle_i32(d):
    """oracle int64 distances -> the library's int32 convention (SPQ_INF_I32 unreachable)."""
    m = spq()
    d = np.asarray(d, dtype=np.int64)
    return np.where(d == oracle.INF_I64, m.SPQ_INF_I32, d)


def assert_pairs_exact(h, g, pairs, on_device=True):
    got = query(h, pairs, on_device).astype(np.int64)
    ref = oracle_i32(oracle.pairs_dist(g.row_ptr, g.col, g.w, pairs))
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, (f"{bad.size}/{len(ref)} differ; first pair {pairs[bad[0]]}: gpu {got[bad[0]]} "
                           f"oracle {ref[bad[0]]}")


def all_pairs(n):
    s, t = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return np.stack([s.ravel(), t.ravel()], 1).astype(np.int32)


def graph_from_edges(n, edges, dtype=np.int32):
    u = np.array([e[0] for e in edges], dtype=np.int64)
    v = np.array([e[1] for e in edges], dtype=np.int64)
    w = np.array([e[2] for e in edges], dtype=dtype)
    rp, col, ww = gen.csr_from_edges(n, u, v, w)
    return gen.Graph(n, rp, col, ww.astype(dtype))


def random_graph(n, m, seed, wmax=50, wmin=1, dtype=np.int32):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    w = rng.integers(wmin, wmax + 1, size=m)
    rp, col, ww = gen.csr_from_edges(n, u, v, w)
    return gen.Graph(n, rp, col, ww.astype(dtype))
