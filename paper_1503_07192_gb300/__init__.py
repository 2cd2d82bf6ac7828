"""Shortest-path distance queries on partitioned planar graphs, on one GB300 GPU.

Thin Python binding of the C ABI in include/spq.h: the functions below have the C
names and only marshal arguments (numpy arrays or torch tensors, host or device) into
pointers.  Every step of the build (Algorithm 1 of Chapuis & Djidjev, arXiv 1503.07192)
and of the queries (Algorithm 2) runs in the library's CUDA kernels; there is no
Python or CPU fallback, and a missing library raises.

    h = spq_build(n, row_ptr, col, w, part, k)     # -> SpqHandle
    d = spq_query(h, pairs)                        # int32[q] (or float32[q])
    spq_free(h)

Importing the binding sets CUDA_DEVICE_MAX_CONNECTIONS to 32 unless the environment
already sets it: the build runs up to 32 independent chains of elimination rounds on
their own streams, and a CUDA context created with the default 8 hardware work queues
serialises them.  It only takes effect if no CUDA context exists yet in the process.
"""

from __future__ import annotations

import ctypes
import os

os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    SPQ_ECUDA,
    SPQ_EINVAL,
    SPQ_ENOMEM,
    SPQ_ETIMEOUT,
    SPQ_EUNSUPPORTED,
    SPQ_OK,
    SPQ_ARITH_AUTO,
    SPQ_ARITH_F32,
    SPQ_ARITH_I32,
    SPQ_F32,
    SPQ_I32,
    SPQ_INF_I32,
    SPQ_NOALLOC_MAX_PAIRS,
    SPQ_BG_AUTO,
    SPQ_BG_ELIM,
    SPQ_BG_FW,
    SPQ_ORDER_AUTO,
    SPQ_ORDER_DISSECTION,
    SPQ_ORDER_ID,
    SPQ_ORDER_VERTEX_DISSECTION,
    SpqError,
    SpqOpts,
)

try:  # torch is optional for host-only callers
    import torch
except Exception:  # pragma: no cover
    torch = None


def _is_torch(x) -> bool:
    return torch is not None and isinstance(x, torch.Tensor)


def _ptr(x, dtype):
    """(pointer, keepalive, is_device) for a numpy array or torch tensor of dtype."""
    if _is_torch(x):
        tdt = {np.int32: torch.int32, np.int64: torch.int64, np.float32: torch.float32}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            x = x.to(tdt).contiguous()
        return ctypes.c_void_p(x.data_ptr()), x, x.is_cuda
    a = np.ascontiguousarray(x, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), a, False


def _stream(stream, device: bool):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if device and torch is not None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def spq_opts_default() -> SpqOpts:
    o = SpqOpts()
    _lib.load().spq_opts_default(ctypes.byref(o))
    return o


class SpqHandle:
    """Owner of one built query structure (the device tables of one graph)."""

    def __init__(self, ptr: ctypes.c_void_p, n: int, k: int, wt: int):
        self._h = ptr
        self.n, self.k, self.wt = n, k, wt

    @property
    def ptr(self):
        if not self._h:
            raise ValueError("handle already freed")
        return self._h

    def stats(self) -> dict:
        nbg, cu, bu, ar = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        _lib.load().spq_stats(self.ptr, ctypes.byref(nbg), ctypes.byref(cu), ctypes.byref(bu), ctypes.byref(ar))
        return {"n_bg": nbg.value, "comp_updates": cu.value, "bg_updates": bu.value, "arith": ar.value,
                "footprint_bytes": int(_lib.load().spq_footprint_bytes(self.ptr))}

    def profile(self) -> dict:
        """Device milliseconds of the build stages (CUDA events), the phase-3 kernel
        timing of the boundary-graph Floyd-Warshall (or elimination) and of the
        back-substitution when built with profile_kernels, the order and the method."""
        ms = (ctypes.c_double * 15)()
        cnt = _lib.load().spq_build_profile(self.ptr, ms, 15)
        names = ["validate", "reorder", "comp_fw", "bg_assemble", "bg_fw", "check", "p3_ms", "p3_launches",
                 "p3_updates", "order_method", "bg_method", "bs_ms", "bs_updates", "bs_items", "bs_launches"]
        return {names[i]: ms[i] for i in range(cnt)}

    def meta(self) -> dict:
        comp = np.empty(self.n, np.int32)
        local = np.empty(self.n, np.int32)
        csize = np.empty(self.k, np.int32)
        nb = np.empty(self.k, np.int32)
        bg_off = np.empty(self.k, np.int32)
        st = _lib.load().spq_get_meta(self.ptr, *(ctypes.c_void_p(a.ctypes.data) for a in
                                                  (comp, local, csize, nb, bg_off)), ctypes.c_void_p(0))
        if st:
            raise SpqError(st, "spq_get_meta")
        return {"comp": comp, "local": local, "csize": csize, "nb": nb, "bg_off": bg_off}

    def apsp(self, c: int) -> np.ndarray:
        sz = int(self.meta()["csize"][c])
        out = np.empty((sz, sz), np.float32 if self.wt == SPQ_F32 else np.int32)
        st = _lib.load().spq_get_apsp(self.ptr, int(c), ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(0))
        if st:
            raise SpqError(st, "spq_get_apsp")
        return out

    def bg(self) -> np.ndarray:
        nbg = self.stats()["n_bg"]
        out = np.empty((nbg, nbg), np.float32 if self.wt == SPQ_F32 else np.int32)
        if nbg:
            st = _lib.load().spq_get_bg(self.ptr, ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(0))
            if st:
                raise SpqError(st, "spq_get_bg")
        return out

    def free(self):
        if self._h and not getattr(self, "plan_owned", False):  # (a build plan's: freed with it)
            _lib.load().spq_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def spq_build(n: int, row_ptr, col, w, part, k: int, opts: SpqOpts | None = None, stream=None) -> SpqHandle:
    """Build the query structure (Algorithm 1) for the symmetric CSR graph and partition."""
    lib = _lib.load()
    wt = SPQ_F32 if (getattr(w, "dtype", None) in (np.float32, np.float64) or
                     (_is_torch(w) and w.is_floating_point())) else SPQ_I32
    rp_p, rp_k, rp_d = _ptr(row_ptr, np.int64)
    col_p, col_k, _ = _ptr(col, np.int32)
    w_p, w_k, _ = _ptr(w, np.float32 if wt == SPQ_F32 else np.int32)
    pt_p, pt_k, _ = _ptr(part, np.int32)
    out = ctypes.c_void_p()
    st = lib.spq_build(int(n), rp_p, col_p, w_p, wt, pt_p, int(k), ctypes.byref(opts) if opts is not None else None,
                       _stream(stream, rp_d), ctypes.byref(out))
    del rp_k, col_k, w_k, pt_k
    if st:
        raise SpqError(st, "spq_build")
    return SpqHandle(out, int(n), int(k), wt)


def spq_build_many(graphs, opts: SpqOpts | None = None, stream=None) -> list:
    """Build many independent graphs at once.  graphs: sequence of (n, row_ptr, col, w,
    part, k) tuples (numpy arrays or tensors, host or device, one weight type for all).
    Returns one SpqHandle per graph (they share one device allocation)."""
    lib = _lib.load()
    keep = []
    arr = (_lib.SpqGraph * len(graphs))()
    wt0 = None
    dev = False
    for i, (n, row_ptr, col, w, part, k) in enumerate(graphs):
        wt = SPQ_F32 if (getattr(w, "dtype", None) in (np.float32, np.float64) or
                         (_is_torch(w) and w.is_floating_point())) else SPQ_I32
        wt0 = wt if wt0 is None else wt0
        rp_p, rp_k, rp_d = _ptr(row_ptr, np.int64)
        col_p, col_k, _ = _ptr(col, np.int32)
        w_p, w_k, _ = _ptr(w, np.float32 if wt == SPQ_F32 else np.int32)
        pt_p, pt_k, _ = _ptr(part, np.int32)
        dev = dev or rp_d
        keep += [rp_k, col_k, w_k, pt_k]
        arr[i] = _lib.SpqGraph(int(n), rp_p, col_p, w_p, wt, pt_p, int(k))
    outs = (ctypes.c_void_p * len(graphs))()
    st = lib.spq_build_many(len(graphs), arr, ctypes.byref(opts) if opts is not None else None,
                            _stream(stream, dev), outs)
    del keep
    if st:
        raise SpqError(st, "spq_build_many")
    return [SpqHandle(ctypes.c_void_p(outs[i]), int(graphs[i][0]), int(graphs[i][5]), arr[i].wt)
            for i in range(len(graphs))]


class SpqBuildPlan:
    """A batched build kept for re-weighting (spq_build_plan_*): run(weights) rebuilds
    every instance's tables from new edge weights by one CUDA graph launch.  .handles
    belong to the plan and stop working when it is freed."""

    def __init__(self, ptr, handles, m, wt):
        self._p = ptr
        self.handles, self.m, self.wt = handles, m, wt

    def run(self, weights, stream=None):
        """weights: one array / tensor per instance (m_i values, CSR slot order)."""
        if not self._p:
            raise ValueError("plan already freed")
        if len(weights) != len(self.handles):
            raise ValueError("one weight array per instance")
        arr = (ctypes.c_void_p * len(weights))()
        keep = []
        dev = False
        for i, w in enumerate(weights):
            w_p, w_k, w_d = _ptr(w, np.float32 if self.wt == SPQ_F32 else np.int32)
            if int(w_k.numel() if _is_torch(w_k) else w_k.size) != self.m[i]:
                raise ValueError(f"instance {i}: {self.m[i]} weights expected")
            dev = dev or w_d
            keep.append(w_k)
            arr[i] = w_p
        st = _lib.load().spq_build_plan_run(self._p, arr, _stream(stream, dev))
        del keep
        if st:
            raise SpqError(st, "spq_build_plan_run")
        return self.handles

    def free(self):
        if self._p:
            for h in self.handles:
                h._h = None  # (released with the plan)
            _lib.load().spq_build_plan_free(self._p)
            self._p = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def spq_build_plan(graphs, opts: SpqOpts | None = None, stream=None) -> SpqBuildPlan:
    """spq_build_many kept as a build plan: graphs as for spq_build_many; the plan copies
    them.  Returns the plan; its .handles are the instances' handles, already built."""
    lib = _lib.load()
    keep = []
    arr = (_lib.SpqGraph * len(graphs))()
    wt0 = None
    dev = False
    ms = []
    for i, (n, row_ptr, col, w, part, k) in enumerate(graphs):
        wt = SPQ_F32 if (getattr(w, "dtype", None) in (np.float32, np.float64) or
                         (_is_torch(w) and w.is_floating_point())) else SPQ_I32
        wt0 = wt if wt0 is None else wt0
        rp_p, rp_k, rp_d = _ptr(row_ptr, np.int64)
        col_p, col_k, _ = _ptr(col, np.int32)
        w_p, w_k, _ = _ptr(w, np.float32 if wt == SPQ_F32 else np.int32)
        pt_p, pt_k, _ = _ptr(part, np.int32)
        dev = dev or rp_d
        keep += [rp_k, col_k, w_k, pt_k]
        ms.append(int(w_k.numel() if _is_torch(w_k) else w_k.size))
        arr[i] = _lib.SpqGraph(int(n), rp_p, col_p, w_p, wt, pt_p, int(k))
    outs = (ctypes.c_void_p * len(graphs))()
    plan = ctypes.c_void_p()
    st = lib.spq_build_plan_create(len(graphs), arr, ctypes.byref(opts) if opts is not None else None,
                                   _stream(stream, dev), ctypes.byref(plan), outs)
    del keep
    if st:
        raise SpqError(st, "spq_build_plan_create")
    hs = [SpqHandle(ctypes.c_void_p(outs[i]), int(graphs[i][0]), int(graphs[i][5]), arr[i].wt)
          for i in range(len(graphs))]
    for h in hs:
        h.plan_owned = True
    return SpqBuildPlan(plan, hs, ms, wt0)


def spq_query_many(handles, pairs_list, outs=None, stream=None) -> list:
    """spq_query for many handles at once (all pairs host or all device)."""
    lib = _lib.load()
    n = len(handles)
    keep, outs_k = [], []
    hp = (ctypes.c_void_p * n)()
    pp = (ctypes.c_void_p * n)()
    qq = (ctypes.c_int64 * n)()
    op = (ctypes.c_void_p * n)()
    dev = False
    for i, (h, pairs) in enumerate(zip(handles, pairs_list)):
        p_p, p_k, p_dev = _ptr(pairs, np.int32)
        dev = dev or p_dev
        q = int(p_k.shape[0]) if p_k.ndim > 1 else int(p_k.shape[0]) // 2
        odt = np.float32 if h.wt == SPQ_F32 else np.int32
        o = outs[i] if outs is not None else (
            torch.empty(q, dtype=torch.float32 if h.wt == SPQ_F32 else torch.int32, device=p_k.device)
            if p_dev else np.empty(q, odt))
        o_p, o_k, _ = _ptr(o, odt)
        keep.append(p_k)
        outs_k.append(o_k)
        hp[i], pp[i], qq[i], op[i] = h.ptr, p_p, q, o_p
    st = lib.spq_query_many(n, hp, pp, qq, op, _stream(stream, dev))
    if st:
        raise SpqError(st, "spq_query_many")
    return outs_k


def spq_query(h: SpqHandle, pairs, out=None, stream=None):
    """dist(v1, v2) for each row of pairs (int32[q, 2]); returns int32[q] (float32 for
    float-weight graphs) in the same memory space as pairs."""
    lib = _lib.load()
    p_p, p_k, p_dev = _ptr(pairs, np.int32)
    q = int(p_k.shape[0]) if p_k.ndim > 1 else int(p_k.shape[0]) // 2
    odt = np.float32 if h.wt == SPQ_F32 else np.int32
    if out is None:
        if p_dev:
            out = torch.empty(q, dtype=torch.float32 if h.wt == SPQ_F32 else torch.int32, device=p_k.device)
        else:
            out = np.empty(q, odt)
    o_p, o_k, _ = _ptr(out, odt)
    st = lib.spq_query(h.ptr, p_p, q, o_p, _stream(stream, p_dev))
    if st:
        raise SpqError(st, "spq_query")
    return o_k


def spq_query_matrix(h: SpqHandle, sources, targets, out=None, stream=None):
    """dist(sources[i], targets[j]) as an [ns, nt] array (int32; float32 for float-weight
    graphs), in the memory space of the inputs (CUDA tensors or numpy arrays)."""
    lib = _lib.load()
    s_p, s_k, s_dev = _ptr(sources, np.int32)
    t_p, t_k, t_dev = _ptr(targets, np.int32)
    if s_dev != t_dev:
        raise ValueError("sources and targets must be in the same memory space")
    ns, nt = int(s_k.reshape(-1).shape[0]), int(t_k.reshape(-1).shape[0])
    odt = np.float32 if h.wt == SPQ_F32 else np.int32
    if out is None:
        if s_dev:
            out = torch.empty((ns, nt), dtype=torch.float32 if h.wt == SPQ_F32 else torch.int32, device=s_k.device)
        else:
            out = np.empty((ns, nt), odt)
    o_p, o_k, _ = _ptr(out, odt)
    st = lib.spq_query_matrix(h.ptr, s_p, ns, t_p, nt, o_p, _stream(stream, s_dev))
    if st:
        raise SpqError(st, "spq_query_matrix")
    return o_k


class SpqQueryPlan:
    """A batched query captured into a CUDA graph (spq_query_plan_*): run() answers the
    pairs the device buffers hold at that time, with one graph launch.  The handles and
    the tensors (pairs, outs) must outlive the plan."""

    def __init__(self, ptr, handles, pairs, outs):
        self._p = ptr
        self.handles, self.pairs, self.outs = list(handles), list(pairs), list(outs)

    def run(self, stream=None):
        if not self._p:
            raise ValueError("plan already freed")
        st = _lib.load().spq_query_plan_run(self._p, _stream(stream, True))
        if st:
            raise SpqError(st, "spq_query_plan_run")
        return self.outs

    def free(self):
        if self._p:
            _lib.load().spq_query_plan_free(self._p)
            self._p = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def spq_query_plan(handles, pairs_list, outs=None, stream=None) -> SpqQueryPlan:
    """Capture spq_query_many for these handles and CUDA pair tensors (int32[q, 2]) into a
    CUDA graph; the call answers the batch once, and plan.run() answers it again."""
    lib = _lib.load()
    n = len(handles)
    hp = (ctypes.c_void_p * n)()
    pp = (ctypes.c_void_p * n)()
    qq = (ctypes.c_int64 * n)()
    op = (ctypes.c_void_p * n)()
    keep, outs_k = [], []
    for i, (h, pairs) in enumerate(zip(handles, pairs_list)):
        p_p, p_k, p_dev = _ptr(pairs, np.int32)
        if not p_dev:
            raise ValueError("a query plan takes device (CUDA) pair tensors")
        q = int(p_k.shape[0]) if p_k.ndim > 1 else int(p_k.shape[0]) // 2
        o = outs[i] if outs is not None else torch.empty(
            q, dtype=torch.float32 if h.wt == SPQ_F32 else torch.int32, device=p_k.device)
        o_p, o_k, _ = _ptr(o, np.float32 if h.wt == SPQ_F32 else np.int32)
        keep.append(p_k)
        outs_k.append(o_k)
        hp[i], pp[i], qq[i], op[i] = h.ptr, p_p, q, o_p
    out = ctypes.c_void_p()
    st = lib.spq_query_plan_create(n, hp, pp, qq, op, _stream(stream, True), ctypes.byref(out))
    if st:
        raise SpqError(st, "spq_query_plan_create")
    return SpqQueryPlan(out, handles, keep, outs_k)


def spq_query_noalloc(h: SpqHandle, pairs, out=None, stream=None):
    """spq_query for callers that cannot let the library allocate device memory: pairs
    (int32[q, 2], q <= SPQ_NOALLOC_MAX_PAIRS) and out must be CUDA tensors; the
    library's fixed device scratch array is used instead of an allocation (the output,
    if not given, is allocated here by torch, outside the library)."""
    lib = _lib.load()
    p_p, p_k, p_dev = _ptr(pairs, np.int32)
    if not p_dev:
        raise ValueError("spq_query_noalloc takes device tensors")
    q = int(p_k.shape[0]) if p_k.ndim > 1 else int(p_k.shape[0]) // 2
    if out is None:
        out = torch.empty(q, dtype=torch.float32 if h.wt == SPQ_F32 else torch.int32, device=p_k.device)
    o_p, o_k, _ = _ptr(out, np.float32 if h.wt == SPQ_F32 else np.int32)
    st = lib.spq_query_noalloc(h.ptr, p_p, q, o_p, _stream(stream, True))
    if st:
        raise SpqError(st, "spq_query_noalloc")
    return o_k


def spq_query_saved(h: SpqHandle, pairs, stream=None):
    """(dist, saved) for CUDA int32[q, 2] pairs: the distances and, per pair, the
    minimising boundary pair (int32[q, 2]; negative markers, see include/spq.h)."""
    lib = _lib.load()
    p_p, p_k, p_dev = _ptr(pairs, np.int32)
    if not p_dev:
        raise ValueError("spq_query_saved takes device tensors")
    q = int(p_k.shape[0])
    dist = torch.empty(q, dtype=torch.float32 if h.wt == SPQ_F32 else torch.int32, device=p_k.device)
    saved = torch.empty((q, 2), dtype=torch.int32, device=p_k.device)
    st = lib.spq_query_saved(h.ptr, p_p, q, ctypes.c_void_p(dist.data_ptr()), ctypes.c_void_p(saved.data_ptr()),
                             _stream(stream, True))
    if st:
        raise SpqError(st, "spq_query_saved")
    return dist, saved


def spq_query_backward(h: SpqHandle, pairs, saved, grad_dist, grad_w, stream=None):
    """grad_w[e] += grad_dist[i] for every CSR slot e on pair i's shortest path (CUDA
    tensors: pairs/saved int32[q, 2], grad_dist float32[q], grad_w float32[m])."""
    lib = _lib.load()
    p_p, p_k, _ = _ptr(pairs, np.int32)
    s_p, s_k, _ = _ptr(saved, np.int32)
    g_p, g_k, _ = _ptr(grad_dist, np.float32)
    if not (grad_w.is_cuda and grad_w.dtype == torch.float32 and grad_w.is_contiguous()):
        raise ValueError("grad_w must be a contiguous CUDA float32 tensor")
    st = lib.spq_query_backward(h.ptr, p_p, int(p_k.shape[0]), s_p, g_p, ctypes.c_void_p(grad_w.data_ptr()),
                                _stream(stream, True))
    if st:
        raise SpqError(st, "spq_query_backward")
    return grad_w


def spq_release_cached_memory():
    """Return the device memory that freed handles left in the library's pool."""
    _lib.load().spq_release_cached_memory()


def spq_query_paths(h: SpqHandle, pairs, saved, max_len, stream=None):
    """(verts int32[q, max_len], lens int32[q]) on the device: the vertices of each pair's
    shortest path in order of travel (lens -1: unreachable; lens > max_len: truncated)."""
    lib = _lib.load()
    p_p, p_k, _ = _ptr(pairs, np.int32)
    s_p, s_k, _ = _ptr(saved, np.int32)
    if not (p_k.is_cuda and s_k.is_cuda):
        raise ValueError("spq_query_paths takes device tensors")
    q = int(p_k.shape[0])
    verts = torch.empty((q, max(int(max_len), 0)), dtype=torch.int32, device=p_k.device)  # (< 0: EINVAL below)
    lens = torch.empty(q, dtype=torch.int32, device=p_k.device)
    st = lib.spq_query_paths(h.ptr, p_p, q, s_p, int(max_len), ctypes.c_void_p(verts.data_ptr()),
                             ctypes.c_void_p(lens.data_ptr()), _stream(stream, True))
    if st:
        raise SpqError(st, "spq_query_paths")
    return verts, lens


if torch is not None:

    class ShortestPathDistance(torch.autograd.Function):
        """dist = ShortestPathDistance.apply(w, row_ptr, col, part, k, pairs): distances of
        the pairs in the graph whose CSR slot weights are w (float32, CUDA, one entry per
        slot; give both slots of an undirected edge the same value).  The forward builds the
        query structure (Algorithm 1) and answers the pairs keeping each one's minimising
        boundary pair; the backward walks every pair's shortest path again and accumulates
        the upstream gradient on the slots it uses."""

        @staticmethod
        def forward(ctx, w, row_ptr, col, part, k, pairs):
            h = spq_build(int(row_ptr.shape[0] - 1), row_ptr, col, w.detach().contiguous(), part, int(k))
            dist, saved = spq_query_saved(h, pairs)
            spq_query_status(h)
            ctx.h = h
            ctx.m = int(w.shape[0])
            ctx.save_for_backward(pairs, saved)
            return dist

        @staticmethod
        def backward(ctx, g):
            pairs, saved = ctx.saved_tensors
            grad_w = torch.zeros(ctx.m, dtype=torch.float32, device=pairs.device)
            spq_query_backward(ctx.h, pairs, saved, g.contiguous().to(torch.float32), grad_w)
            spq_query_status(ctx.h)
            ctx.h.free()
            return grad_w, None, None, None, None, None


def spq_query_status(h: SpqHandle, stream=None):
    st = _lib.load().spq_query_status(h.ptr, _stream(stream, True))
    if st:
        raise SpqError(st, "spq_query_status")


def spq_free(h: SpqHandle):
    h.free()


def spq_query_tuning() -> dict:
    """The grouped query's autotuner choices so far: {(device, size class): configuration}
    (0: 4 pairs per warp, two CTAs per SM; 1: 2 pairs per warp, three CTAs per SM)."""
    lib = _lib.load()
    n = int(lib.spq_query_tuning(None, None, 0))
    keys = (ctypes.c_int32 * max(n, 1))()
    ch = (ctypes.c_int32 * max(n, 1))()
    n = min(n, int(lib.spq_query_tuning(keys, ch, n)))
    return {(keys[i] // 256, keys[i] % 256): int(ch[i]) for i in range(n)}


def spq_build_tuning() -> dict:
    """The build's autotuner so far: {(device, size class): {"depth": chosen depth of
    concurrent elimination runs (-1 while trying), "ms": [stage ms at depth 3, 4, 5]}}."""
    lib = _lib.load()
    n = int(lib.spq_build_tuning(None, None, None, 0))
    keys = (ctypes.c_int32 * max(n, 1))()
    dep = (ctypes.c_int32 * max(n, 1))()
    ms = (ctypes.c_double * (3 * max(n, 1)))()
    n = min(n, int(lib.spq_build_tuning(keys, dep, ms, n)))
    return {(keys[i] // 256, keys[i] % 256): {"depth": int(dep[i]), "ms": [ms[3 * i + j] for j in range(3)]}
            for i in range(n)}


def spq_query_profile(h) -> dict | None:
    """The last grouped query launch on h (built with opts.profile_kernels = 1): the
    block-copy kernel's device ms, its min-plus updates and algorithmic bytes; None if
    there is none."""
    ms, upd, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = _lib.load().spq_query_profile(h.ptr, ctypes.byref(ms), ctypes.byref(upd), ctypes.byref(by))
    if st:
        return None
    return {"kernel_ms": ms.value, "updates": upd.value, "bytes": by.value}


def spq_kernel_launches() -> int:
    return int(_lib.load().spq_kernel_launches())


def spq_strerror(status: int) -> str:
    return _lib.load().spq_strerror(status).decode()


def build(force: bool = False) -> str:
    """Compile libspq.so (nvcc, sm_103a) in-tree."""
    from .build_ext import build as _b

    return _b(force=force)
