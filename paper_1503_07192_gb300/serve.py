"""Continuous-batching query server over device-resident query structures.

NativeQueryServer wraps the library's own server (spq_server_*): a native scheduler
thread with buffers allocated once.  Requests (a graph id and a batch of (v1, v2) pairs)
arrive at any time.  The scheduler keeps up to `slots` launches in flight, each on its
own CUDA stream: whenever a slot is free it takes the oldest waiting request and every
other waiting request for the same graph (up to `max_pairs` pairs in total), copies their
pairs to the device, answers them with one launch, and copies the distances back; a
completion is detected with a CUDA event, and each request's ticket gets its own slice of
the answers.  Work of different slots overlaps on the device, and requests that arrive
while others are on the GPU join the next free slot.

Admission: a graph is only registered if its table footprint fits the device-memory
budget next to the graphs already resident; a request may hold at most `max_pairs` pairs.

Each pair's distance is computed independently of the other pairs of its launch (the
grouped kernel takes the same minimum over the same table entries for it), so an answer
is bit-identical whether its request ran alone or fused with others.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib, spq_build, spq_free
from ._lib import SPQ_ECUDA, SPQ_EINVAL, SPQ_ENOMEM, SPQ_F32, SpqError


class AdmissionError(RuntimeError):
    pass


class NativeTicket:
    """One request queued in a NativeQueryServer; result() blocks until its answers are in."""

    __slots__ = ("_srv", "ticket", "out", "_done")

    def __init__(self, srv, ticket, out):
        self._srv, self.ticket, self.out, self._done = srv, ticket, out, False

    def done(self) -> bool:
        if not self._done:
            v = _lib.load().spq_server_poll(self._srv._s, self.ticket)
            if v < 0:
                raise SpqError(SPQ_ECUDA, "spq_server_poll")
            self._done = v == 1
        return self._done

    def result(self, timeout=None):
        if not self._done:
            st = _lib.load().spq_server_wait(self._srv._s, self.ticket, 1e9 if timeout is None else float(timeout))
            if st:
                raise SpqError(st, "spq_server_wait")
            self._done = True
        return self.out


class NativeQueryServer:
    """The continuous-batching server run by the library's own scheduler thread
    (spq_server_*): waiting requests fused per graph, `slots` launches overlapped, pinned
    staging, device buffers and query scratch allocated once, and no Python on the
    request path after submission."""

    def __init__(self, device=0, memory_budget_bytes=None, slots=4, max_pairs=1 << 20):
        lib = _lib.load()
        s = ctypes.c_void_p()
        st = lib.spq_server_create(int(device), int(slots), int(max_pairs),
                                   int(memory_budget_bytes or 0), ctypes.byref(s))
        if st:
            raise SpqError(st, "spq_server_create")
        self._s = s
        self.max_pairs = int(max_pairs)
        self.graphs = {}
        self.resident_bytes = 0

    def add_graph(self, gid, n, row_ptr, col, w, part, k, opts=None):
        """Build a graph's query structure and admit it, if it fits the budget."""
        h = spq_build(n, row_ptr, col, w, part, k, opts=opts)
        try:
            return self.add_handle(gid, h)
        except AdmissionError:
            spq_free(h)
            raise

    def add_handle(self, gid, h):
        """Admit a built handle; the server keeps it alive until remove_graph / close."""
        st = _lib.load().spq_server_add_graph(self._s, int(gid), h.ptr)
        if st == SPQ_ENOMEM:
            raise AdmissionError(f"graph {gid}: {h.stats()['footprint_bytes']} bytes do not fit")
        if st:
            raise SpqError(st, "spq_server_add_graph")
        self.graphs[gid] = h
        fp = h.stats()["footprint_bytes"]
        self.resident_bytes += fp
        return fp

    def remove_graph(self, gid, free=True):
        st = _lib.load().spq_server_remove_graph(self._s, int(gid))
        if st:
            raise SpqError(st, "spq_server_remove_graph")
        h = self.graphs.pop(gid)
        self.resident_bytes -= h.stats()["footprint_bytes"]
        if free:
            spq_free(h)

    def submit(self, gid, pairs) -> NativeTicket:
        """Queue a request (int32[q, 2] host pairs); its ticket's result() is int32[q]
        (float32 for float-weight graphs).  Thread-safe."""
        p = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        h = self.graphs.get(gid)
        if h is None:
            raise KeyError(gid)
        if p.shape[0] > self.max_pairs:
            raise AdmissionError(f"request of {p.shape[0]} pairs exceeds max_pairs={self.max_pairs}")
        out = np.empty(p.shape[0], np.float32 if h.wt == SPQ_F32 else np.int32)
        if p.shape[0] == 0:
            t = NativeTicket(self, 0, out)
            t._done = True
            return t
        tk = ctypes.c_int64()
        st = _lib.load().spq_server_submit(self._s, int(gid), ctypes.c_void_p(p.ctypes.data), p.shape[0],
                                           ctypes.c_void_p(out.ctypes.data), ctypes.byref(tk))
        if st == SPQ_EINVAL:
            raise ValueError("vertex id out of range")
        if st:
            raise SpqError(st, "spq_server_submit")
        return NativeTicket(self, tk.value, out)

    def query(self, gid, pairs):
        return self.submit(gid, pairs).result()

    def latency_stats(self, reset=False):
        """p50 / p99 latency (ms, submission to answer) and the requests and pairs answered."""
        p50, p99 = ctypes.c_double(), ctypes.c_double()
        nr, npairs = ctypes.c_int64(), ctypes.c_int64()
        st = _lib.load().spq_server_stats(self._s, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(nr),
                                          ctypes.byref(npairs), int(bool(reset)))
        if st:
            raise SpqError(st, "spq_server_stats")
        return {"requests": nr.value, "pairs": npairs.value, "p50_ms": p50.value, "p99_ms": p99.value}

    def close(self, free_graphs=True):
        if self._s:
            _lib.load().spq_server_destroy(self._s)
            self._s = None
        if free_graphs:
            for h in self.graphs.values():
                spq_free(h)
        self.graphs.clear()

    def __del__(self):
        try:
            if self._s:
                _lib.load().spq_server_destroy(self._s)
                self._s = None
        except Exception:
            pass
