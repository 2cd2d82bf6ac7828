"""Continuous-batching query servers over device-resident query structures.

NativeQueryServer wraps the library's own server (spq_server_*: the scheduler below runs
as a native thread with buffers allocated once); QueryServer is the same policy written
in Python over the C ABI.

Requests (a graph id and a batch of (v1, v2) pairs) arrive at any time.  A scheduler
thread keeps up to `slots` launches in flight, each on its own CUDA stream: whenever a
slot is free it takes the oldest waiting request and every other waiting request for
the same graph (up to `max_pairs` pairs in total), copies their pairs to the device,
answers them with one spq_query launch, and copies the distances back; a completion is
detected with a CUDA event, and each request's future is resolved with its own slice of
the answers.  Work of different slots overlaps on the device, and requests that arrive
while others are on the GPU join the next free slot.

Admission: a graph is only registered (built on the device) if its table footprint fits
the device-memory budget next to the graphs already resident; in-flight pairs are also
capped (each pair holds 28 bytes of staging and sort scratch on the device).

Each pair's distance is computed independently of the other pairs of its launch (the
grouped kernel takes the same minimum over the same table entries for it), so an answer
is bit-identical whether its request ran alone or fused with others.
"""

from __future__ import annotations

import collections
import ctypes
import threading
import time
from concurrent.futures import Future

import numpy as np

from . import _lib, spq_build, spq_free, spq_query
from ._lib import SPQ_ECUDA, SPQ_EINVAL, SPQ_ENOMEM, SPQ_F32, SpqError

try:
    import torch
except Exception:  # pragma: no cover
    torch = None


class AdmissionError(RuntimeError):
    pass


class _Slot:
    def __init__(self, dev, cap):
        self.stream = torch.cuda.Stream(device=dev)
        self.d_pairs = torch.empty((cap, 2), dtype=torch.int32, device=dev)
        self.d_out = torch.empty(cap, dtype=torch.int32, device=dev)
        self.h_pairs = torch.empty((cap, 2), dtype=torch.int32).pin_memory()
        self.h_out = torch.empty(cap, dtype=torch.int32).pin_memory()
        self.done = torch.cuda.Event()
        self.busy = False
        self.reqs = []  # (request, offset, count)
        self.h = None


class _Request:
    __slots__ = ("gid", "pairs", "future", "t_arrival", "t_done")

    def __init__(self, gid, pairs, t_arrival=None):
        self.gid = gid
        self.pairs = pairs
        self.future = Future()
        self.t_arrival = time.perf_counter() if t_arrival is None else t_arrival
        self.t_done = None


class QueryServer:
    """Serve distance queries on several graphs (int32 weights) from one GPU."""

    def __init__(self, device=0, memory_budget_bytes=None, slots=4, max_pairs=1 << 20):
        if torch is None or not torch.cuda.is_available():
            raise RuntimeError("QueryServer needs a CUDA device")
        self.dev = torch.device("cuda", device)
        torch.cuda.set_device(self.dev)
        free, _ = torch.cuda.mem_get_info(self.dev)
        self.budget = int(memory_budget_bytes if memory_budget_bytes is not None else 0.9 * free)
        self.graphs = {}
        self.resident_bytes = 0
        self.max_pairs = int(max_pairs)
        self._slots = [_Slot(self.dev, self.max_pairs) for _ in range(slots)]
        self._queue = collections.deque()
        self._cv = threading.Condition()
        self._stop = False
        self.completed = []  # (latency seconds, pairs) per request
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()

    # ---- graphs ----
    def add_graph(self, gid, n, row_ptr, col, w, part, k, opts=None):
        """Build and keep the query structure of a graph, if it fits the budget."""
        h = spq_build(n, row_ptr, col, w, part, k, opts=opts)
        fp = h.stats()["footprint_bytes"]
        if self.resident_bytes + fp > self.budget:
            spq_free(h)
            raise AdmissionError(f"graph {gid}: {fp} bytes do not fit ({self.resident_bytes} of {self.budget} used)")
        self.graphs[gid] = h
        self.resident_bytes += fp
        return fp

    def add_handle(self, gid, h):
        fp = h.stats()["footprint_bytes"]
        if self.resident_bytes + fp > self.budget:
            raise AdmissionError(f"graph {gid}: {fp} bytes do not fit")
        self.graphs[gid] = h
        self.resident_bytes += fp
        return fp

    def remove_graph(self, gid):
        with self._cv:
            h = self.graphs.pop(gid)
        self.resident_bytes -= h.stats()["footprint_bytes"]
        spq_free(h)

    # ---- requests ----
    def submit(self, gid, pairs, t_arrival=None) -> Future:
        """Queue a request; the future resolves to int32[q] distances (numpy).  Latency
        is measured from t_arrival (a time.perf_counter() value; default: now)."""
        p = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        h = self.graphs.get(gid)
        if h is None:
            raise KeyError(gid)
        if p.shape[0] > self.max_pairs:
            raise AdmissionError(f"request of {p.shape[0]} pairs exceeds max_pairs={self.max_pairs}")
        if p.size and (p.min() < 0 or p.max() >= h.n):
            raise ValueError("vertex id out of range")
        r = _Request(gid, p, t_arrival)
        with self._cv:
            self._queue.append(r)
            self._cv.notify()
        return r.future

    def query(self, gid, pairs):
        return self.submit(gid, pairs).result()

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify()
        self._thread.join()
        for h in list(self.graphs.values()):
            spq_free(h)
        self.graphs.clear()

    # ---- scheduler ----
    def _launch(self, slot, reqs):
        total = 0
        slot.reqs = []
        for r in reqs:
            q = r.pairs.shape[0]
            slot.h_pairs[total:total + q].numpy()[:] = r.pairs
            slot.reqs.append((r, total, q))
            total += q
        h = self.graphs[reqs[0].gid]
        with torch.cuda.stream(slot.stream):
            slot.d_pairs[:total].copy_(slot.h_pairs[:total], non_blocking=True)
            spq_query(h, slot.d_pairs[:total], out=slot.d_out[:total], stream=slot.stream.cuda_stream)
            slot.h_out[:total].copy_(slot.d_out[:total], non_blocking=True)
            slot.done.record(slot.stream)
        slot.busy = True
        slot.h = h

    def _complete(self, slot):
        now = time.perf_counter()
        out = slot.h_out.numpy()
        for r, off, q in slot.reqs:  # (pair ids were range-checked at submission)
            r.t_done = now
            self.completed.append((now - r.t_arrival, q))
            r.future.set_result(out[off:off + q].copy())
        slot.reqs = []
        slot.busy = False

    def _take(self):
        """The oldest request and every other waiting request for its graph, up to
        max_pairs pairs (called with the lock held)."""
        first = self._queue.popleft()
        batch, total = [first], first.pairs.shape[0]
        keep = collections.deque()
        while self._queue:
            r = self._queue.popleft()
            if r.gid == first.gid and total + r.pairs.shape[0] <= self.max_pairs:
                batch.append(r)
                total += r.pairs.shape[0]
            else:
                keep.append(r)
        self._queue = keep
        return batch

    def _run(self):
        torch.cuda.set_device(self.dev)
        while True:
            progressed = False
            for s in self._slots:
                if s.busy and s.done.query():
                    self._complete(s)
                    progressed = True
            with self._cv:
                if self._stop and not self._queue and not any(s.busy for s in self._slots):
                    return
                free = [s for s in self._slots if not s.busy]
                while free and self._queue:
                    self._launch(free.pop(), self._take())
                    progressed = True
                if not progressed and not any(s.busy for s in self._slots):
                    self._cv.wait(timeout=0.01)
            if not progressed:
                time.sleep(20e-6)

    # ---- statistics ----
    def latency_stats(self):
        if not self.completed:
            return {}
        lat = np.array([c[0] for c in self.completed])
        q = np.array([c[1] for c in self.completed])
        return {"requests": int(lat.size), "pairs": int(q.sum()), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}


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
    (spq_server_*): the same fusing of waiting requests per graph and the same overlap of
    `slots` launches as QueryServer, with pinned staging, device buffers and query scratch
    allocated once, and no Python on the request path after submission."""

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
