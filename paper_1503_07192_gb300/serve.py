"""Continuous-batching query server over device-resident query structures.

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
import threading
import time
from concurrent.futures import Future

import numpy as np

from . import spq_build, spq_free, spq_query

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
