"""The library's own continuous-batching server, spq_server_* (needs a GPU).

Answers must be bit-identical to spq_query on the request alone, whether a request ran
by itself or fused with others of its graph, for integer and float weights, with requests
submitted from several threads at once; admission (budget, duplicate ids, request size,
id range), removal of a graph with requests in flight, polling and latency statistics.
"""

import threading

import numpy as np
import pytest

from _util import build, spq

import gen

pytestmark = pytest.mark.gpu


def _server(**kw):
    from paper_1503_07192_gb300.serve import NativeQueryServer

    return NativeQueryServer(**kw)


def _graphs():
    w0 = gen.configs.delaunay_rcb(20000, 4, 10, seed=91)
    g1 = gen.delaunay(6000, seed=92, weight="f32_lognormal", scale=float(np.sqrt(6000)))
    part1, k1 = gen.rcb(g1.xy, 3)
    return [(w0.graph, build(w0.graph, w0.part, w0.k)), (g1, build(g1, part1, k1))]


def test_native_server_answers_equal_queries_alone_under_three_threads():
    m = spq()
    gs = _graphs()
    srv = _server(slots=3, max_pairs=1 << 14)
    for gid, (_, h) in enumerate(gs):
        srv.add_handle(gid, h)
    results = [[] for _ in range(3)]

    def producer(t):
        rng = np.random.default_rng(100 + t)
        for _ in range(60):
            gid = int(rng.integers(0, 2))
            q = int(rng.choice([1, 7, 300, 4096, 5000, 1 << 14]))
            p = rng.integers(0, gs[gid][0].n, size=(q, 2)).astype(np.int32)
            results[t].append((gid, p, srv.submit(gid, p)))

    ths = [threading.Thread(target=producer, args=(t,)) for t in range(3)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    n_req = 0
    for t in range(3):
        for gid, p, tk in results[t]:
            got = tk.result(timeout=120)
            ref = m.spq_query(gs[gid][1], p)
            assert got.dtype == ref.dtype and np.array_equal(got, ref)
            n_req += 1
    st = srv.latency_stats(reset=True)
    assert st["requests"] == n_req and st["pairs"] == sum(p.shape[0] for r in results for _, p, _ in r)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert srv.latency_stats()["requests"] == 0
    srv.close()


def test_native_server_admission_and_errors():
    m = spq()
    gs = _graphs()
    h0, h1 = gs[0][1], gs[1][1]
    fp0 = h0.stats()["footprint_bytes"]
    from paper_1503_07192_gb300.serve import AdmissionError

    srv = _server(slots=1, max_pairs=1000, memory_budget_bytes=fp0 + 1)
    assert srv.add_handle(0, h0) == fp0
    with pytest.raises(AdmissionError):  # over the budget
        srv.add_handle(1, h1)
    with pytest.raises(m.SpqError):  # id in use
        srv.add_handle(0, h1)
    with pytest.raises(AdmissionError):  # above max_pairs
        srv.submit(0, np.zeros((1001, 2), np.int32))
    with pytest.raises(ValueError):
        srv.submit(0, np.array([[0, gs[0][0].n]], np.int32))
    with pytest.raises(KeyError):
        srv.submit(5, np.zeros((1, 2), np.int32))
    assert srv.submit(0, np.zeros((0, 2), np.int32)).result().shape == (0,)
    p = np.array([[0, 1], [2, 3]], np.int32)
    tk = srv.submit(0, p)
    while not tk.done():
        pass
    assert np.array_equal(tk.result(), m.spq_query(h0, p))
    srv.close(free_graphs=False)
    h0.free()
    h1.free()


def test_native_server_remove_graph_waits_for_its_requests():
    m = spq()
    gs = _graphs()
    srv = _server(slots=2, max_pairs=1 << 16)
    srv.add_handle(0, gs[0][1])
    srv.add_handle(1, gs[1][1])
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(40):
        gid = i % 2
        p = rng.integers(0, gs[gid][0].n, size=(20000, 2)).astype(np.int32)
        reqs.append((gid, p, srv.submit(gid, p)))
    srv.remove_graph(0, free=False)  # returns only once graph 0's requests are answered
    for gid, p, tk in reqs:
        if gid == 0:
            assert tk.done()
    with pytest.raises(KeyError):
        srv.submit(0, reqs[0][1])
    for gid, p, tk in reqs:
        assert np.array_equal(tk.result(timeout=120), m.spq_query(gs[gid][1], p))
    srv.close()
    gs[0][1].free()
