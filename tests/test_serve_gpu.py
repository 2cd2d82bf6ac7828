"""The continuous-batching server (needs a GPU).

Requests of 1..4096 pairs on several resident graphs are submitted from three threads
at once, so that requests are fused into shared launches and several launches overlap
on different streams.  Every answer must equal the answer of the same request run
alone (bit-identical: integer distances) and the oracle's distances.  Admission limits
(device-memory budget, request size, vertex range) raise instead of queueing.
"""

import threading

import numpy as np
import pytest

from _util import oracle_i32, spq, torch_dev

import gen
import oracle

pytestmark = pytest.mark.gpu


def _graphs():
    ws = [gen.configs.grid64(q=10),
          gen.configs.delaunay_rcb(8000, 3, 10, seed=71),
          gen.configs.batch_instances(count=2, seed=73, q_per=10, n_lo=2000, n_hi=6000, leaf_lo=100,
                                      leaf_hi=400)[1]]
    return {i: w for i, w in enumerate(ws)}


def test_results_are_the_same_alone_and_in_the_mix():
    m = spq()
    from paper_1503_07192_gb300.serve import QueryServer

    torch, dev = torch_dev()
    ws = _graphs()
    srv = QueryServer(device=0, slots=4, max_pairs=20000)
    for gid, w in ws.items():
        srv.add_graph(gid, w.graph.n, w.graph.row_ptr, w.graph.col, w.graph.w, w.part, w.k)
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(240):
        gid = int(rng.integers(0, len(ws)))
        q = int(rng.integers(1, 4097))
        reqs.append((gid, rng.integers(0, ws[gid].graph.n, size=(q, 2)).astype(np.int32)))
    futs = [None] * len(reqs)

    def producer(lo):
        for i in range(lo, len(reqs), 3):
            futs[i] = srv.submit(*reqs[i])

    ths = [threading.Thread(target=producer, args=(t,)) for t in range(3)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    results = [f.result(timeout=120) for f in futs]
    for i, ((gid, p), got) in enumerate(zip(reqs, results)):
        alone = m.spq_query(srv.graphs[gid], p)
        assert np.array_equal(got, alone), i
        if i < 40:
            g = ws[gid].graph
            ref = oracle_i32(oracle.pairs_dist(g.row_ptr, g.col, g.w, p[:25]))
            assert np.array_equal(got[:25].astype(np.int64), ref), i
    st = srv.latency_stats()
    assert st["requests"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_admission_limits():
    from paper_1503_07192_gb300.serve import AdmissionError, QueryServer

    w = gen.configs.grid64(q=10)
    small = QueryServer(device=0, memory_budget_bytes=1 << 10, slots=1, max_pairs=100)
    with pytest.raises(AdmissionError):
        small.add_graph(0, w.graph.n, w.graph.row_ptr, w.graph.col, w.graph.w, w.part, w.k)
    small.close()
    srv = QueryServer(device=0, slots=1, max_pairs=100)
    srv.add_graph(0, w.graph.n, w.graph.row_ptr, w.graph.col, w.graph.w, w.part, w.k)
    with pytest.raises(AdmissionError):
        srv.submit(0, np.zeros((101, 2), np.int32))
    with pytest.raises(ValueError):
        srv.submit(0, np.array([[0, w.graph.n]], np.int32))
    with pytest.raises(KeyError):
        srv.submit(7, np.zeros((1, 2), np.int32))
    assert srv.query(0, np.array([[0, 0]], np.int32))[0] == 0
    srv.close()
