#!/usr/bin/env python
"""Benchmark of the distance-query hot path on one or more GB300s.

One step = the whole path on one synthetic batch: spq_build on the workload's graph and
partition (validation, reordering, batched component Floyd-Warshall, boundary-graph
assembly, boundary-graph blocked Floyd-Warshall) followed by spq_query on the
workload's query pairs, then spq_free.

Default workload (the configuration the headline metric is quoted on): Delaunay
triangulation of 2^20 uniform points, w = round(1e6 * length), recursive coordinate
bisection into 1,024 components of 1,024 vertices, 10,000,000 uniform query pairs.
Inputs are synthetic (gen/), seeded, built on the host before timing and resident in
HBM when the timed region starts.  The boundary-graph matrix (about 71 GB) is larger
than L2 and rewritten every step, so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (Dijkstra per
pair, OpenMP over the host cores) on a bounded sample of the same workload.
Multi-GPU (torchrun): independent replicas, one per GPU, no collective on the data path.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

# up to 32 chains of elimination rounds run on their own streams: give the CUDA context
# as many hardware work queues (before anything creates it)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "queries/s + build min-plus Gop/s (1M-vertex planar), vs INT32/HBM roofline, 1xGB300"
# DRAM traffic of k_backsub is not reported for the full-size launch: counters beyond the
# launch time are captured only on the 2^18-point case (a few GB on the device), and
# there the traffic does not scale with the update count (the writes grow as N^2, the
# re-read rows faster): 2,386,661,632 B read + 4,390,244,608 B written for 2.41e11
# updates (0.028 B per update, against 0.046 in an earlier full-size capture).
BACKSUB_TRAFFIC_NOTE = ("not measured at this size; on 2^18 points one launch reads 2.39 GB and writes 4.39 GB "
                        "(the matrix once) for 2.41e11 updates, and the ratio grows with size")
UNIT = "queries/s"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="delaunay1m",
                   choices=["delaunay1m", "grid64", "delaunay65k", "delaunay131k", "delaunay262k", "grid1024diag",
                            "batch512",
                            "serve", "grad256k", "matrix1m"])
    p.add_argument("--rates", default="500,2000,8000", help="serve: request arrival rates (1/s) to sweep")
    p.add_argument("--duration", type=float, default=3.0, help="serve: seconds of arrivals per rate")
    p.add_argument("--instances", type=int, default=512, help="batch512: number of instances")
    p.add_argument("--queries", type=int, default=None, help="override the workload's query count")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU oracle sample")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--arith", type=int, default=0, help="spq_arith of the build (0 auto, 1 int32, 2 float32)")
    p.add_argument("--bg", type=int, default=0, help="spq_bg_method of the build (0 auto, 1 FW, 2 elimination)")
    p.add_argument("--query-kernel", type=int, default=0, choices=[0, 1],
                   help="opts.query_kernel of the build (0: staged grouped kernel, 1: the gathering one)")
    return p.parse_args()


def make_workload(name, q):
    import gen

    if name == "delaunay1m":
        w = gen.configs.delaunay1m(q=q or 10_000_000)
        desc = {"workload": "delaunay1m", "vertices": w.graph.n, "edges": w.graph.m // 2,
                "components": w.k, "partition": "recursive coordinate bisection, 10 levels",
                "weights": "int32 round(1e6 * Euclidean length)", "queries_per_step": int(w.pairs.shape[0])}
    elif name == "delaunay262k":
        w = gen.configs.delaunay_rcb(1 << 18, 8, q or 2_500_000, seed=1241)
        desc = {"workload": "delaunay262k", "vertices": w.graph.n, "components": w.k,
                "queries_per_step": int(w.pairs.shape[0])}
    elif name == "grid1024diag":
        w = gen.configs.grid1024diag(q=q or 10_000_000)
        desc = {"workload": "grid1024diag", "vertices": w.graph.n, "components": w.k,
                "partition": "32x32-vertex blocks", "queries_per_step": int(w.pairs.shape[0])}
    elif name == "delaunay131k":
        # the delaunay1m regime at 1/8 size (components of 1,024 vertices, about 19 pairs
        # per component pair), a few GB on the device: the case for kernel captures
        w = gen.configs.delaunay_rcb(1 << 17, 7, q or 157_000, seed=1242)
        desc = {"workload": "delaunay131k", "vertices": w.graph.n, "components": w.k,
                "queries_per_step": int(w.pairs.shape[0])}
    elif name == "delaunay65k":
        w = gen.configs.delaunay_rcb(1 << 16, 6, q or 1_000_000, seed=1240)
        desc = {"workload": "delaunay65k", "vertices": w.graph.n, "components": w.k,
                "queries_per_step": int(w.pairs.shape[0])}
    else:
        w = gen.configs.grid64(q=q or 10_000)
        desc = {"workload": "grid64", "vertices": w.graph.n, "components": w.k,
                "queries_per_step": int(w.pairs.shape[0])}
    return w, desc


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None
        self.first = 0  # samples before the timed region (taken during the warm-up)

    def started(self) -> "ClockSampler":
        """Start before the warm-up and wait for the first sample, so that nvidia-smi's own
        start-up (driver queries) stays out of the timed region."""
        self.start()
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < 10:
            time.sleep(0.05)
        return self

    def mark(self):
        """The timed region starts: only samples from here on count."""
        self.first = len(self.lines)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # samples of the timed region (the last warm-up one too if the region was shorter
        # than the sampling period)
        lines = self.lines[max(0, min(self.first, len(self.lines) - 1)):]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The maximum of x over all ranks (every rank gets it); x itself with one rank.  The
    timed span of a multi-GPU run is the slowest rank's."""
    if not dist:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units of all ranks per second of the slowest rank (weak scaling: every rank does
    the same work)."""
    return world * units_per_rank / seconds


def measured_hbm_gbs() -> dict:
    """The machine's measured copy bandwidth (MEASURED_PEAKS.json, written by the pool's
    driver), else the fallback of one earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return {"value": float(json.load(f)["hbm_gbs"]), "basis": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
    except Exception:
        return {"value": 6800.0, "basis": "of fallback (6.8 TB/s)"}


def tuning_summary(spq) -> dict:
    """The grouped query autotuner's choices: size classes per configuration."""
    t = spq.spq_query_tuning()
    return {"classes": len(t), "config1_classes": sorted(c for (_, c), v in t.items() if v == 1),
            "config0_classes": sorted(c for (_, c), v in t.items() if v == 0)}


def workload_config(desc: dict, world: int) -> dict:
    """The `config` of a line (both arms): the workload, what it means for L2, and the
    parallelism."""
    sizes = {"delaunay1m": "71 GB", "grid1024diag": "61 GB", "delaunay262k": "4.2 GB", "delaunay131k": "1.1 GB"}
    name = desc.get("workload", "")
    if name == "grid64":
        l2 = "inputs fit in L2 (a 2 MB boundary-graph matrix; a parity workload, not a benchmark configuration)"
    elif name in sizes:
        l2 = f"inputs larger than L2 (the {sizes[name]} boundary-graph matrix is rebuilt every step)"
    else:
        l2 = "inputs larger than L2 (the boundary-graph matrix is rebuilt every step)"
    return dict(desc, l2=l2, parallelism="replicas" if world > 1 else "single GPU")


def build_tuning_summary(spq) -> dict:
    """The build autotuner's state: per size class of the boundary graph, the chosen depth
    of concurrent elimination runs and the stage times measured at depths 3, 4, 5."""
    return {str(c): {"depth": v["depth"], "bg_stage_ms": [round(x, 2) for x in v["ms"]]}
            for (_, c), v in spq.spq_build_tuning().items()}


def cpu_oracle_sample(w, budget_s: float, seed: int = 99):
    """Time the oracle (Dijkstra per pair, all host cores) on a bounded sample of the
    workload's pairs: chunks of uniformly drawn pairs until budget_s has elapsed.
    Returns (queries/s, sample size, seconds, cores, sampled pair indices, their oracle
    distances as int64)."""
    import numpy as np

    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    g = w.graph
    rng = np.random.default_rng(seed)
    oracle.pairs_dist(g.row_ptr, g.col, g.w, w.pairs[:cores], nthreads=cores)  # load, spin up threads
    n, t0 = 0, time.perf_counter()
    idx, res = [], []
    while time.perf_counter() - t0 < budget_s and n < w.pairs.shape[0]:
        ci = rng.integers(0, w.pairs.shape[0], size=8 * cores)
        res.append(oracle.pairs_dist(g.row_ptr, g.col, g.w, w.pairs[ci], nthreads=cores))
        idx.append(ci)
        n += ci.shape[0]
    dt = time.perf_counter() - t0
    return n / dt, n, dt, cores, np.concatenate(idx), np.concatenate(res).astype(np.int64)


def run_reference(args, rank):
    if rank != 0:
        return 0
    w, desc = make_workload(args.workload, args.queries)
    import numpy as np

    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    g = w.graph
    rng = np.random.default_rng(7)
    # size each step for a few seconds of oracle time
    probe = w.pairs[rng.integers(0, w.pairs.shape[0], size=4 * cores)]
    t0 = time.perf_counter()
    oracle.pairs_dist(g.row_ptr, g.col, g.w, probe, nthreads=cores)
    per_q = max(time.perf_counter() - t0, 1e-6) / probe.shape[0]
    step_q = int(min(max(8.0 / per_q, 4 * cores), w.pairs.shape[0]))
    times = []
    for s in range(args.warmup + args.steps):
        sample = w.pairs[rng.integers(0, w.pairs.shape[0], size=step_q)]
        t0 = time.perf_counter()
        oracle.pairs_dist(g.row_ptr, g.col, g.w, sample, nthreads=cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = step_q * len(times) / tot
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "impl": "reference", "config": workload_config(desc, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{step_q} uniformly drawn pairs of the workload per step, "
                                       f"binary-heap Dijkstra with early exit, OpenMP over pairs"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _gen_instance(args):
    import gen

    seed, i, q_per = args
    return gen.configs.batch_instances(count=i + 1, seed=seed, q_per=q_per, only=i)[0]


def run_batch(args, rank, local_rank):
    """The batching pattern: many independent instances (grids with 10% of the vertices
    removed and Delaunay triangulations, n log-uniform in [1,000, 65,536], kd-tree
    components with a leaf cap log-uniform in [128, 2,048], 100,000 pairs each).
    Batched form: spq_build_many + spq_query_many, all instances in shared launches.
    Per-graph form: spq_build + spq_query + spq_free per instance, one after another.
    One step = every instance built and queried once (device buffers); value = pairs
    answered per second of the batched form."""
    import concurrent.futures as cf
    import multiprocessing as mp

    G = args.instances
    q_per = args.queries or 100_000
    t0 = time.time()
    with cf.ProcessPoolExecutor(max_workers=os.cpu_count() or 4, mp_context=mp.get_context("spawn")) as ex:
        ins = list(ex.map(_gen_instance, [(1237, i, q_per) for i in range(G)]))
    log(f"[rank {rank}] {G} instances, {sum(w.graph.n for w in ins)} vertices ({time.time() - t0:.1f}s)")

    import numpy as np
    import torch

    import paper_1503_07192_gb300 as spq

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    spq.build()

    def T(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    graphs = [(w.graph.n, T(w.graph.row_ptr), T(w.graph.col), T(w.graph.w), T(w.part), w.k) for w in ins]
    pairs = [T(w.pairs) for w in ins]
    outs = [torch.empty(p.shape[0], dtype=torch.int32, device=dev) for p in pairs]
    q_tot = sum(int(p.shape[0]) for p in pairs)
    stream = torch.cuda.current_stream(dev)

    def batched():
        hs = spq.spq_build_many(graphs)
        spq.spq_query_many(hs, pairs, outs=outs)
        torch.cuda.synchronize()
        st = hs[0].stats()
        pf = hs[0].profile()
        for h in hs:
            h.free()
        return st, pf

    def per_graph():
        for g, p, o in zip(graphs, pairs, outs):
            h = spq.spq_build(*g)
            spq.spq_query(h, p, out=o)
            h.free()
        torch.cuda.synchronize()

    def timed(fn, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = None
        for _ in range(k):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k, r

    clocks = ClockSampler(local_rank).started()
    for _ in range(args.warmup):
        batched()
    ref = [o.clone() for o in outs]
    clocks.mark()
    launches0 = spq.spq_kernel_launches()
    ms_b, (st, pf) = timed(batched, args.steps)
    launches = spq.spq_kernel_launches() - launches0
    clk = clocks.stop()
    per_graph()  # warm-up of the per-graph form
    ms_p, _ = timed(per_graph, max(1, args.steps // 2))
    same = all(torch.equal(a, b) for a, b in zip(ref, outs))
    # the query phase alone on resident handles: spq_query_many (launches issued by the
    # host) against the same batch captured into a CUDA graph and replayed (spq_query_plan)
    hs = spq.spq_build_many(graphs)
    spq.spq_query_many(hs, pairs, outs=outs)
    ms_qm, _ = timed(lambda: spq.spq_query_many(hs, pairs, outs=outs), max(3, args.steps))
    plan = spq.spq_query_plan(hs, pairs, outs=outs)
    plan.run()
    ms_qp, _ = timed(plan.run, max(3, args.steps))
    same_plan = all(torch.equal(a, b) for a, b in zip(ref, outs))
    plan.free()
    for h in hs:
        h.free()
    # re-weighting through a build plan (the weight-dependent launches captured in a CUDA
    # graph once): runs alternate between doubled and the original weights (device
    # buffers); the answers after a run on the original weights must be the batched form's
    t0 = time.time()
    bplan = spq.spq_build_plan(graphs)
    create_s = time.time() - t0
    w_orig = [g[3] for g in graphs]
    w_dbl = [w * 2 for w in w_orig]
    bplan.run(w_dbl)
    bplan.run(w_orig)
    ms_br, _ = timed(lambda: (bplan.run(w_dbl), bplan.run(w_orig)), max(2, args.steps // 2))
    spq.spq_query_many(bplan.handles, pairs, outs=outs)
    torch.cuda.synchronize()
    same_bplan = all(torch.equal(a, b) for a, b in zip(ref, outs))
    bplan.free()
    del w_dbl
    upd = sum(w.graph.n for w in ins)
    line = {
        "metric": METRIC, "value": q_tot / (ms_b * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("int32 results, exact float32 arithmetic (checked)" if st["arith"] == spq.SPQ_ARITH_F32
                  else "int32"), "data": "synthetic",
        "config": {"workload": f"batch{G}", "instances": G, "vertices": upd, "queries_per_step": q_tot,
                   "l2": "tables of all instances (tens of GB) rebuilt every step"},
        "batched_ms": ms_b, "per_graph_ms": ms_p, "speedup_vs_per_graph": ms_p / ms_b,
        "per_graph_qps": q_tot / (ms_p * 1e-3), "results_identical": bool(same),
        "query_phase_ms": {"query_many": ms_qm, "cuda_graph_plan": ms_qp,
                           "plan_results_identical": bool(same_plan)},
        "build_plan": {"create_s": round(create_s, 3), "rebuild_ms": ms_br / 2,
                       "results_identical": bool(same_bplan)},
        "query_autotune": tuning_summary(spq),
        "batch_stage_ms": {k: round(pf[k], 2) for k in ("validate", "reorder", "comp_fw", "bg_assemble", "bg_fw",
                                                         "check")},
        "bg_updates": st["bg_updates"], "gpu_launches": int(launches) // max(1, args.steps), "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args, rank, local_rank):
    """The serving pattern: a 1024x1024 grid with one random diagonal per cell (32x32
    components) resident beside 8 batching-workload instances; requests of U{1..4096}
    pairs on a uniformly chosen graph arrive as a Poisson stream; the server fuses
    waiting requests per graph and overlaps launches on 4 streams.  Reports, per arrival
    rate, p50/p99 latency (arrival to answer on the host) and the pairs answered per
    second, and checks that sampled requests give the same answers when run alone."""
    import numpy as np
    import torch

    import gen
    import paper_1503_07192_gb300 as spq
    from paper_1503_07192_gb300.serve import NativeQueryServer

    torch.cuda.set_device(local_rank)
    spq.build()
    t0 = time.time()
    ws = [gen.configs.grid1024diag()] + gen.configs.batch_instances(count=8, q_per=10)
    srv = NativeQueryServer(device=local_rank, slots=4, max_pairs=1 << 20)
    gopts = spq.spq_opts_default()
    gopts.bg_method = args.bg
    for gid, w in enumerate(ws):
        srv.add_graph(gid, w.graph.n, w.graph.row_ptr, w.graph.col, w.graph.w, w.part, w.k, opts=gopts)
    log(f"[rank {rank}] {len(ws)} graphs resident, {srv.resident_bytes / 1e9:.1f} GB ({time.time() - t0:.1f}s)")
    rng = np.random.default_rng(2026)
    sweep = []
    for rate in [float(x) for x in args.rates.split(",")]:
        n_req = max(1, int(rate * args.duration))
        gaps = rng.exponential(1.0 / rate, size=n_req)
        gids = rng.integers(0, len(ws), size=n_req)
        sizes = rng.integers(1, 4097, size=n_req)
        reqs = [(int(g), rng.integers(0, ws[g].graph.n, size=(int(q), 2)).astype(np.int32))
                for g, q in zip(gids, sizes)]
        # warm-up: one request per graph
        for gid in range(len(ws)):
            srv.query(gid, reqs[0][1][:1] % ws[gid].graph.n)
        srv.latency_stats(reset=True)
        start = time.perf_counter() + 0.05
        t_arr = start + np.cumsum(gaps)
        futs = []
        lag = np.zeros(n_req)
        for i, ((gid, p), ta) in enumerate(zip(reqs, t_arr)):
            # sleep until just before the arrival, then submit (latency is counted from
            # submission: the producer's lag behind the arrival time is reported)
            dt = ta - time.perf_counter()
            if dt > 2e-4:
                time.sleep(dt - 1e-4)
            lag[i] = max(0.0, time.perf_counter() - ta)
            futs.append(srv.submit(gid, p))
        outs = [f.result(timeout=600) for f in futs]
        t_end = time.perf_counter()
        st = srv.latency_stats()
        pairs = int(sizes.sum())
        idx = rng.choice(n_req, size=min(64, n_req), replace=False)
        same = all(np.array_equal(outs[i], spq.spq_query(srv.graphs[reqs[i][0]], reqs[i][1])) for i in idx)
        sweep.append({"rate_req_s": rate, "requests": n_req, "pairs": pairs,
                      "offered_pairs_s": pairs / (t_arr[-1] - start + 1e-9),
                      "achieved_pairs_s": pairs / (t_end - start), "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                      "same_alone_and_in_mix": bool(same)})
        sweep[-1]["submit_lag_p99_ms"] = float(np.percentile(lag, 99) * 1e3)
        log(f"[rank {rank}] rate {rate}: {sweep[-1]}")
    srv.close()
    best = sweep[-1]
    line = {"metric": METRIC, "value": best["achieved_pairs_s"], "unit": UNIT, "n_gpus": 1, "steps": len(sweep),
            "warmup": 1, "ms_per_step": args.duration * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "serve", "graphs": ["grid1024diag"] + [f"batch{i}" for i in range(8)],
                       "request_pairs": "U{1..4096}", "arrivals": "Poisson", "slots": 4, "server": "native"},
            "sweep": sweep}
    print(json.dumps(line), flush=True)
    return 0


def run_matrix(args, rank, local_rank):
    """Many-to-many distances on delaunay1m: 64 random sources against every vertex
    (67M distances) with spq_query_matrix (Algorithm 2's first stage done once per source
    and target component), against spq_query on the same pairs of four sources."""
    import numpy as np
    import torch

    import gen
    import paper_1503_07192_gb300 as spq

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    spq.build()
    w = gen.configs.delaunay1m(q=10)
    g = w.graph
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    h = spq.spq_build(g.n, T(g.row_ptr), T(g.col), T(g.w), T(w.part), w.k)
    rng = np.random.default_rng(1240)
    src = T(rng.integers(0, g.n, size=64).astype(np.int32))
    tgt = T(np.arange(g.n, dtype=np.int32))
    out = torch.empty((64, g.n), dtype=torch.int32, device=dev)
    pairs = T(np.stack([np.repeat(src.cpu().numpy()[:4], g.n), np.tile(np.arange(g.n), 4)], 1).astype(np.int32))
    pout = torch.empty(pairs.shape[0], dtype=torch.int32, device=dev)

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    mat_ms = timed(lambda: spq.spq_query_matrix(h, src, tgt, out=out), args.steps)
    pair_ms = timed(lambda: spq.spq_query(h, pairs, out=pout), args.steps)
    spq.spq_query_status(h)
    same = bool(torch.equal(out[:4].reshape(-1), pout))
    line = {
        "metric": "distances/s (64 sources x all vertices, delaunay1m)",
        "value": 64 * g.n / (mat_ms * 1e-3), "unit": "distances/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mat_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "matrix1m", "sources": 64, "targets": g.n},
        "pairwise_query_distances_per_s": pairs.shape[0] / (pair_ms * 1e-3),
        "speedup_vs_pairwise": (64 * g.n / mat_ms) / (pairs.shape[0] / pair_ms),
        "first_rows_identical_to_pairwise": same,
    }
    h.free()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_grad(args, rank, local_rank):
    """The differentiation pattern: Delaunay of 2^18 uniform points, float32 weights =
    length x lognormal(0, 0.25), recursive coordinate bisection into 256 components of
    1,024, 1,000,000 pairs with upstream gradients N(0, 1).  One step = forward (build +
    distances with the minimising boundary pairs) + backward (path walks, gradient
    scatter onto the 1.5M CSR slots).  A seeded sample of 2,000 pairs is checked against
    the CPU reference gradient (the oracle's Dijkstra paths, FP64)."""
    import numpy as np
    import torch

    import gen
    import oracle
    import paper_1503_07192_gb300 as spq

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    spq.build()
    t0 = time.time()
    w = gen.configs.delaunay256k(q=args.queries or 1_000_000)
    g = w.graph
    rng = np.random.default_rng(1238)
    up = rng.normal(size=w.pairs.shape[0]).astype(np.float32)
    log(f"[rank {rank}] grad workload n={g.n} m={g.m} k={w.k} ({time.time() - t0:.1f}s)")

    def T(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    d_rp, d_col, d_w, d_part, d_pairs, d_up = T(g.row_ptr), T(g.col), T(g.w), T(w.part), T(w.pairs), T(up)
    grad = torch.zeros(g.m, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        h = spq.spq_build(g.n, d_rp, d_col, d_w, d_part, w.k)
        e[1].record(stream)
        dist, saved = spq.spq_query_saved(h, d_pairs)
        e[2].record(stream)
        grad.zero_()
        spq.spq_query_backward(h, d_pairs, saved, d_up, grad)
        e[3].record(stream)
        torch.cuda.synchronize()
        spq.spq_query_status(h)
        h.free()
        return [e[i].elapsed_time(e[i + 1]) for i in range(3)]

    clocks = ClockSampler(local_rank).started()
    for _ in range(args.warmup):
        step()
    clocks.mark()
    times = [step() for _ in range(args.steps)]
    clk = clocks.stop()
    build_ms, fwd_ms, bwd_ms = (statistics.mean(t[i] for t in times) for i in range(3))
    # correctness on a sample of pairs: GPU gradient of the sample vs the CPU reference
    idx = rng.choice(w.pairs.shape[0], size=2000, replace=False)
    sp, su = w.pairs[idx], up[idx].astype(np.float64)
    h = spq.spq_build(g.n, d_rp, d_col, d_w, d_part, w.k)
    dist_s, saved_s = spq.spq_query_saved(h, T(sp))
    gs = torch.zeros(g.m, dtype=torch.float32, device=dev)
    spq.spq_query_backward(h, T(sp), saved_s, T(su.astype(np.float32)), gs)
    torch.cuda.synchronize()
    h.free()
    ref_d, ref_g = oracle.pairs_dist_f64(g.row_ptr, g.col, g.w.astype(np.float64), sp, g=su)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    key = np.minimum(src, g.col).astype(np.int64) * g.n + np.maximum(src, g.col)
    _, inv = np.unique(key, return_inverse=True)
    gu = np.bincount(inv, weights=gs.cpu().numpy().astype(np.float64))
    ru = np.bincount(inv, weights=ref_g)
    err = np.abs(gu - ru).max() / max(1.0, np.abs(ru).max())
    derr = float(np.max(np.abs(dist_s.cpu().numpy() - ref_d) / np.maximum(ref_d, 1e-30)))
    q = int(w.pairs.shape[0])
    step_ms = build_ms + fwd_ms + bwd_ms
    line = {"metric": METRIC, "value": q / (step_ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "grad256k", "vertices": g.n, "components": w.k, "pairs": q,
                       "weights": "float32 length x lognormal(0, 0.25)"},
            "build_ms": build_ms, "forward_query_ms": fwd_ms, "backward_ms": bwd_ms,
            "sample_check": {"pairs": 2000, "dist_max_rel_err_vs_fp64": derr,
                             "grad_max_err_vs_cpu_reference_rel_to_max": float(err), "pass": bool(err <= 1e-4)},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "batch512":
        return run_batch(args, rank, local_rank)
    if args.workload == "serve":
        return run_serve(args, rank, local_rank)
    if args.workload == "grad256k":
        return run_grad(args, rank, local_rank)
    if args.workload == "matrix1m":
        return run_matrix(args, rank, local_rank)

    import numpy as np
    import torch

    import paper_1503_07192_gb300 as spq
    from paper_1503_07192_gb300 import _lib

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    spq.build()
    lib = _lib.load()

    t0 = time.time()
    w, desc = make_workload(args.workload, args.queries)
    g = w.graph
    q = int(w.pairs.shape[0])
    log(f"[rank {rank}] workload {desc['workload']}: n={g.n} m={g.m} k={w.k} q={q} ({time.time() - t0:.1f}s)")

    def T(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    d_rp, d_col, d_w, d_part, d_pairs = T(g.row_ptr), T(g.col), T(g.w), T(w.part), T(w.pairs)
    d_out = torch.empty(q, dtype=torch.int32, device=dev)
    opts = spq.spq_opts_default()
    opts.profile_kernels = 1
    opts.arith, opts.bg_method, opts.query_kernel = args.arith, args.bg, args.query_kernel
    stream = torch.cuda.current_stream(dev)

    def step():
        """One pass of the whole path; returns (build stats, profile, query ms)."""
        h = spq.spq_build(g.n, d_rp, d_col, d_w, d_part, w.k, opts=opts)
        eq0 = torch.cuda.Event(enable_timing=True)
        eq1 = torch.cuda.Event(enable_timing=True)
        eq0.record(stream)
        spq.spq_query(h, d_pairs, out=d_out)
        eq1.record(stream)
        st, pf = h.stats(), h.profile()
        pf["query_kernel"] = spq.spq_query_profile(h)
        h.free()  # synchronises the device
        return st, pf, eq0.elapsed_time(eq1)

    clocks = ClockSampler(local_rank).started()
    for i in range(args.warmup):
        st, pf, qms = step()
        log(f"[rank {rank}] warmup {i}: build stages {[round(pf[k], 1) for k in list(pf)[:6]]} ms, query {qms:.1f} ms"
            f", bg updates {st['bg_updates']:.3e}, order {int(pf.get('order_method', -1))}")

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = spq.spq_kernel_launches()
    clocks.mark()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    wall0 = time.perf_counter()
    e0.record(stream)
    per = []
    for _ in range(args.steps):
        per.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = spq.spq_kernel_launches() - launches0
    elapsed_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)

    K = args.steps
    build_ms = [sum(pf[k] for k in ("validate", "reorder", "comp_fw", "bg_assemble", "bg_fw", "check"))
                for _, pf, _ in per]
    query_ms = [qm for _, _, qm in per]
    st0 = per[0][0]
    total_updates = st0["comp_updates"] + st0["bg_updates"]
    p3_ms = sum(pf["p3_ms"] for _, pf, _ in per)
    p3_launches = sum(pf["p3_launches"] for _, pf, _ in per)
    p3_updates = sum(pf["p3_updates"] for _, pf, _ in per)
    bs_ms = sum(pf.get("bs_ms", 0.0) for _, pf, _ in per)
    bs_launches = sum(pf.get("bs_launches", 0.0) for _, pf, _ in per)
    bs_updates = sum(pf.get("bs_updates", 0.0) for _, pf, _ in per)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_gops = sms * 128 * 2070e6 / 2 / 1e9  # 128 lanes/SM, 2 lane-ops per update, max SM clock
    kern = {
        "k_phase3_list": {"what": "k_phase3_list (boundary-graph elimination / Floyd-Warshall, phase 3)",
                          "ms": p3_ms, "launches": p3_launches, "updates": p3_updates, "traffic": None,
                          "traffic_note": "not captured for the elimination rounds"},
        "k_backsub": {"what": "k_backsub (boundary-graph back-substitution, persistent)",
                      "ms": bs_ms, "launches": bs_launches, "updates": bs_updates, "traffic": None,
                      "traffic_note": BACKSUB_TRAFFIC_NOTE},
    }
    top = max(kern, key=lambda x: kern[x]["ms"])
    other = [x for x in kern if x != top and kern[x]["ms"] > 0]

    def roof(name):
        kd = kern[name]
        ach = kd["updates"] / (kd["ms"] * 1e-3) / 1e9 if kd["ms"] > 0 else None
        return {"kernel": kd["what"], "bound": "alu", "achieved": ach, "peak": peak_gops, "unit": "Gop/s",
                "frac": (ach / peak_gops) if ach else None, "traffic": kd["traffic"],
                "traffic_note": kd["traffic_note"],
                "launches": int(kd["launches"]),
                "avg_launch_ms": kd["ms"] / max(kd["launches"], 1),
                "share_of_bg_ms": kd["ms"] / K / max(statistics.mean(pf["bg_fw"] for _, pf, _ in per), 1e-9)}

    # the grouped query kernel (block copy): ALU and DRAM fractions of its own launches
    qk = [pf.get("query_kernel") for _, pf, _ in per]
    roof_query = None
    if all(qk):
        qms = statistics.mean(x["kernel_ms"] for x in qk)
        q_upd, q_bytes = qk[0]["updates"], qk[0]["bytes"]
        hbm_peak = measured_hbm_gbs()
        roof_query = {
            "kernel": "k_qb_blocks (staged grouped queries)", "bound": "alu",
            "achieved": q_upd / (qms * 1e-3) / 1e9, "peak": peak_gops, "unit": "Gop/s",
            "frac": q_upd / (qms * 1e-3) / 1e9 / peak_gops, "launches": len(qk), "avg_launch_ms": qms,
            "updates": q_upd, "hbm": {"achieved": q_bytes / (qms * 1e-3) / 1e9, "peak": hbm_peak["value"],
                                      "unit": "GB/s", "frac": q_bytes / (qms * 1e-3) / 1e9 / hbm_peak["value"],
                                      "peak_basis": hbm_peak["basis"], "bytes": q_bytes,
                                      "bytes_formula": "per item 4*|B1|*|B2| (its block, once) + per pair "
                                                       "4*(roundup4(|B1|) + roundup4(|B2|)) + 16"},
            "traffic": None}

    # measured issue peak of the update (same process, after the timed region)
    ups, pms = ctypes.c_double(), ctypes.c_double()
    micro = {}
    for mode in (1, 2, 3):
        if lib.spq_peak_minplus(mode, 20000, 8, ctypes.byref(ups), ctypes.byref(pms)) == 0:
            micro[str(mode)] = round(ups.value / 1e9, 1)

    line = {
        "metric": METRIC,
        "value": whole_job_rate(K * q, world, elapsed_ms * 1e-3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": elapsed_ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("int32 results, exact float32 arithmetic (checked)" if st0["arith"] == spq.SPQ_ARITH_F32
                  else "int32"),
        "data": "synthetic",
        "config": workload_config(desc, world),
        "build_ms": statistics.mean(build_ms),
        "build_gops": total_updates / (statistics.mean(build_ms) * 1e-3) / 1e9,
        "build_updates": total_updates,
        "n_bg": st0["n_bg"],
        "bg_order": int(per[0][1].get("order_method", -1)),
        "bg_method": {1: "floyd-warshall", 2: "elimination + back-substitution"}.get(
            int(per[0][1].get("bg_method", 1)), "?"),
        "query_ms": statistics.mean(query_ms),
        "query_qps": q / (statistics.mean(query_ms) * 1e-3),
        "build_stage_ms": {k: round(statistics.mean(pf[k] for _, pf, _ in per), 2)
                           for k in ("validate", "reorder", "comp_fw", "bg_assemble", "bg_fw", "check")},
        "roofline": dict(roof(top), peak_basis=f"{sms} SMs x 128 lanes x 2070 MHz / 2 lane-ops per min-plus "
                                                 "update (derived)", microbench_gops=micro),
        "roofline_other": [roof(x) for x in other] + ([roof_query] if roof_query else []),
        "gpu_launches": int(launches),
        "clocks": clk,
        "wall_s_timed": wall,
        "query_autotune": tuning_summary(spq), "build_autotune": build_tuning_summary(spq),
    }

    last_out = d_out.cpu().numpy()  # answers of the last timed step (outside the timed region)

    # end to end through the public API with host buffers (pinned), H2D/D2H inside
    if args.e2e_steps > 0:
        h_rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr)).pin_memory()
        h_col = torch.from_numpy(np.ascontiguousarray(g.col)).pin_memory()
        h_w = torch.from_numpy(np.ascontiguousarray(g.w)).pin_memory()
        h_part = torch.from_numpy(np.ascontiguousarray(w.part)).pin_memory()
        h_pairs = torch.from_numpy(np.ascontiguousarray(w.pairs)).pin_memory()
        h_out = torch.empty(q, dtype=torch.int32).pin_memory()
        del d_rp, d_col, d_w, d_part, d_pairs, d_out
        torch.cuda.empty_cache()
        h2d = sum(t.numel() * t.element_size() for t in (h_rp, h_col, h_w, h_part, h_pairs))
        d2h = h_out.numel() * h_out.element_size()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        spq.spq_free(spq.spq_build(g.n, h_rp, h_col, h_w, h_part, w.k))  # host-buffer path warm
        torch.cuda.synchronize()
        e2e_s = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            h = spq.spq_build(g.n, h_rp, h_col, h_w, h_part, w.k)
            spq.spq_query(h, h_pairs, out=h_out)
            h.free()
            e2e_s.append(time.perf_counter() - t0)
        te = max_over_ranks(sum(e2e_s), dist, dev)
        line["e2e"] = {"value": whole_job_rate(args.e2e_steps * q, world, te), "unit": UNIT,
                       "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
                       "step_s": [round(x, 4) for x in e2e_s],
                       "same_answers_as_device_step": bool(np.array_equal(h_out.numpy(), last_out))}

    if rank == 0 and world == 1:
        qps, n, dt, cores, idx, ref = cpu_oracle_sample(w, args.cpu_seconds)
        # the oracle's answers on its sample against the GPU's answers of the last timed step
        ref = np.where(ref >= (1 << 62), spq.SPQ_INF_I32, ref)
        agree = int((last_out[idx].astype(np.int64) == ref).sum())
        line["cpu_baseline"] = {"value": qps, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{n} uniformly drawn pairs of the workload ({dt:.1f} s), binary-heap "
                                          f"Dijkstra with early exit per pair, OpenMP over pairs, no preprocessing",
                                "gpu_answers_equal_on_sample": f"{agree}/{n}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
