"""The multi-rank (N > 1) host path of the benchmark on CPU, with two gloo ranks.

A run on N GPUs is N replicas of the single-GPU step (the path has no exchange step on
one GPU); what the ranks share is the timing: a barrier around the timed region, the
timed span taken as the slowest rank's (a MAX all-reduce), and the whole-job rate = all
ranks' units over that span.  Here each rank reports a different span; every rank must
get the maximum, and the rate must count both ranks' work.  The reference arm under a
launcher: rank 0 alone runs, the others return 0 without work.
"""

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        span = [2.5, 4.0][rank]                      # seconds of this rank's timed region
        slowest = bench.max_over_ranks(span, dist)    # every rank: the slowest span
        rate = bench.whole_job_rate(1000.0, world, slowest)
        alone = bench.max_over_ranks(span, None)      # no process group: the value itself

        class A:
            pass

        ref = bench.run_reference(A(), rank) if rank != 0 else 0  # non-zero ranks: no work
        out[rank] = (slowest, rate, alone, ref)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_span_and_the_whole_job_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    assert res[0][0] == res[1][0] == 4.0
    assert res[0][1] == pytest.approx(2 * 1000.0 / 4.0)
    assert (res[0][2], res[1][2]) == (2.5, 4.0)
    assert res[1][3] == 0
