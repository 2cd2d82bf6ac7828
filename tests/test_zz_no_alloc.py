"""spq_query_noalloc, the query entry point that allocates no memory (needs a GPU).

It exists for callers that cannot let the library allocate device memory while they
serve requests (a process whose free device memory is all in its own pool, or one under
a fixed budget where an allocation could fail or stall).  Its scratch is the library's
fixed device array instead of a stream-ordered allocation; its answers must equal those
of spq_query.  Distances here are integers, so "equal" means bit-identical, the same
bar as every integer parity test.  This file is collected last, so a run that stops at
the first failure has already run every other test.
"""

import ctypes
import gc

import numpy as np
import pytest

from _util import build, spq, torch_dev

import gen

pytestmark = pytest.mark.gpu


def _call(lib, h, pairs, out, torch):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.spq_query_noalloc(h.ptr, ctypes.c_void_p(pairs.data_ptr()), int(pairs.shape[0]),
                                 ctypes.c_void_p(out.data_ptr()), stream)


def _pool_used(lib, torch):
    used, reserved = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    assert lib.spq_pool_usage(torch.cuda.current_device(), ctypes.byref(used), ctypes.byref(reserved)) == 0
    return used.value, reserved.value


def test_noalloc_matches_spq_query_on_two_calls_in_a_row():
    m = spq()
    torch, dev = torch_dev()
    lib = m._lib.load()
    w = gen.configs.delaunay_rcb(1 << 14, 4, 60000, seed=23)
    h = build(w.graph, w.part, w.k)
    rng = np.random.default_rng(23)
    batches = [w.pairs, np.ascontiguousarray(w.pairs[rng.permutation(w.pairs.shape[0])[:41000], ::-1])]
    for i, b in enumerate(batches):
        pairs = torch.from_numpy(np.ascontiguousarray(b)).to(dev)
        ref = m.spq_query(h, pairs)
        out = torch.full((pairs.shape[0],), -7, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        # the call must take no memory from the library's pool, from torch's caching
        # allocator or (after the first call, which may load the array's module under
        # CUDA's lazy module loading) from the device: its scratch is the fixed array.
        # (Memory released meanwhile by the garbage collector may make a count drop: the
        # check is that none grows.)
        gc.collect()
        gc.disable()
        try:
            pool0 = _pool_used(lib, torch)
            torch0 = torch.cuda.memory_allocated(dev)
            free0 = torch.cuda.mem_get_info(dev)[0]
            assert _call(lib, h, pairs, out, torch) == 0
            torch.cuda.synchronize()
            assert _pool_used(lib, torch)[0] <= pool0[0]
            assert torch.cuda.memory_allocated(dev) <= torch0
            if i > 0:
                assert torch.cuda.mem_get_info(dev)[0] >= free0
        finally:
            gc.enable()
        m.spq_query_status(h)
        assert torch.equal(out, ref)
    h.free()


def test_noalloc_rejects_oversized_batches_and_host_buffers():
    m = spq()
    torch, dev = torch_dev()
    lib = m._lib.load()
    w = gen.configs.grid_blocks_workload(32, 32, 8, 8, 50, 100, seed=29)
    h = build(w.graph, w.part, w.k)
    q = m.SPQ_NOALLOC_MAX_PAIRS + 1
    pairs = torch.zeros((q, 2), dtype=torch.int32, device=dev)
    out = torch.full((q,), -7, dtype=torch.int32, device=dev)
    assert _call(lib, h, pairs, out, torch) == m.SPQ_EINVAL
    torch.cuda.synchronize()
    assert int(out[0]) == -7  # nothing was queued
    hp = torch.from_numpy(np.ascontiguousarray(w.pairs))
    ho = torch.empty(hp.shape[0], dtype=torch.int32)
    assert _call(lib, h, hp, ho, torch) == m.SPQ_EINVAL
    h.free()
