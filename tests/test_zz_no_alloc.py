"""Allocation-free NEAREST (mrpop_nearest_noalloc) checked against mrpop_nearest.

Some callers cannot allocate device memory while they plan: a real-time
replanning loop must neither stall on the allocator nor risk an out-of-memory
failure in the middle of a control cycle, and a process may already have its
device memory reserved by another framework's caching allocator.  For them
mrpop_nearest_noalloc keeps its partial minima in one fixed device array
instead of stream-ordered scratch.

Both entry points are called through the C ABI on the same inputs, two calls
in a row with different shapes (so stale contents of the shared array would
show), and must return identical indices -- the tolerance of the NEAREST tests
for two GPU results: the key (distance, g, index) is a total order, so how the
tree is split across blocks cannot change the answer.  A second test checks
the defining property itself: after a warm-up call, a call of the no-alloc
entry point leaves the library's scratch pool and the device's default
stream-ordered pool (their high-water marks), torch's caching allocator and
the device's free memory unchanged, while the same check does see
mrpop_nearest's split-tree scratch (a positive control).  This file is
collected last and also passes when run on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2609_30644_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2609_30644_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return m.lib


def _call(fn, tree, qs, cs, out, n_vertices):
    dim = tree.shape[0] - 1
    return fn(tree.data_ptr(), n_vertices, tree.shape[1], dim, qs.data_ptr(), cs.data_ptr(),
              qs.shape[1], out.data_ptr(), torch.cuda.current_stream().cuda_stream)


def _inputs(D, N, Q, seed):
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    tree = torch.from_numpy(synth.random_tree_fast(D, N, lo, hi, seed=seed)).cuda()
    qs_np, cs_np = synth.nn_queries(D, Q, lo, hi, seed=seed + 10, budget_lo=2.0, budget_hi=30.0)
    return tree, torch.from_numpy(qs_np).cuda(), torch.from_numpy(cs_np).cuda()


@pytest.mark.parametrize("shapes", [((14, 200_000, 5), (7, 50_000, 4096))])
def test_noalloc_matches_nearest_two_calls(lib, shapes):
    for call, (D, N, Q) in enumerate(shapes):
        tree, qs, cs = _inputs(D, N, Q, 40 + call)
        ref = torch.full((Q,), -7, dtype=torch.int64, device="cuda")
        got = torch.full((Q,), -7, dtype=torch.int64, device="cuda")
        assert _call(lib.mrpop_nearest, tree, qs, cs, ref, N) == 0
        assert _call(lib.mrpop_nearest_noalloc, tree, qs, cs, got, N) == 0, \
            lib.mrpop_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {call}: {(got != ref).sum().item()} indices differ"
        assert (got >= 0).any() and (got >= -1).all()


class _Pool:
    """The current device's default stream-ordered memory pool, through the
    CUDA driver API (cuDeviceGetDefaultMemPool, cuMemPoolGet/SetAttribute)."""
    USED_MEM_CURRENT = 7   # CU_MEMPOOL_ATTR_USED_MEM_CURRENT
    USED_MEM_HIGH = 8      # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)   # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH,
                                             ctypes.byref(zero)) == 0

    def free_bytes(self):
        free, total = ctypes.c_size_t(), ctypes.c_size_t()
        assert self.cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
        return free.value


def _scratch(lib, reset_high):
    """The library's scratch pool on this device: (in use, high-water mark)."""
    v = (ctypes.c_int64 * 3)()
    assert lib.mrpop_scratch_stats(int(reset_high), v) == 0
    return v[0], v[1]


def _allocations_during(lib, fn):
    """Runs fn (one library call, then a synchronize) and returns the growth of
    the pools' high-water marks (the library's scratch pool plus the device's
    default pool) over their use before, the change of torch's allocation
    count and the change of the device's free memory."""
    pool = _Pool()
    torch.cuda.synchronize()
    pool.reset_high()
    used0 = pool.get(_Pool.USED_MEM_CURRENT)
    lib_used0, _ = _scratch(lib, reset_high=True)
    torch_allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    free0 = pool.free_bytes()
    fn()
    torch.cuda.synchronize()
    _, lib_high = _scratch(lib, reset_high=False)
    return (pool.get(_Pool.USED_MEM_HIGH) - used0 + lib_high - lib_used0,
            torch.cuda.memory_stats().get("allocation.all.allocated", 0) - torch_allocs0,
            free0 - pool.free_bytes())


def test_noalloc_allocates_nothing(lib):
    D, N, Q = 14, 200_000, 5           # few queries, large tree: split across blocks
    tree, qs, cs = _inputs(D, N, Q, 60)
    ref = torch.empty(Q, dtype=torch.int64, device="cuda")
    got = torch.empty(Q, dtype=torch.int64, device="cuda")
    # warm-up: loads the modules (and with them the fixed array) on this device
    assert _call(lib.mrpop_nearest, tree, qs, cs, ref, N) == 0
    assert _call(lib.mrpop_nearest_noalloc, tree, qs, cs, got, N) == 0
    torch.cuda.synchronize()
    # positive control: the split-tree scratch of mrpop_nearest shows in the pool
    pool_grew, _, _ = _allocations_during(
        lib, lambda: _call(lib.mrpop_nearest, tree, qs, cs, ref, N))
    assert pool_grew > 0, "the check does not see stream-ordered scratch"
    # the no-alloc entry point, twice: nothing from the pool, torch or cudaMalloc
    for _ in range(2):
        pool_grew, torch_allocs, free_drop = _allocations_during(
            lib, lambda: _call(lib.mrpop_nearest_noalloc, tree, qs, cs, got, N))
        # (free memory may rise when the pool trims what the control left)
        assert pool_grew == 0 and torch_allocs == 0 and free_drop <= 0, \
            (pool_grew, torch_allocs, free_drop)
        assert torch.equal(got, ref)


def test_noalloc_rejects_batches_beyond_its_limit(lib):
    D, N = 7, 1000
    limit = 65536                                     # MRPOP_NEAREST_NOALLOC_MAX_QUERIES
    tree = torch.zeros((D + 1, N), dtype=torch.float32, device="cuda")
    qs = torch.zeros((D, limit + 1), dtype=torch.float32, device="cuda")
    cs = torch.ones(limit + 1, dtype=torch.float32, device="cuda")
    out = torch.empty(limit + 1, dtype=torch.int64, device="cuda")
    assert _call(lib.mrpop_nearest_noalloc, tree, qs, cs, out, N) == 1   # MRPOP_EINVAL
    assert b"MRPOP_NEAREST_NOALLOC_MAX_QUERIES" in lib.mrpop_last_error()
