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
tree is split across blocks cannot change the answer.  This file is collected
last and also passes when run on its own in a fresh process.
"""
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


@pytest.mark.parametrize("shapes", [((14, 200_000, 5), (7, 50_000, 4096))])
def test_noalloc_matches_nearest_two_calls(lib, shapes):
    for call, (D, N, Q) in enumerate(shapes):
        lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
        tree = torch.from_numpy(synth.random_tree_fast(D, N, lo, hi, seed=40 + call)).cuda()
        qs_np, cs_np = synth.nn_queries(D, Q, lo, hi, seed=50 + call, budget_lo=2.0,
                                        budget_hi=30.0)
        qs, cs = torch.from_numpy(qs_np).cuda(), torch.from_numpy(cs_np).cuda()
        ref = torch.full((Q,), -7, dtype=torch.int64, device="cuda")
        got = torch.full((Q,), -7, dtype=torch.int64, device="cuda")
        assert _call(lib.mrpop_nearest, tree, qs, cs, ref, N) == 0
        assert _call(lib.mrpop_nearest_noalloc, tree, qs, cs, got, N) == 0, \
            lib.mrpop_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {call}: {(got != ref).sum().item()} indices differ"
        assert (got >= 0).any() and (got >= -1).all()


def test_noalloc_rejects_batches_beyond_its_limit(lib):
    D, N = 7, 1000
    limit = 65536                                     # MRPOP_NEAREST_NOALLOC_MAX_QUERIES
    tree = torch.zeros((D + 1, N), dtype=torch.float32, device="cuda")
    qs = torch.zeros((D, limit + 1), dtype=torch.float32, device="cuda")
    cs = torch.ones(limit + 1, dtype=torch.float32, device="cuda")
    out = torch.empty(limit + 1, dtype=torch.int64, device="cuda")
    assert _call(lib.mrpop_nearest_noalloc, tree, qs, cs, out, N) == 1   # MRPOP_EINVAL
    assert b"MRPOP_NEAREST_NOALLOC_MAX_QUERIES" in lib.mrpop_last_error()
