"""The allocation-free range_map entry point.

Callers that cannot allocate device memory inside a call (their memory is all
handed to another allocator up front, or they must not hit the device-wide
synchronisation that cudaFree implies) use cpma_range_map_noalloc, whose
scratch is a fixed array inside the library.  Through the C ABI, two calls in a
row must give exactly what cpma_range_map gives on the same queries and what
the CPU oracle's plain sorted set gives (integer sums and counts: bit for
bit), on batches that take the offset scan's one-block path (q <= 8192) and
its multi-block path, and oversized batches must be rejected.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_2305_05055_gb300 import cpma as cp
from paper_2305_05055_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def T(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.uint64)).view(np.int64)).cuda()


def _call(fn, h, lo, hi, s, c):
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(h, C.c_void_p(lo.data_ptr()), C.c_void_p(hi.data_ptr()), lo.numel(),
              C.c_void_p(s.data_ptr()), C.c_void_p(c.data_ptr()), st)


def test_noalloc_range_map_matches_range_map_twice():
    assert torch.cuda.is_available()
    lib = cp.lib()
    base = W.uniform_keys(71, 400000, bits=40)
    extra = W.zipf_keys(72, 50000, bits=34)
    g = cp.CPMA(T(base), leaf_bytes=512)
    g.insert_batch(T(extra))
    p = oracle.PlainSet(base)
    p.insert_batch(extra)
    S = p.S
    # 1 and 5000 queries: the one-block offset scan; 20000 and the maximum:
    # the multi-block scan
    cases = [(1, 76), (5000, 77), (20000, 73), (cp.RANGE_NOALLOC_MAX_QUERIES, 74)]
    for rnd, (nq, seed) in enumerate(cases):
        lo, hi, _ = W.range_queries_by_rank(S, seed, nq, 1, 100000)
        ws, wc = p.range_map(lo, hi)
        lo, hi = T(lo), T(hi)
        s0 = torch.empty(nq, dtype=torch.int64, device="cuda")
        c0 = torch.empty_like(s0)
        s1 = torch.full_like(s0, 12345)      # stale values must not survive
        c1 = torch.full_like(s0, 678)
        assert _call(lib.cpma_range_map, g.handle, lo, hi, s0, c0) == 0
        assert _call(lib.cpma_range_map_noalloc, g.handle, lo, hi, s1, c1) == 0
        torch.cuda.synchronize()
        assert torch.equal(c0, c1), "counts differ in call %d" % rnd
        assert torch.equal(s0, s1), "sums differ in call %d" % rnd
        assert np.array_equal(cp.to_u64(c1), wc), "counts differ from the oracle in call %d" % rnd
        assert np.array_equal(cp.to_u64(s1), ws), "sums differ from the oracle in call %d" % rnd
        assert int(c1.sum().item()) > 0


def test_noalloc_rejects_oversized_batches():
    lib = cp.lib()
    g = cp.CPMA(T(W.uniform_keys(75, 10000, bits=40)), leaf_bytes=512)
    q = cp.RANGE_NOALLOC_MAX_QUERIES + 1
    lo = torch.zeros(q, dtype=torch.int64, device="cuda")
    hi = torch.ones(q, dtype=torch.int64, device="cuda")
    s = torch.empty(q, dtype=torch.int64, device="cuda")
    c = torch.empty(q, dtype=torch.int64, device="cuda")
    assert _call(lib.cpma_range_map_noalloc, g.handle, lo, hi, s, c) == cp.CPMA_EINVAL
