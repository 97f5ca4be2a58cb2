"""Parity at large sizes.  At the benchmark's full size, in the benchmark's
launch configuration: a CPMA of 1e8 uniform 40-bit keys receives a 1e6-key
insert batch and a 1e6-key delete batch (the headline step), and its answers
are checked on samples the plain definition computes directly (numpy set
operations on the same seeded keys): counts, size, full sum, has on 2e4
keys and range sums / counts / map_range_length on 2e3 rank-based ranges.
At 1e7 keys the whole layout (every leaf byte, used count and head entry)
is compared with the sequential CPMA after a uniform insert, a delete and a
skewed insert of 1e5 keys each (Sec. 4: merge, counting, redistribution at
the leaf count and fill of a large set)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_05055_gb300 import cpma as cp
from paper_2305_05055_gb300 import workloads as W
from setops import member, sorted_unique

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def range_sums(S, lo, hi):
    """Sum (mod 2^64) and count of S in [lo, hi) by prefix sums."""
    pre = np.zeros(S.size + 1, dtype=np.uint64)
    np.cumsum(S, dtype=np.uint64, out=pre[1:])
    i = np.searchsorted(S, lo, side="left")
    j = np.maximum(i, np.searchsorted(S, hi, side="left"))
    return pre[j] - pre[i], (j - i).astype(np.uint64)


def test_headline_size_parity():
    n, k = 10 ** 8, 10 ** 6
    base = W.uniform_keys(2, n, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    S = sorted_unique(base)
    del base
    assert g.size() == S.size
    # insert: new keys go in at their binary-search positions
    ins = W.uniform_keys(10 ** 6, k, bits=40)
    added = int(g.insert_batch(T(ins)).item())
    U = sorted_unique(ins)
    new = U[~member(U, S)]
    assert added == new.size
    S = np.insert(S, np.searchsorted(S, new), new)
    # delete: half present keys of the batch, half fresh keys
    dele = np.concatenate([U[W.permuted_indices(U.size, k // 2, 7)],
                           W.uniform_keys(8, k // 2, bits=40)])
    removed = int(g.delete_batch(T(dele)).item())
    D = sorted_unique(dele)
    hit = D[member(D, S)]
    assert removed == hit.size
    S = np.delete(S, np.searchsorted(S, hit))
    assert g.size() == S.size
    s, c = g.sum()
    assert int(cp.to_u64(s)[0]) == int(np.sum(S, dtype=np.uint64)) and int(c.item()) == S.size
    q = np.concatenate([S[W.permuted_indices(S.size, 10 ** 4, 9)], W.uniform_keys(11, 10 ** 4, bits=40),
                        np.array([0, M64], np.uint64)])
    assert np.array_equal(g.has_batch(T(q)).cpu().numpy(), member(q, S).astype(np.uint8))
    lo, hi, cnt = W.range_queries_by_rank(S, 12, 2000, 10, 10 ** 6)
    gs, gc = g.range_map(T(lo), T(hi))
    ws, wc = range_sums(S, lo, hi)
    assert np.array_equal(cp.to_u64(gc), wc) and np.array_equal(cp.to_u64(gs), ws)
    ls, lc = g.range_map_length(T(lo), T(cnt.astype(np.uint64)))
    assert np.array_equal(cp.to_u64(lc), wc) and np.array_equal(cp.to_u64(ls), ws)


def same_layout(g, o):
    assert g.leaves() == o.leaves() and g.leaf_bytes() == o.leaf_bytes()
    data, used, heads = g.layout()
    od, ou, oh = o.layout()
    gu = used.cpu().numpy().view(np.uint32)
    bad = np.nonzero(gu != ou)[0][:10]
    assert bad.size == 0, ("used differs", bad, gu[bad], ou[bad])
    assert np.array_equal(cp.to_u64(heads), oh)
    assert np.array_equal(data.cpu().numpy(), od)
    assert g.size() == o.size() and g.bytes() == o.bytes()


def test_layout_parity_at_1e7_keys():
    n, k = 10 ** 7, 10 ** 5
    base = W.uniform_keys(61, n, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    del base
    same_layout(g, o)
    ins = W.uniform_keys(62, k, bits=40)
    assert int(g.insert_batch(T(ins)).item()) == o.insert_batch(ins)
    same_layout(g, o)
    dele = W.sample_present(o.elements(), 63, k)
    assert int(g.delete_batch(T(dele)).item()) == o.delete_batch(dele)
    same_layout(g, o)
    z = W.zipf_keys(64, k, bits=34)
    assert int(g.insert_batch(T(z)).item()) == o.insert_batch(z)
    same_layout(g, o)
    assert o.check() == 0
