"""Edge set over the CPMA (F-Graph style, keys u << 32 | v) on R-MAT graphs:
degrees, neighbour sums and neighbour lists against the plain set of the
same keys; breadth-first levels against a plain Python BFS over the
oracle's sorted edge list."""
from collections import deque

import numpy as np
import pytest
import torch

import oracle
from paper_2305_05055_gb300 import cpma as cp
from paper_2305_05055_gb300 import graph
from paper_2305_05055_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def keys_of(src, dst):
    return (src.astype(np.uint64) << np.uint64(32)) | dst.astype(np.uint64)


def plain_bfs(S, source, nv):
    adj = {}
    for k in S.tolist():
        adj.setdefault(k >> 32, []).append(k & 0xFFFFFFFF)
    level = [-1] * nv
    level[source] = 0
    q = deque([source])
    while q:
        u = q.popleft()
        for v in adj.get(u, ()):
            if v < nv and level[v] < 0:
                level[v] = level[u] + 1
                q.append(v)
    return level


@pytest.mark.parametrize("LB", [256, 1024])
def test_edge_set_matches_plain_set(LB):
    scale = 12
    nv = 1 << scale
    src, dst = W.rmat_edges(5, scale, 40000)
    es = graph.EdgeSet(src, dst, leaf_bytes=LB)
    p = oracle.PlainSet(keys_of(src, dst))
    assert es.num_edges() == len(p)
    for step in range(3):
        verts = np.arange(nv, dtype=np.int64)
        lo = verts.astype(np.uint64) << np.uint64(32)
        hi = (verts + 1).astype(np.uint64) << np.uint64(32)
        ws, wc = p.range_map(lo, hi)
        assert np.array_equal(cp.to_u64(es.degrees(verts)), wc)
        s, c = es.neighbor_sums(verts)
        assert np.array_equal(cp.to_u64(s), ws - wc * lo)
        sample = np.concatenate([verts[::37], np.array([0, nv - 1, nv + 5], np.int64)])
        off, nb = es.neighbors(sample)
        woff, wkeys = p.range_extract(sample.astype(np.uint64) << np.uint64(32),
                                      (sample + 1).astype(np.uint64) << np.uint64(32))
        assert np.array_equal(cp.to_u64(off), woff)
        assert np.array_equal(cp.to_u64(nb), wkeys & np.uint64(0xFFFFFFFF))
        # a batch of new edges and a batch of removals
        a, b = W.rmat_edges(50 + step, scale, 5000)
        assert es.add_edges(a, b) == p.insert_batch(keys_of(a, b))
        S = p.S
        gone = W.sample_present(S, 60 + step, 3000)
        assert es.remove_edges((gone >> np.uint64(32)).astype(np.int64),
                               (gone & np.uint64(0xFFFFFFFF)).astype(np.int64)) == \
            p.delete_batch(gone)
    src0 = int((p.S[0] >> np.uint64(32)))
    assert es.bfs(src0, nv).cpu().tolist() == plain_bfs(p.S, src0, nv)


def test_edge_set_rejects_out_of_range_vertices():
    es = graph.EdgeSet(np.array([1]), np.array([2]))
    with pytest.raises(ValueError):
        es.add_edges(np.array([1 << 31]), np.array([0]))
    with pytest.raises(ValueError):
        es.degrees(np.array([-1]))
