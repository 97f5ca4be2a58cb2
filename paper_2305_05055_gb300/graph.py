"""Directed edge set over the CPMA, in the style of the paper's F-Graph
(Sec. 6 "graph application": a graph kept as one compressed set of edges).

Edge (u, v) is the 64-bit key ``u << 32 | v``, so the out-edges of u are the
keys of [u << 32, (u + 1) << 32) and sorted by destination.  Vertex ids are
below 2^31 (so every key and range bound fits a non-negative int64).
Updates are the CPMA's batch insert and delete; a neighbour scan of a batch
of vertices is one range_map (degrees, sums of neighbour ids) or one
range_extract (the neighbour lists, packed CSR-style).  Breadth-first search
expands a frontier by one range_extract per level; the frontier bookkeeping
(visited marks, dedup) is plain torch.
"""
from __future__ import annotations

import numpy as np
import torch

from . import cpma as cp

MAX_VERTEX = (1 << 31) - 1


def edge_keys(src, dst) -> torch.Tensor:
    """u << 32 | v as int64 keys on the device of src."""
    src = torch.as_tensor(src, dtype=torch.int64)
    dst = torch.as_tensor(dst, dtype=torch.int64, device=src.device)
    if src.numel() and (int(src.max()) > MAX_VERTEX or int(dst.max()) > MAX_VERTEX
                        or int(src.min()) < 0 or int(dst.min()) < 0):
        raise ValueError("vertex ids must be in [0, 2^31)")
    return (src << 32) | dst


class EdgeSet:
    """A directed graph as one CPMA of edge keys."""

    def __init__(self, src=None, dst=None, device="cuda", **config):
        self.dev = torch.device(device)
        keys = None
        if src is not None:
            keys = edge_keys(torch.as_tensor(np.asarray(src, dtype=np.int64)).to(self.dev),
                             torch.as_tensor(np.asarray(dst, dtype=np.int64)).to(self.dev))
        self.g = cp.CPMA(keys, **config)

    def _vkeys(self, src, dst):
        src = torch.as_tensor(np.asarray(src, dtype=np.int64) if not torch.is_tensor(src) else src)
        dst = torch.as_tensor(np.asarray(dst, dtype=np.int64) if not torch.is_tensor(dst) else dst)
        return edge_keys(src.to(self.dev), dst.to(self.dev))

    def add_edges(self, src, dst) -> int:
        """Insert a batch of edges; returns how many were new."""
        return int(self.g.insert_batch(self._vkeys(src, dst)).item())

    def remove_edges(self, src, dst) -> int:
        """Delete a batch of edges; returns how many were present."""
        return int(self.g.delete_batch(self._vkeys(src, dst)).item())

    def num_edges(self) -> int:
        return self.g.size()

    def _bounds(self, vertices):
        v = torch.as_tensor(vertices, dtype=torch.int64).to(self.dev)
        if v.numel() and (int(v.min()) < 0 or int(v.max()) > MAX_VERTEX):
            raise ValueError("vertex ids must be in [0, 2^31)")
        return v << 32, (v + 1) << 32

    def degrees(self, vertices) -> torch.Tensor:
        """Out-degree of every vertex of the batch (one range_map launch)."""
        lo, hi = self._bounds(vertices)
        return self.g.range_map(lo, hi)[1]

    def neighbor_sums(self, vertices):
        """(sum of out-neighbour ids, out-degree) per vertex: the range sum
        minus degree * (u << 32), all modulo 2^64."""
        lo, hi = self._bounds(vertices)
        s, c = self.g.range_map(lo, hi)
        return s - c * lo, c

    def neighbors(self, vertices):
        """Out-neighbour lists of a batch of vertices, packed: (offsets,
        dst) with vertex i's neighbours at dst[offsets[i]:offsets[i+1]]."""
        lo, hi = self._bounds(vertices)
        off, keys = self.g.range_extract(lo, hi)
        return off, keys & 0xFFFFFFFF

    def bfs(self, source: int, num_vertices: int) -> torch.Tensor:
        """Breadth-first levels from `source` (-1 for unreached vertices):
        one neighbour extraction per level."""
        level = torch.full((num_vertices,), -1, dtype=torch.int64, device=self.dev)
        frontier = torch.tensor([int(source)], dtype=torch.int64, device=self.dev)
        level[frontier] = 0
        d = 0
        while frontier.numel():
            _, nb = self.neighbors(frontier)
            nb = nb[nb < num_vertices]
            nb = torch.unique(nb[level[nb] < 0])
            d += 1
            level[nb] = d
            frontier = nb
        return level
