"""Cluster tree T^L (Section 2.1), as a binary KD bisection.

The paper analyses a balanced 2^d-tree; the workloads here use a binary tree
(reading R1): a cluster at level l < L is split at the median of the
coordinate with the largest bounding-box extent (ties on extent go to the
lowest axis), sorting by (coordinate, original index); the left child takes
the first floor(|C|/2) points.  Every cluster at a level below L is split, so
level l has exactly 2^l clusters and L is the smallest depth at which every
leaf holds at most n_max points, L = ceil(log2(N / n_max)) (Section 2.1 with
2^d replaced by 2).

The geometry of a cluster is the tight axis-aligned bounding box of its
points (reading R5).  Nodes are numbered in heap order: node 2^l - 1 + i is
cluster i at level l; its children are 2n+1 and 2n+2.

Parity: pinned by tests (complete tree, permutation, median split property,
leaf sizes, ceil-log depth).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def tree_depth(n: int, leaf_size: int) -> int:
    """Smallest L with ceil(n / 2^L) <= leaf_size (0 when n <= leaf_size)."""
    L = 0
    while -(-n // (1 << L)) > leaf_size:
        L += 1
    return L


@dataclass
class Tree:
    L: int
    perm: np.ndarray      # perm[p] = original index of the point at tree position p
    off: np.ndarray       # per node: first tree position
    size: np.ndarray      # per node: number of points
    lo: np.ndarray        # per node: bounding box lower corner (dim,)
    hi: np.ndarray        # per node: bounding box upper corner (dim,)

    def node(self, level: int, i: int) -> int:
        return (1 << level) - 1 + i

    def rng(self, level: int, i: int) -> tuple[int, int]:
        n = self.node(level, i)
        return int(self.off[n]), int(self.size[n])


def build_tree(points: np.ndarray, leaf_size: int) -> Tree:
    pts = np.asarray(points, dtype=np.float64)
    n, dim = pts.shape
    L = tree_depth(n, leaf_size)
    nn = (1 << (L + 1)) - 1
    perm = np.arange(n, dtype=np.int64)
    off = np.zeros(nn, dtype=np.int64)
    size = np.zeros(nn, dtype=np.int64)
    lo = np.zeros((nn, dim))
    hi = np.zeros((nn, dim))
    off[0], size[0] = 0, n
    for node in range(nn):
        o, s = int(off[node]), int(size[node])
        idx = perm[o:o + s]
        p = pts[idx]
        if s > 0:
            lo[node] = p.min(axis=0)
            hi[node] = p.max(axis=0)
        level = (node + 1).bit_length() - 1
        if level == L:
            continue
        ext = hi[node] - lo[node]
        axis = int(np.argmax(ext))               # first maximum: lowest axis
        order = np.lexsort((idx, p[:, axis]))    # by coordinate, then original index
        perm[o:o + s] = idx[order]
        h = s // 2
        off[2 * node + 1], size[2 * node + 1] = o, h
        off[2 * node + 2], size[2 * node + 2] = o + h, s - h
    return Tree(L=L, perm=perm, off=off, size=size, lo=lo, hi=hi)
