"""Cluster tree T^L (Section 2.1): a binary KD bisection, and the paper's
geometrically balanced 2^d-tree.

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

The balanced 2^d-tree (Section 2.1: quad-tree in 2-D, oct-tree in 3-D) is
held in the same heap as a binary tree whose binary level b splits its cell
at the midpoint of axis b mod d, so that 2^d-tree level l is binary level
d l and a cluster's 2^d children are its descendants d binary levels down.
The root cell is the smallest axis-aligned hypercube containing the points
(centred on their bounding box, side the largest extent); a point goes to
the upper half-cell when its coordinate is >= the midpoint, and each cell
keeps the order of its parent (stable).  The depth is the smallest L with
ceil(N / 2^{dL}) <= n_max, which is L = ceil(log_{2^d}(N / n_max)) of the
paper for a perfectly balanced tree; cells may hold any number of points,
including none.  The geometry of a 2^d-tree cluster is its cell, the
hypercube of Section 2.1's analysis (so the interaction-list sizes obey the
closed forms of Eqs. 2.3, 2.5 and 2.8), stored in lo / hi.

Parity: pinned by tests (complete tree, permutation, median split property,
leaf sizes, ceil-log depth; for the 2^d-tree: every point inside its cell,
cells the 2^d sub-cubes of their parent, exact balance on a regular grid).
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


def tree_depth_2d(n: int, dim: int, leaf_size: int) -> int:
    """Smallest L with ceil(n / 2^{dim L}) <= leaf_size (2^d-tree levels)."""
    L = 0
    while -(-n // (1 << (dim * L))) > leaf_size:
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

    step: int = 1         # binary levels per tree level (d for the 2^d-tree)
    cell_lo: np.ndarray | None = None   # 2^d-tree: the cell of every node
    cell_hi: np.ndarray | None = None

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


def build_tree_2d(points: np.ndarray, leaf_size: int) -> Tree:
    """The balanced 2^d-tree, in binary-level form (step = d)."""
    pts = np.asarray(points, dtype=np.float64)
    n, dim = pts.shape
    L = dim * tree_depth_2d(n, dim, leaf_size)
    nn = (1 << (L + 1)) - 1
    perm = np.arange(n, dtype=np.int64)
    off = np.zeros(nn, dtype=np.int64)
    size = np.zeros(nn, dtype=np.int64)
    clo = np.zeros((nn, dim))     # cell of every node: the cluster geometry
    chi = np.zeros((nn, dim))
    mn, mx = pts.min(axis=0), pts.max(axis=0)
    half = 0.5 * float(np.max(mx - mn))
    for a in range(dim):
        c = 0.5 * (float(mn[a]) + float(mx[a]))
        clo[0, a], chi[0, a] = c - half, c + half
    off[0], size[0] = 0, n
    for node in range(nn):
        o, s = int(off[node]), int(size[node])
        idx = perm[o:o + s]
        p = pts[idx]
        level = (node + 1).bit_length() - 1
        if level == L:
            continue
        axis = level % dim
        mid = 0.5 * (float(clo[node, axis]) + float(chi[node, axis]))
        upper = p[:, axis] >= mid
        perm[o:o + s] = np.concatenate([idx[~upper], idx[upper]])
        h = int(s - np.count_nonzero(upper))
        for c, (co, cs) in ((2 * node + 1, (o, h)), (2 * node + 2, (o + h, s - h))):
            off[c], size[c] = co, cs
            clo[c], chi[c] = clo[node], chi[node]
        chi[2 * node + 1, axis] = mid
        clo[2 * node + 2, axis] = mid
    return Tree(L=L, perm=perm, off=off, size=size, lo=clo, hi=chi, step=dim, cell_lo=clo, cell_hi=chi)
