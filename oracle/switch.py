"""Algorithm 2: the switching level with the largest storage gain of the
H_h matrix over the H_s matrix.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The storage of the H_s matrix (standard admissibility down to the leaves) and
of the H_h matrix with switching level ell share the far-field blocks of
levels 1..ell and the dense diagonal (Section 3.3, Eqs. 3.3-3.6), so
S_s - S_h(ell) = S_1(ell) - S_2(ell), and the level that maximizes the gain
S_1(ell) - S_2(ell) is the one with the smallest H_h storage.  Storage is
counted as in Section 5.2: p (m + n) b / 64 fp64 words for a low-rank block
in a b-bit format, m n for a dense block (HMatrix.storage), so in the mixed
precision setting the gain takes every block's assigned format into account
(the paper notes that the optimal level may then differ from the uniform
precision one).  H_s is the build with ell = L (with Section 4.3's
beneficial compression of leaf neighbours, as everywhere in this oracle), so
the gain at ell = L is zero, as Algorithm 2 states.

Algorithm 2 walks the tree from the leaves up: start at ell = L with gain 0,
evaluate ell - 1, move there while its gain is strictly larger than the
current one, and stop at the first level whose gain does not exceed it.  S_2
of a level is obtained by constructing that H_h matrix (Algorithm 1).

Parity: pinned in tests/test_oracle_switch.py against the block-list form of
S_1 - S_2, against an exhaustive evaluation of every level, and against the
zero gain at ell = L.
"""
from __future__ import annotations

import numpy as np

from .build import build
from .tree import tree_depth, tree_depth_2d


def storage_gain(points: np.ndarray, kernel: int, kernel_param: float, leaf_size: int, eta: float, tol: float,
                 fmt_mask: int, ell: int, storage_s: float, tree_kind: str = "kd") -> float:
    """S_1(ell) - S_2(ell) = S_s - S_h(ell) for one switching level (tree levels)."""
    H = build(points, kernel, kernel_param, leaf_size, eta, ell, tol, fmt_mask, tree_kind)
    return storage_s - H.storage()


def optimal_switch_level(points: np.ndarray, kernel: int, kernel_param: float, leaf_size: int, eta: float,
                         tol: float, fmt_mask: int, tree_kind: str = "kd") -> tuple[int, dict]:
    """Algorithm 2: returns (ell*, {ell: gain} for every level it evaluated),
    levels counted in the tree's own levels."""
    n, dim = np.shape(points)
    L = tree_depth_2d(n, dim, leaf_size) if tree_kind == "2d" else tree_depth(n, leaf_size)
    Hs = build(points, kernel, kernel_param, leaf_size, eta, L, tol, fmt_mask, tree_kind)
    ss = Hs.storage()
    ell, s = L, 0.0
    gains = {L: 0.0}
    while ell > 0:
        s_new = storage_gain(points, kernel, kernel_param, leaf_size, eta, tol, fmt_mask, ell - 1, ss, tree_kind)
        gains[ell - 1] = s_new
        if s_new <= s:
            break
        s, ell = s_new, ell - 1
    return ell, gains
