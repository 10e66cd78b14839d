"""Admissibility conditions and the H_h block partition.

adm_s (Eq. 2.2): min(diam C_i, diam C_j) <= eta * dist(C_i, C_j), inclusive,
  with diam/dist of the tight bounding boxes (reading R5), evaluated as
  sqrt of the squared extents summed in axis order.
adm_w (Eq. 2.4): i != j.
adm_h (Eq. 3.1 and the three steps that follow it): standard admissibility
  on levels 1..ell; at level ell the remaining off-diagonal ("finer
  neighbour") pairs are admissible too; weak admissibility on levels
  ell+1..L; leaf-level diagonal blocks stay dense (Algorithm 1).

The partition recurses on cluster pairs from (root, root); a pair at level
l >= 1 becomes
  'std'   if l <= ell and adm_s holds,
  'finer' else if l == ell < L and i != j,
  'weak'  else if l > ell and i != j,
  dense   else if l == L (the diagonal; with ell == L also the leaf
          neighbours, 'nbr', which Algorithm 3's special case may still
          compress when that pays off),
and otherwise its four child pairs are visited.  ell = L gives an H_s
matrix and ell = 0 a HODLR matrix (Section 3.2 special cases).

On a 2^d-tree (tree.step = d, levels in binary-level form) only the levels
that are multiples of d are tree levels: a pair is refined into the
2^d x 2^d pairs of its clusters' children d binary levels down, ell is
given as a binary level (d times the tree level), and pairs with an empty
cluster are dropped (they hold no entries).

Sparsity constants C', C'', C''' (Eqs. 2.3, 2.5, 2.8) in closed form, and the
measured C_sp(l) = max over row clusters i at level l of the number of
admissible blocks in row i (reading R3).

Parity: pinned by tests (coverage of N x N exactly once, special cases, the
closed forms 27/8/3 and 189/26/7 at eta = sqrt(d), brute-force admissibility).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from .tree import Tree

KIND_STD, KIND_FINER, KIND_WEAK, KIND_NBR = 0, 1, 2, 3


def diam(t: Tree, node: int) -> float:
    s = 0.0
    for a in range(t.lo.shape[1]):
        e = float(t.hi[node, a]) - float(t.lo[node, a])
        s = s + e * e
    return math.sqrt(s)


def dist(t: Tree, n1: int, n2: int) -> float:
    s = 0.0
    for a in range(t.lo.shape[1]):
        g = max(0.0, float(t.lo[n2, a]) - float(t.hi[n1, a]), float(t.lo[n1, a]) - float(t.hi[n2, a]))
        s = s + g * g
    return math.sqrt(s)


# On the 2^d-tree the clusters are congruent cells, and at eta = sqrt(d) two
# cells one cell apart meet Eq. 2.2 with equality (the case the closed forms
# of Eqs. 2.3 and 2.5 count as admissible); rounding decides such a tie
# either way, so there the comparison carries a relative slack of 1e-12.
TIE_SLACK_2D = 1.0 + 1e-12


def adm_s(t: Tree, n1: int, n2: int, eta: float) -> bool:
    rhs = eta * dist(t, n1, n2)
    if t.step > 1:
        rhs = rhs * TIE_SLACK_2D
    return min(diam(t, n1), diam(t, n2)) <= rhs


@dataclass
class Partition:
    L: int
    ell: int
    lowrank: list = field(default_factory=list)   # (level, i, j, kind)
    dense: list = field(default_factory=list)     # (level, i, j, kind) kind 'diag'=-1 or KIND_NBR


def partition(t: Tree, eta: float, ell: int) -> Partition:
    L, step = t.L, t.step
    if not (0 <= ell <= L) or ell % step:
        raise ValueError("switch level must satisfy 0 <= ell <= L (a tree level)")
    P = Partition(L=L, ell=ell)
    stack = [(0, 0, 0)]
    while stack:
        l, i, j = stack.pop()
        ni, nj = t.node(l, i), t.node(l, j)
        if step > 1 and (t.size[ni] == 0 or t.size[nj] == 0):
            continue
        if l >= 1:
            if l <= ell and adm_s(t, ni, nj, eta):
                P.lowrank.append((l, i, j, KIND_STD))
                continue
            if l == ell and ell < L and i != j:
                P.lowrank.append((l, i, j, KIND_FINER))
                continue
            if l > ell and i != j:
                P.lowrank.append((l, i, j, KIND_WEAK))
                continue
        if l == L:
            P.dense.append((l, i, j, -1 if i == j else KIND_NBR))
            continue
        # children pairs, pushed in reverse so they pop in (0,0),(0,1),(1,0),(1,1) order
        c = 1 << step
        for a in range(c - 1, -1, -1):
            for b in range(c - 1, -1, -1):
                stack.append((l + step, c * i + a, c * j + b))
    return P


def sparsity_closed_form(d: int, eta: float) -> tuple[float, float, float]:
    """C' = (2^d - 1)(1 + 2 sqrt(d)/eta)^d, C'' = (1 + 2 sqrt(d)/eta)^d - 1, C''' = 2^d - 1."""
    g = (1.0 + 2.0 * math.sqrt(d) / eta) ** d
    return (2 ** d - 1) * g, g - 1.0, float(2 ** d - 1)


def measured_csp(levels_rows: list[tuple[int, int]], L: int) -> list[int]:
    """C_sp(l) for l = 0..L from (level, row cluster) of every admissible block."""
    counts: dict = {}
    for l, i in levels_rows:
        counts[(l, i)] = counts.get((l, i), 0) + 1
    out = [0] * (L + 1)
    for (l, _), c in counts.items():
        out[l] = max(out[l], c)
    return out
