"""The level factor of Algorithm 3's precision rule, pinned by maximality.

Theorem 4.2 holds when every admissible block at 2^d-tree level l is stored
with a unit roundoff u <= eps / (2^{d l / 2} xi), xi = ||H~_IJ|| / ||H~||
(Eq. 4.6, the hypothesis of the theorem in Section 4.2); Algorithm 3 takes the
LARGEST allowed u meeting it.  A rule with a too-large factor (2^{d l}, or
2^{l/2} mistaken for 2^{d l/2} in the other direction) still satisfies the
theorem, so sufficiency tests cannot see it; it only loses storage.  These
tests recompute every block's bound from quantities the rule never touches:

* ||H~_IJ|| from the singular values of the dense block U V^T (numpy SVD),
  ||H~|| from the assembled dense H~;
* the factor in the paper's form 2^{d l / 2} at 2^d-tree level l (the
  binary-level form of the oracle is converted back), and on the binary KD
  tree the square root of the number of clusters counted at the block's
  level (reading R2);
* the unit roundoffs of Table 1 (golden file) as the powers of two they
  print rounded, and 2^-4 for e4m3 (reading R6);

and assert that each block's format is the largest allowed one within the
bound (fp64 when none is).  Each configuration also checks that the plausible
mistakes (factor 2^{d l}, factor 1, and on the 2^d-tree 2^{l/2}) would
change the format of some block, so the test can fail on them.
"""
import json
import math
import os

import numpy as np
import pytest

import hh_workloads as W
from oracle import build as B
from oracle import formats as F
from oracle import matvec as M

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
ALL = W.F64 | W.F32 | W.F16 | W.BF16 | W.E4M3


def _table1_u():
    """Unit roundoffs from Table 1 as exact powers of two (the table prints
    them to three digits); e4m3: 2^-4 (reading R6 of the printed 2.5e-1)."""
    t = GOLD["table1_formats"]
    out = {}
    for name, fmt in (("fp64", F.FP64), ("fp32", F.FP32), ("fp16", F.FP16), ("bf16", F.BF16)):
        printed = t[name]["u"]
        e = round(-math.log2(printed))
        assert abs(2.0 ** -e / printed - 1) < 5e-3
        out[fmt] = 2.0 ** -e
    out[F.E4M3] = 2.0 ** -4
    return out


U_TABLE = _table1_u()


def _largest_within(bound, allowed):
    best, best_u = F.FP64, U_TABLE[F.FP64]
    for f in allowed:
        if U_TABLE[f] <= bound and U_TABLE[f] > best_u:
            best, best_u = f, U_TABLE[f]
    return best


def _check(H, factor_of, alternatives, allowed):
    """factor_of(block) -> the paper's level factor; alternatives: name ->
    wrong factor function.  Returns the number of blocks each alternative
    would store in another format."""
    nH = float(np.linalg.norm(M.dense_htilde(H)))
    changed = {k: 0 for k in alternatives}
    near = 0
    for b in H.lowrank:
        s = np.linalg.svd(b.U @ b.V.T, compute_uv=False)
        xi = math.sqrt(float(np.sum(s * s))) / nH
        if xi == 0.0:
            assert b.fmt == max(allowed, key=lambda f: U_TABLE[f])
            continue
        bound = H.tol / (factor_of(b) * xi)
        if any(abs(bound / U_TABLE[f] - 1) < 1e-9 for f in allowed):
            near += 1                                  # a tie: rounding of xi decides
            continue
        want = _largest_within(bound, allowed)
        assert b.fmt == want, (b.level, b.i, b.j, bound, b.fmt, want)
        for k, fn in alternatives.items():
            if _largest_within(H.tol / (fn(b) * xi), allowed) != want:
                changed[k] += 1
    assert near <= 1
    return changed


@pytest.mark.parametrize("dim,kernel,param,leaf,n,tol", [
    (2, W.LOG, 1.0, 16, 4096, 1e-2),
    (2, W.EXP, 1.0, 16, 4096, 1e-3),
    (2, W.LOG, 1.0, 16, 4096, 1e-4),
    (3, W.INV_R, 1.0, 64, 4096, 1e-2),
    (3, W.EXP, 1.0, 64, 4096, 1e-3),
])
def test_rule_level_factor_on_the_2d_tree_is_maximal(dim, kernel, param, leaf, n, tol):
    pts = 2.0 * W.points(n, dim, 500 + dim) - 1.0        # [-1,1]^d, as in Section 5
    ell = -1
    H = B.build(pts, kernel, param, leaf, math.sqrt(dim), ell, tol, ALL, tree_kind="2d")
    step = H.tree.step
    assert step == dim

    def tree_level(b):
        assert b.level % step == 0                     # blocks live on 2^d-tree levels
        return b.level // step

    paper = lambda b: 2.0 ** (dim * tree_level(b) / 2.0)          # noqa: E731
    alts = {"2^{dl}": lambda b: 2.0 ** (dim * tree_level(b)),
            "1": lambda b: 1.0,
            "2^{l/2}": lambda b: 2.0 ** (tree_level(b) / 2.0)}
    changed = _check(H, paper, alts, B.allowed_formats(ALL))
    assert len({b.fmt for b in H.lowrank}) >= 2
    for k, c in changed.items():
        assert c > 0, f"factor {k} is indistinguishable on this configuration"


def test_rule_level_factor_on_the_kd_tree_is_maximal():
    """Binary KD tree: the factor is the square root of the number of
    clusters at the block's level, counted in the tree (reading R2)."""
    pts = W.points(3000, 3, 611)
    H = B.build(pts, W.GAUSS, 0.02, 32, 1.0, 3, 1e-2, ALL)
    t = H.tree

    def clusters_at(level):
        return int(np.count_nonzero(t.size[(1 << level) - 1:(1 << (level + 1)) - 1] > 0))

    paper = lambda b: math.sqrt(clusters_at(b.level))            # noqa: E731
    alts = {"2^l": lambda b: 2.0 ** b.level, "1": lambda b: 1.0}
    changed = _check(H, paper, alts, B.allowed_formats(ALL))
    assert len({b.fmt for b in H.lowrank}) >= 2
    for k, c in changed.items():
        assert c > 0, f"factor {k} is indistinguishable on this configuration"
