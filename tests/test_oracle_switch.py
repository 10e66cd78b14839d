"""Algorithm 2 (optimal switching level): the oracle pinned against the
storage decomposition of Section 3.3 and against an exhaustive evaluation of
every level, and the library's implementation against the oracle."""
import numpy as np
import pytest

import hh_workloads as W
from oracle import build as B
from oracle import formats as F
from oracle import partition as PT
from oracle import switch as S
from oracle.tree import tree_depth, tree_depth_2d

ALL = W.F64 | W.F32 | W.F16 | W.BF16 | W.E4M3


def s1_minus_s2(Hs, Hh, ell):
    """S_1(ell) - S_2(ell) from the block lists (Eqs. 3.4 and 3.6): the H_s
    blocks below level ell and its dense leaf neighbours, against the H_h
    blocks that are not standard-admissible far field."""
    bits = lambda b: F.BITS[b.fmt] / 64.0  # noqa: E731
    s1 = sum(b.k * (b.m + b.n) * bits(b) for b in Hs.lowrank if b.level > ell) + \
        sum(d.m * d.n for d in Hs.dense if d.i != d.j)
    s2 = sum(b.k * (b.m + b.n) * bits(b) for b in Hh.lowrank if b.kind != PT.KIND_STD)
    return s1 - s2


def test_gain_is_s1_minus_s2_in_uniform_precision():
    """In uniform fp64 the far-field blocks of levels 1..ell and the dense
    diagonal are identical in H_s and H_h(ell), so the gain Algorithm 2 uses
    is exactly S_1(ell) - S_2(ell), and it is zero at ell = L."""
    pts = W.points(2048, 2, 21)
    L = tree_depth(2048, 32)
    Hs = B.build(pts, W.INV_R, 1.0, 32, 1.0, L, 1e-6, W.F64)
    ell_star, gains = S.optimal_switch_level(pts, W.INV_R, 1.0, 32, 1.0, 1e-6, W.F64)
    assert gains[L] == 0.0
    for ell, g in gains.items():
        if ell == L:
            continue
        Hh = B.build(pts, W.INV_R, 1.0, 32, 1.0, ell, 1e-6, W.F64)
        assert g == pytest.approx(Hs.storage() - Hh.storage(), rel=1e-12)
        assert g == pytest.approx(s1_minus_s2(Hs, Hh, ell), rel=1e-12, abs=1e-9)


@pytest.mark.parametrize("mask", [W.F64, ALL])
def test_walk_matches_exhaustive_evaluation(mask):
    """Algorithm 2 walks up from the leaves while the gain grows strictly:
    against the gains of every level 0..L it stops at the first level whose
    parent does not improve, and, the gains here being unimodal, that level
    is the maximizer of S_1 - S_2."""
    pts = W.points(2048, 3, 22)
    L = tree_depth(2048, 32)
    Hs = B.build(pts, W.EXP, 1.0, 32, 1.0, L, 1e-4, mask)
    every = {ell: S.storage_gain(pts, W.EXP, 1.0, 32, 1.0, 1e-4, mask, ell, Hs.storage()) for ell in range(L + 1)}
    assert every[L] == 0.0
    ell_star, gains = S.optimal_switch_level(pts, W.EXP, 1.0, 32, 1.0, 1e-4, mask)
    for ell, g in gains.items():
        assert g == pytest.approx(every[ell], rel=1e-12, abs=1e-9)
    for ell in range(L, ell_star, -1):
        assert every[ell - 1] > every[ell]
    assert ell_star == 0 or every[ell_star - 1] <= every[ell_star]
    seq = [every[ell] for ell in range(L, -1, -1)]
    peak = int(np.argmax(seq))
    if all(seq[i] < seq[i + 1] for i in range(peak)) and all(seq[i] >= seq[i + 1] for i in range(peak, L)):
        assert ell_star == max(every, key=every.get)


def test_mixed_precision_can_move_the_level():
    """The optimal level depends on the format bits (the paper's remark after
    Algorithm 2): for this matrix the adaptive representation prefers a finer
    switching level than uniform fp64."""
    pts = W.points(2048, 3, 13)
    e64, _ = S.optimal_switch_level(pts, W.EXP, 1.0, 32, 1.0, 1e-4, W.F64)
    eall, _ = S.optimal_switch_level(pts, W.EXP, 1.0, 32, 1.0, 1e-4, ALL)
    assert eall > e64


@pytest.mark.parametrize("case", [(4096, 2, W.INV_R, 64, 1e-6, W.F64, "kd"), (2048, 3, W.EXP, 32, 1e-4, ALL, "kd"),
                                  (4096, 2, W.LOG, 16, 1e-6, ALL, "2d")])
def test_library_matches_oracle(case):
    """hh_optimal_switch_level against the oracle: the same tree depth and
    level; gains equal up to the rank differences of the two compressions."""
    P = pytest.importorskip("paper_2604_09147_gb300")
    n, dim, kern, leaf, tol, mask, tree = case
    pts = W.points(n, dim, 13)
    ell, depth, gains = P.optimal_switch_level(pts, kern, 1.0, leaf, 1.0, tol, mask, tree=tree)
    o_ell, o_gains = S.optimal_switch_level(pts, kern, 1.0, leaf, 1.0, tol, mask, tree_kind=tree)
    assert depth == (tree_depth_2d(n, dim, leaf) if tree == "2d" else tree_depth(n, leaf))
    assert ell == o_ell
    assert set(gains) == set(o_gains)
    scale = max(abs(v) for v in o_gains.values())
    for l, g in o_gains.items():
        assert abs(gains[l] - g) <= 0.02 * scale


def test_library_search_equals_independent_builds():
    """The library's search shares block compressions between the levels it
    evaluates (a block's compression depends only on its clusters and tol):
    each gain equals, exactly, S_s - S_h(ell) from separate builds."""
    P = pytest.importorskip("paper_2604_09147_gb300")
    pts = W.points(3000, 3, 17)
    args = (W.EXP, 1.0, 32, 1.0)
    ell, depth, gains = P.optimal_switch_level(pts, *args, 1e-5, ALL)
    ss = P.HMatrix.build(pts, *args, depth, 1e-5, ALL, device=-1).info()["storage_amp"]
    assert len(gains) >= 2
    for l, g in gains.items():
        sh = P.HMatrix.build(pts, *args, l, 1e-5, ALL, device=-1).info()["storage_amp"]
        assert g == ss - sh
