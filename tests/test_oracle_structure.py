"""Pins of the oracle's cluster tree and hybrid partition (Sections 2-3)."""
import json
import math
import os

import numpy as np
import pytest

import hh_workloads as W
from oracle import partition as P
from oracle.tree import build_tree, tree_depth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("n,dim,leaf", [(4096, 2, 64), (5000, 3, 128), (3001, 2, 64), (100, 3, 128),
                                        (1, 2, 8), (129, 3, 128)])
def test_tree_is_complete_balanced_bisection(n, dim, leaf):
    pts = W.points(n, dim, 7)
    t = build_tree(pts, leaf)
    assert t.L == tree_depth(n, leaf)
    if n > leaf:
        assert t.L == math.ceil(math.log2(n / leaf))
    assert np.array_equal(np.sort(t.perm), np.arange(n))
    for l in range(t.L + 1):
        sizes = [t.rng(l, i)[1] for i in range(1 << l)]
        offs = [t.rng(l, i)[0] for i in range(1 << l)]
        assert sum(sizes) == n and offs == list(np.cumsum([0] + sizes[:-1]))
        assert set(sizes) <= {n // (1 << l), -(-n // (1 << l))}
    assert max(t.rng(t.L, i)[1] for i in range(1 << t.L)) <= leaf
    tp = pts[t.perm]
    for node in range((1 << t.L) - 1):
        o, s = int(t.off[node]), int(t.size[node])
        if s == 0:
            continue
        c = tp[o:o + s]
        assert np.allclose(t.lo[node], c.min(0)) and np.allclose(t.hi[node], c.max(0))
        ax = int(np.argmax(t.hi[node] - t.lo[node]))
        h = s // 2
        if 0 < h < s:
            assert c[:h, ax].max() <= c[h:, ax].min()       # median split on the widest axis


def test_admissibility_geometry_brackets_point_distances():
    rng = np.random.default_rng(0)
    pts = W.points(2048, 3, 3)
    t = build_tree(pts, 64)
    tp = pts[t.perm]
    for _ in range(200):
        l = int(rng.integers(1, t.L + 1))
        a, b = rng.integers(0, 1 << l, 2)
        na, nb = t.node(l, int(a)), t.node(l, int(b))
        A = tp[t.off[na]:t.off[na] + t.size[na]]
        B = tp[t.off[nb]:t.off[nb] + t.size[nb]]
        dAB = np.sqrt(((A[:, None, :] - B[None, :, :]) ** 2).sum(-1))
        dAA = np.sqrt(((A[:, None, :] - A[None, :, :]) ** 2).sum(-1))
        assert P.dist(t, na, nb) <= dAB.min() + 1e-15
        assert P.diam(t, na) >= dAA.max() - 1e-15
        assert P.diam(t, na) <= math.sqrt(3) * dAA.max() + 1e-15


def _coverage(t, part):
    n = int(t.size[0])
    cov = np.zeros((n, n), dtype=np.int32)
    for (l, i, j, _) in part.lowrank + part.dense:
        ro, m = t.rng(l, i)
        co, nn = t.rng(l, j)
        cov[ro:ro + m, co:co + nn] += 1
    return cov


@pytest.mark.parametrize("n,dim,leaf,ell", [(2048, 2, 64, 2), (2048, 3, 64, 3), (1500, 3, 50, 1),
                                            (2048, 2, 64, 0), (2048, 2, 64, 5), (900, 2, 64, 4)])
def test_partition_tiles_matrix_exactly_once(n, dim, leaf, ell):
    t = build_tree(W.points(n, dim, 11), leaf)
    ell = min(ell, t.L)
    part = P.partition(t, 1.0, ell)
    assert np.all(_coverage(t, part) == 1)


def test_hybrid_rules_per_level():
    t = build_tree(W.points(4096, 2, 5), 64)
    L, ell, eta = t.L, 3, 1.0
    part = P.partition(t, eta, ell)
    for (l, i, j, kind) in part.lowrank:
        ni, nj = t.node(l, i), t.node(l, j)
        if kind == P.KIND_STD:
            assert l <= ell and P.adm_s(t, ni, nj, eta)
            assert l == 1 or not P.adm_s(t, (ni - 1) // 2, (nj - 1) // 2, eta)   # parents inadmissible
        elif kind == P.KIND_FINER:
            assert l == ell and i != j and not P.adm_s(t, ni, nj, eta)
        else:
            assert kind == P.KIND_WEAK and l > ell and (i ^ 1) == j        # siblings only
    assert all(i == j and l == L for (l, i, j, _) in part.dense)         # dense only on the diagonal


def test_special_case_hodlr():
    """ell = 0: weak admissibility at every level (Section 3.2)."""
    t = build_tree(W.points(4096, 3, 6), 64)
    part = P.partition(t, 1.0, 0)
    per_level = {}
    for (l, i, j, kind) in part.lowrank:
        assert kind == P.KIND_WEAK and (i ^ 1) == j
        per_level[l] = per_level.get(l, 0) + 1
    assert per_level == {l: 1 << l for l in range(1, t.L + 1)}
    assert len(part.dense) == 1 << t.L and all(i == j for (_, i, j, _) in part.dense)


def test_special_case_hs():
    """ell = L: standard admissibility everywhere, dense leaf neighbours."""
    t = build_tree(W.points(4096, 2, 8), 64)
    part = P.partition(t, 1.0, t.L)
    assert all(k == P.KIND_STD for (_, _, _, k) in part.lowrank)
    nbr = [(l, i, j) for (l, i, j, k) in part.dense if k == P.KIND_NBR]
    assert nbr and all(not P.adm_s(t, t.node(l, i), t.node(l, j), 1.0) for (l, i, j) in nbr)
    assert np.all(_coverage(t, part) == 1)


def test_sparsity_constants_closed_form_match_paper():
    g = GOLD["sparsity_constants"]
    c = P.sparsity_closed_form(2, math.sqrt(2))
    assert c == pytest.approx((g["d2"]["C1"], g["d2"]["C2"], g["d2"]["C3"]))
    c = P.sparsity_closed_form(3, math.sqrt(3))
    assert c == pytest.approx((g["d3"]["C1"], g["d3"]["C2"], g["d3"]["C3"]))


def test_measured_csp():
    assert P.measured_csp([(1, 0), (1, 0), (1, 1), (2, 3)], 2) == [0, 2, 1]
