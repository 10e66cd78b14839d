"""The balanced 2^d-tree (Section 2.1) and the H_h partition on it: the
oracle pinned against the tree's definition, the closed-form sparsity
constants of Eqs. 2.3, 2.5 and 2.8, the exact coverage of N x N, Theorem
4.2's bound against the exact matrix, and the S_1 / S_2 > 1 trend of Table 2
(on the library's builder, which must match the oracle)."""
import math
from collections import Counter

import numpy as np
import pytest

import hh_workloads as W
from oracle import bounds as BD
from oracle import build as OB
from oracle import hhfile
from oracle import matvec as M
from oracle import partition as PT
from oracle.tree import build_tree_2d, tree_depth_2d

ALL = W.F64 | W.F32 | W.F16 | W.BF16 | W.E4M3


@pytest.mark.parametrize("dim", [2, 3])
def test_cells_halve_and_hold_their_points(dim):
    """Every binary level halves its cells along axis level mod d; d levels
    down a cell has become its 2^d congruent sub-cubes; every point lies in
    the cell of each node on its path (the upper face belongs to the upper
    cell)."""
    pts = W.points(3000, dim, 40) * 2 - 1
    t = build_tree_2d(pts, 16)
    assert t.step == dim and t.L % dim == 0 and t.L == dim * tree_depth_2d(3000, dim, 16)
    side = t.cell_hi[0] - t.cell_lo[0]
    assert np.allclose(side, side[0])                      # a hypercube
    assert np.all(t.cell_lo[0] <= pts.min(axis=0)) and np.all(pts.max(axis=0) <= t.cell_hi[0])
    nn = len(t.off)
    for node in range(nn):
        level = (node + 1).bit_length() - 1
        o, s = int(t.off[node]), int(t.size[node])
        p = pts[t.perm[o:o + s]]
        assert np.all(p >= t.cell_lo[node]) and np.all(p <= t.cell_hi[node])
        if level % dim == 0:                                # a 2^d-tree cell: congruent at its level
            assert np.allclose(t.cell_hi[node] - t.cell_lo[node], side / 2 ** (level // dim))
        if level == t.L:
            continue
        a = level % dim
        lc, rc = 2 * node + 1, 2 * node + 2
        mid = 0.5 * (t.cell_lo[node, a] + t.cell_hi[node, a])
        assert t.cell_hi[lc, a] == mid and t.cell_lo[rc, a] == mid
        assert t.size[lc] + t.size[rc] == s
        assert np.all(pts[t.perm[int(t.off[lc]):int(t.off[lc]) + int(t.size[lc])], a] < mid)
        assert np.all(pts[t.perm[int(t.off[rc]):int(t.off[rc]) + int(t.size[rc])], a] >= mid)
    assert sorted(t.perm.tolist()) == list(range(3000))


@pytest.mark.parametrize("dim,nside,leaf", [(2, 16, 4), (3, 8, 8)])
def test_regular_grid_is_perfectly_balanced(dim, nside, leaf):
    """On a regular grid every leaf holds n_max points and
    L = log_{2^d}(N / n_max) exactly (Section 2.1)."""
    ax = (np.arange(nside) + 0.5) / nside
    g = np.stack(np.meshgrid(*([ax] * dim), indexing="ij"), -1).reshape(-1, dim)
    t = build_tree_2d(g, leaf)
    L2 = round(math.log(len(g) / leaf, 2 ** dim))
    assert t.L == dim * L2
    assert np.all(t.size[-(1 << t.L):] == leaf)


@pytest.mark.parametrize("dim,n", [(2, 20000), (3, 30000)])
def test_sparsity_constants_attained(dim, n):
    """With eta = sqrt(d): the largest standard interaction list, neighbour
    list and weak interaction list of any cluster are C' = (2^d-1)(1+2sqrt(d)/eta)^d,
    C'' = (1+2sqrt(d)/eta)^d - 1 and C''' = 2^d - 1 (Eqs. 2.3, 2.5, 2.8):
    27 / 8 / 3 in 2-D and 189 / 26 / 7 in 3-D."""
    pts = W.points(n, dim, 31) * 2 - 1
    t = build_tree_2d(pts, 32)
    eta = math.sqrt(dim)
    cp, cpp, cppp = PT.sparsity_closed_form(dim, eta)
    hs = PT.partition(t, eta, t.L)                         # standard admissibility everywhere
    il = Counter((l, i) for (l, i, j, k) in hs.lowrank)
    nb = Counter((l, i) for (l, i, j, k) in hs.dense if k == PT.KIND_NBR)
    hw = PT.partition(t, eta, dim)                         # weak admissibility below tree level 1
    wk = Counter((l, i) for (l, i, j, k) in hw.lowrank if k == PT.KIND_WEAK)
    assert max(il.values()) == round(cp) and max(nb.values()) == round(cpp) and max(wk.values()) == round(cppp)


@pytest.mark.parametrize("dim,ell", [(2, 0), (2, 1), (2, 3), (3, 1), (3, 2)])
def test_partition_covers_each_entry_once(dim, ell):
    """Blocks at tree levels only (multiples of d), every entry of N x N in
    exactly one block, ell = L (H_s) and ell = 0 included."""
    pts = W.points(1500 if dim == 2 else 2500, dim, 33) * 2 - 1
    t = build_tree_2d(pts, 24)
    L2 = t.L // dim
    ell = min(ell, L2)
    P = PT.partition(t, math.sqrt(dim), dim * ell)
    n = len(pts)
    cover = np.zeros((n, n), dtype=np.int32)
    for (l, i, j, k) in P.lowrank + P.dense:
        assert l % dim == 0
        ro, m = t.rng(l, i)
        co, nc = t.rng(l, j)
        assert m > 0 and nc > 0
        cover[ro:ro + m, co:co + nc] += 1
    assert np.all(cover == 1)
    if ell == 0:
        assert all(k == PT.KIND_WEAK for (_, _, _, k) in P.lowrank)


@pytest.mark.parametrize("dim,kernel", [(2, W.LOG), (3, W.INV_R)])
def test_error_within_theorem_4_2_on_2d_tree(dim, kernel):
    pts = W.points(2000, dim, 5) * 2 - 1
    O = OB.build(pts, kernel, 1.0, 32, math.sqrt(dim), 1, 1e-6, ALL, tree_kind="2d")
    assert O.tree.step == dim and O.ell == dim
    Hd = M.dense_h(pts, kernel, 1.0)
    err = np.linalg.norm(Hd - M.dense_hhat(O)) / np.linalg.norm(Hd)
    assert err <= BD.thm42_measured(O)


@pytest.mark.parametrize("dim,kernel", [(2, W.LOG), (3, W.INV_R)])
def test_library_2d_tree_matches_oracle(tmp_path, dim, kernel):
    """hh_build_ex with the 2^d-tree against the oracle: same permutation,
    cells, partition, ranks within +-2 and formats; the file records d."""
    P = pytest.importorskip("paper_2604_09147_gb300")
    pts = W.points(2000, dim, 5) * 2 - 1
    H = P.HMatrix.build(pts, kernel, 1.0, 32, math.sqrt(dim), 1, 1e-6, ALL, device=-1, tree="2d")
    assert H.info()["tree_step"] == dim and H.info()["ell"] == dim
    path = str(tmp_path / "t2d.hhm")
    H.save(path)
    G = hhfile.read(path)
    O = OB.build(pts, kernel, 1.0, 32, math.sqrt(dim), 1, 1e-6, ALL, tree_kind="2d")
    assert G.tree.step == dim
    assert np.array_equal(G.perm, O.perm)
    assert np.array_equal(G.tree.off, O.tree.off) and np.array_equal(G.tree.size, O.tree.size)
    assert np.array_equal(G.tree.lo, O.tree.lo) and np.array_equal(G.tree.hi, O.tree.hi)
    kg = {(b.level, b.i, b.j): b for b in G.lowrank}
    ko = {(b.level, b.i, b.j): b for b in O.lowrank}
    assert set(kg) == set(ko)
    assert {(d.i, d.j) for d in G.dense} == {(d.i, d.j) for d in O.dense}
    assert max(abs(kg[k].k - ko[k].k) for k in ko) <= 2
    assert np.mean([kg[k].fmt == ko[k].fmt for k in ko]) >= 0.99


def test_table_2_trend_s1_over_s2_above_one(tmp_path):
    """Table 2's observation on the oct-tree: for 1/r in [-1,1]^3 with
    ell = L - 1, S_1(ell) / S_2(ell) > 1 at every tolerance, so the H_h
    matrix stores less than the H_s matrix (here N = 4,096, n_max = 64,
    L = 2, uniform fp64; the library's builder)."""
    P = pytest.importorskip("paper_2604_09147_gb300")
    pts = W.points(4096, 3, 64) * 2 - 1
    for tol in (1e-2, 1e-6, 1e-10):
        mats = []
        for ell in (2, 1):
            H = P.HMatrix.build(pts, W.INV_R, 1.0, 64, math.sqrt(3), ell, tol, W.F64, device=-1, tree="2d")
            path = str(tmp_path / f"m{ell}.hhm")
            H.save(path)
            mats.append((H.info()["storage_amp"], hhfile.read(path)))
        (ss, Gs), (sh, Gh) = mats
        assert Gs.ell == Gs.tree.L == 6 and Gh.ell == 3
        s1 = sum(b.k * (b.m + b.n) for b in Gs.lowrank if b.level > Gh.ell) + \
            sum(d.m * d.n for d in Gs.dense if d.i != d.j)
        s2 = sum(b.k * (b.m + b.n) for b in Gh.lowrank if b.kind != PT.KIND_STD)
        assert ss - sh == pytest.approx(s1 - s2, rel=1e-9)
        assert s1 / s2 > 1.0


@pytest.mark.parametrize("name", ["one_point", "n_equals_leaf", "duplicates", "one_dim", "line_in_3d"])
def test_degenerate_point_sets(tmp_path, name):
    """One point, a single leaf, repeated points, d = 1 and a line in 3-D
    (most cells empty): the library and the oracle agree and the blocks
    cover N x N once."""
    P = pytest.importorskip("paper_2604_09147_gb300")
    pts = {"one_point": np.array([[0.5, 0.5]]),
           "n_equals_leaf": W.points(32, 2, 1),
           "duplicates": np.repeat(W.points(40, 3, 2), 5, axis=0),
           "one_dim": W.points(500, 1, 3),
           "line_in_3d": np.c_[np.linspace(0, 1, 300), np.zeros(300), np.zeros(300)]}[name]
    eta = math.sqrt(pts.shape[1])
    H = P.HMatrix.build(pts, W.EXP, 1.0, 32, eta, -1, 1e-6, ALL, device=-1, tree="2d")
    path = str(tmp_path / "d.hhm")
    H.save(path)
    G = hhfile.read(path)
    O = OB.build(pts, W.EXP, 1.0, 32, eta, -1, 1e-6, ALL, tree_kind="2d")
    assert np.array_equal(G.perm, O.perm)
    assert {(b.level, b.i, b.j) for b in G.lowrank} == {(b.level, b.i, b.j) for b in O.lowrank}
    n = len(pts)
    cover = np.zeros((n, n), dtype=np.int32)
    for b in G.lowrank:
        cover[b.row_off:b.row_off + b.m, b.col_off:b.col_off + b.n] += 1
    for d in G.dense:
        cover[d.row_off:d.row_off + d.m, d.col_off:d.col_off + d.n] += 1
    assert np.all(cover == 1)


@pytest.mark.parametrize("kernel,param", [(W.INV_R, 1.0), (W.GAUSS, 2.0)])
def test_library_global_error_follows_eps(tmp_path, kernel, param):
    """Section 5.1's experiment on the library's builder (2^d-tree, eta = sqrt(3),
    ell = L - 1, all five formats): ||H - H_hat||_F / ||H||_F stays within
    Theorem 4.2's bound and follows eps (not far below it either)."""
    P = pytest.importorskip("paper_2604_09147_gb300")
    pts = W.points(2500, 3, 9) * 2 - 1
    Hd = M.dense_h(pts, kernel, param)
    for eps in (1e-2, 1e-6):
        H = P.HMatrix.build(pts, kernel, param, 64, math.sqrt(3), 1, eps, ALL, device=-1, tree="2d")
        path = str(tmp_path / "g.hhm")
        H.save(path)
        err = np.linalg.norm(Hd - M.dense_hhat(hhfile.read(path))) / np.linalg.norm(Hd)
        assert 0.1 * eps <= err <= H.info()["bound_thm42"]


def test_hodlr_h_s_and_h_h_storage(tmp_path):
    """Section 3's comparison (1/r in 2-D, uniform fp64, library builder):
    weak admissibility admits near-field blocks whose ranks grow with the
    cluster size, so HODLR's low-rank storage exceeds H_s's (far field only)
    at both tolerances, and H_h stores less than H_s with its leaf neighbours
    dense (standard admissibility alone)."""
    P = pytest.importorskip("paper_2604_09147_gb300")
    pts = W.points(16384, 2, 21) * 2 - 1
    store = {}
    for eps in (1e-2, 1e-8):
        for name, ell in (("s", 4), ("h", 3), ("hodlr", 0)):
            H = P.HMatrix.build(pts, W.INV_R, 1.0, 64, math.sqrt(2), ell, eps, W.F64, device=-1, tree="2d")
            assert H.info()["L"] == 2 * 4
            path = str(tmp_path / "s.hhm")
            H.save(path)
            G = hhfile.read(path)
            nbr = name == "s"
            lr = sum(b.k * (b.m + b.n) for b in G.lowrank if not (nbr and b.kind == PT.KIND_NBR))
            dn = sum(d.m * d.n for d in G.dense) + sum(b.m * b.n for b in G.lowrank if nbr and b.kind == PT.KIND_NBR)
            store[name, eps] = (lr, dn)
    for eps in (1e-2, 1e-8):
        assert store["hodlr", eps][0] > store["s", eps][0]
        assert sum(store["h", eps]) < sum(store["s", eps])
