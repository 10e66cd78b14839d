"""Pins of the oracle's compression, precision assignment, matvec and bounds
against closed forms, brute force and the paper's lemmas and theorems."""
import json
import math
import os

import numpy as np
import pytest

import hh_workloads as W
from oracle import bounds as BD
from oracle import build as B
from oracle import compress as C
from oracle import formats as F
from oracle import hhfile
from oracle import matvec as M
from oracle import partition as P

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
ALL = W.F64 | W.F32 | W.F16 | W.BF16 | W.E4M3


def test_kernel_entries_closed_forms():
    x = np.array([[0.0, 0.0, 0.0]])
    y = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 0.0]])
    assert C.kernel_entries(C.EXP, 2.0, x, y)[0] == pytest.approx([math.exp(-2.5), 1.0])
    assert C.kernel_entries(C.GAUSS, 0.5, x, y)[0] == pytest.approx([math.exp(-50.0), 1.0])
    assert list(C.kernel_entries(C.INV_R, 1.0, x, y)[0]) == [0.2, 0.0]
    assert list(C.kernel_entries(C.INV_R2, 1.0, x, y)[0]) == pytest.approx([0.04, 0.0])
    assert C.kernel_entries(C.LOG, 1.0, x, y)[0] == pytest.approx([math.log(5.0), 0.0])


def test_svd_truncation_is_the_optimal_rank():
    """Eckart-Young: the kept rank is the smallest meeting the eps tail bound."""
    rng = np.random.default_rng(0)
    a = rng.standard_normal((120, 90)) @ np.diag(np.logspace(0, -12, 90)) @ rng.standard_normal((90, 90))
    for eps in (1e-2, 1e-6, 1e-10):
        U, V, s = C.svd_truncate(a, eps)
        r = U.shape[1]
        err = np.linalg.norm(a - U @ V.T)
        assert err <= eps * np.linalg.norm(a) * (1 + 1e-10)
        assert np.allclose(U.T @ U, np.eye(r), atol=1e-12)
        sv = np.linalg.svd(a, compute_uv=False)
        assert np.sqrt(np.sum(sv[r - 1:] ** 2)) > eps * np.linalg.norm(a)   # rank r-1 is not enough
    assert C.truncation_rank(np.zeros(4), 0.1) == 0


@pytest.mark.parametrize("kernel,param,dim", [(C.INV_R, 1.0, 3), (C.EXP, 1.0, 2), (C.GAUSS, 0.01, 3),
                                              (C.LOG, 1.0, 2)])
def test_aca_path_meets_block_tolerance(kernel, param, dim):
    """Eq. 2.1 for the ACA + recompression path on adjacent clusters."""
    pts = W.points(2048, dim, 21)
    order = np.argsort(pts[:, 0], kind="stable")
    xs, ys = pts[order[:1024]], pts[order[1024:]]              # two touching halves
    assert xs.shape[0] * ys.shape[0] > C.DENSE_SVD_MAX
    A = C.kernel_entries(kernel, param, xs, ys)
    for eps in (1e-4, 1e-8):
        U, V, s = C.lr_compress(kernel, param, xs, ys, eps)
        assert np.linalg.norm(A - U @ V.T) <= eps * np.linalg.norm(A)
        assert np.allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-10)
        assert np.sqrt(np.sum(s ** 2)) == pytest.approx(np.linalg.norm(U @ V.T), rel=1e-10)


def _build(n, dim, kernel, param, leaf, ell, tol, mask, seed=31):
    pts = W.points(n, dim, seed)
    return pts, B.build(pts, kernel, param, leaf, 1.0, ell, tol, mask)


@pytest.mark.parametrize("dim,kernel,param,ell", [(2, C.EXP, 1.0, 2), (3, C.INV_R, 1.0, 2),
                                                  (2, C.LOG, 1.0, 0), (3, C.GAUSS, 0.05, 5)])
def test_lemma31_and_algorithm5(dim, kernel, param, ell):
    """Lemma 3.1: ||H - H~|| <= eps ||H||; Algorithm 5: ||H~|| from blocks."""
    n = 2048
    for tol in (1e-3, 1e-7):
        pts, H = _build(n, dim, kernel, param, 64, ell, tol, W.F64)
        Hd = M.dense_h(pts, kernel, param)
        Ht = M.dense_htilde(H)
        assert np.linalg.norm(Hd - Ht) <= tol * np.linalg.norm(Hd)
        # with ell == L, Algorithm 5 adds leaf neighbours densely even when
        # Section 4.3 then stores them low rank: equal up to eps, not rounding
        assert H.norm_Ht == pytest.approx(np.linalg.norm(Ht), rel=tol if H.ell == H.L else 1e-12)
        for b in H.lowrank:                       # each admissible block, Eq. 4.1
            Hb = C.kernel_entries(kernel, param, pts[H.perm[b.row_off:b.row_off + b.m]],
                                  pts[H.perm[b.col_off:b.col_off + b.n]])
            assert np.linalg.norm(Hb - b.U @ b.V.T) <= tol * np.linalg.norm(Hb) * (1 + 1e-9)


@pytest.mark.parametrize("dim,kernel,param,ell,tol", [(2, C.LOG, 1.0, 2, 1e-2), (3, C.INV_R, 1.0, 3, 1e-4),
                                                      (3, C.GAUSS, 0.01, 2, 1e-3), (3, C.EXP, 1.0, 5, 1e-2),
                                                      (3, C.INV_R2, 1.0, 0, 1e-3)])
def test_theorem42_and_theorem44(dim, kernel, param, ell, tol):
    """Mixed precision global error (Thm 4.2) and matvec backward error (Thm 4.4)."""
    pts, H = _build(2048, dim, kernel, param, 64, ell, tol, ALL)
    assert sum(1 for b in H.lowrank if b.fmt != F.FP64) > 0
    Hd = M.dense_h(pts, kernel, param)
    Hh = M.dense_hhat(H)
    nH = np.linalg.norm(Hd)
    err = np.linalg.norm(Hd - Hh) / nH
    assert err <= BD.thm42_measured(H)
    # a-posteriori form of the rounding part (Eq. 4.3) bounds ||H~ - H_hat|| exactly
    assert np.linalg.norm(M.dense_htilde(H) - Hh) / H.norm_Ht <= BD.aposteriori_rounding(H) * (1 + 1e-9)
    x = W.rhs(2048, 1, "unit", 5)[:, 0]
    b = M.matvec(H, x)
    assert np.linalg.norm(Hd @ x - b) / (nH * np.linalg.norm(x)) <= BD.thm44_measured(H)


def test_format_assignment_follows_rule_and_is_monotone_in_xi():
    pts, H = _build(4096, 3, C.GAUSS, 0.01, 64, 3, 1e-3, ALL)
    allowed = B.allowed_formats(ALL)
    seen = set()
    for b in H.lowrank:
        tau = B.block_tau(H.tol, b.level, b.norm, H.norm_Ht)
        assert b.fmt == F.choose_format(tau, allowed)
        assert F.UNIT_ROUNDOFF[b.fmt] <= tau or b.fmt == F.FP64
        seen.add(b.fmt)
    assert len(seen) >= 3
    for l in range(1, H.L + 1):                    # same level: smaller xi never gets a finer format
        bl = sorted((b for b in H.lowrank if b.level == l), key=lambda b: b.norm)
        us = [F.UNIT_ROUNDOFF[b.fmt] for b in bl]
        assert all(a >= c for a, c in zip(us, us[1:]))


def test_small_eps_selects_only_fp64():
    """Section 5.2: for 1e-12 <= eps <= 1e-10 only fp64 is selected."""
    for eps in GOLD["only_fp64_range"]["eps"]:
        _, H = _build(1024, 3, C.INV_R, 1.0, 64, 2, eps, ALL)
        assert all(b.fmt == F.FP64 for b in H.lowrank)


def test_beneficial_compression_worked_example():
    g = GOLD["beneficial_compression_example"]
    m, n, p = g["m"], g["n"], g["p"]
    assert p * (m + n) == g["fp64_lowrank_words"] and p * (m + n) * 32 / 64 == g["fp32_lowrank_words"]
    assert not B.lowrank_pays_off(p, m, n, 64)
    assert B.lowrank_pays_off(p, m, n, 32)
    assert m * n == g["dense_words"]


def test_hs_special_case_compresses_neighbours_only_when_paying_off():
    pts, H = _build(2048, 2, C.EXP, 1.0, 64, 5, 1e-2, ALL)
    assert H.ell == H.L
    nbr = [b for b in H.lowrank if b.kind == P.KIND_NBR]
    assert nbr
    for b in nbr:
        assert B.lowrank_pays_off(b.k, b.m, b.n, F.BITS[b.fmt])
    Hd = M.dense_h(pts, C.EXP, 1.0)
    assert np.linalg.norm(Hd - M.dense_hhat(H)) / np.linalg.norm(Hd) <= BD.thm42_measured(H)


def test_storage_criterion_common_terms():
    """S_s - S_h = S_1(ell) - S_2(ell): the far-field blocks of levels 1..ell
    and the dense diagonal are common to H_s and H_h (Section 3.3)."""
    pts = W.points(4096, 2, 13)
    Hh = B.build(pts, C.INV_R, 1.0, 64, 1.0, 3, 1e-6, W.F64)
    Hs = B.build(pts, C.INV_R, 1.0, 64, 1.0, Hh.L, 1e-6, W.F64)
    ell = Hh.ell
    common_h = {(b.level, b.i, b.j): b.k for b in Hh.lowrank if b.kind == P.KIND_STD}
    common_s = {(b.level, b.i, b.j): b.k for b in Hs.lowrank if b.level <= ell}
    assert common_h == common_s
    S1 = sum(b.k * (b.m + b.n) for b in Hs.lowrank if b.level > ell) + \
        sum(d.m * d.n for d in Hs.dense if d.i != d.j)
    S2 = sum(b.k * (b.m + b.n) for b in Hh.lowrank if b.kind != P.KIND_STD)
    assert Hs.storage() - Hh.storage() == pytest.approx(S1 - S2, rel=1e-12)
    assert (Hs.storage() > Hh.storage()) == (S1 / S2 > 1)


def test_matvec_equals_dense_hhat_and_transpose():
    pts, H = _build(1500, 3, C.INV_R, 1.0, 40, 2, 1e-3, ALL)
    A = M.dense_hhat(H)
    x = W.rhs(1500, 3, "uniform", 1)
    y = W.rhs(1500, 3, "normal", 2)
    assert np.allclose(M.matvec(H, x), A @ x, rtol=0, atol=1e-12 * np.abs(A).sum(1).max())
    assert np.allclose(M.matvec_T(H, y), A.T @ y, rtol=0, atol=1e-12 * np.abs(A).sum(0).max())
    assert np.allclose(M.matvec(H, x[:, 0]), M.matvec(H, x)[:, 0])
    lhs = np.sum(y * M.matvec(H, x))
    rhs = np.sum(M.matvec_T(H, y) * x)
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_small_n_is_a_single_dense_block():
    pts, H = _build(50, 2, C.EXP, 1.0, 64, -1, 1e-6, W.F64)
    assert H.L == 0 and not H.lowrank and len(H.dense) == 1
    x = W.rhs(50, 1, "uniform", 3)[:, 0]
    assert np.allclose(M.matvec(H, x), M.dense_h(pts, C.EXP, 1.0) @ x, rtol=1e-14, atol=1e-14)


def test_file_roundtrip(tmp_path):
    pts, H = _build(3001, 3, C.GAUSS, 0.02, 64, 3, 1e-3, ALL)
    path = str(tmp_path / "h.hhm")
    hhfile.write(H, path)
    G = hhfile.read(path)
    assert np.array_equal(G.perm, H.perm) and np.array_equal(G.points, H.points)
    assert len(G.lowrank) == len(H.lowrank) and len(G.dense) == len(H.dense)
    for a, b in zip(H.lowrank, G.lowrank):
        assert (a.fmt, a.exp_u, a.exp_v, a.row_off, a.col_off) == (b.fmt, b.exp_u, b.exp_v, b.row_off, b.col_off)
        assert np.array_equal(a.Us, b.Us) and np.array_equal(a.Vs, b.Vs)
    x = W.rhs(3001, 2, "uniform", 4)
    assert np.array_equal(M.matvec(H, x), M.matvec(G, x))
