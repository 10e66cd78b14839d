"""Algorithm 4 in a working precision u (oracle/matvec.py: matvec_wp), the
setting of the backward error experiment in Section 5, pinned against the
exact-arithmetic cases and the standard rounding-error bound, and the
paper's observation that u must stay below about eps for Theorem 4.4's
bound to hold."""
import numpy as np
import pytest

import hh_workloads as W
from oracle import bounds as BD
from oracle import build as OB
from oracle import formats as F
from oracle import matvec as M
from oracle.tree import tree_depth

MASK = W.F64 | W.F32 | W.F16 | W.BF16
U_WP = {F.FP64: 2.0 ** -53, F.FP32: 2.0 ** -24, F.FP16: 2.0 ** -11}


@pytest.fixture(scope="module")
def small():
    pts = W.points(1200, 3, 90)
    return pts, OB.build(pts, W.INV_R, 1.0, 64, 1.0, 2, 1e-6, MASK)


def test_fp64_working_precision_is_algorithm_4(small):
    _, O = small
    x = W.rhs(1200, 1, "unit", 91)[:, 0]
    b = M.matvec(O, x)
    assert np.linalg.norm(M.matvec_wp(O, x, F.FP64) - b) <= 1e-14 * np.linalg.norm(b)


def test_exactly_representable_data_is_computed_exactly(small):
    """Integer factors, dense blocks and input whose every partial sum is an
    integer below 2^11: fp16 working precision rounds nothing, so it returns
    Algorithm 4's result exactly; any extra scaling or rounding would not."""
    _, O = small
    rng = np.random.default_rng(92)
    for b in O.lowrank:
        b.Us = rng.choice([-1.0, 0.0, 1.0], size=(b.m, b.k), p=[0.01, 0.98, 0.01])
        b.Vs = rng.choice([-1.0, 0.0, 1.0], size=(b.n, b.k), p=[0.01, 0.98, 0.01])
        b.exp_u = b.exp_v = 0
    for d in O.dense:
        d.D = rng.choice([-1.0, 0.0, 1.0], size=d.D.shape, p=[0.02, 0.96, 0.02])
    x = rng.integers(-2, 3, size=1200).astype(np.float64)
    b = M.matvec(O, x)
    assert np.abs(b).max() < 2 ** 11
    for wp in (F.FP16, F.FP32):
        assert np.array_equal(M.matvec_wp(O, x, wp), b)


@pytest.mark.parametrize("wp", [F.FP32, F.FP16])
def test_componentwise_rounding_bound(small, wp):
    """|b_u - b| <= gamma_c (sum_b |U_b| |V_b|^T |x_J| + |D| |x|) row by row,
    gamma_c = c u / (1 - c u), c = the longest chain of rounded operations
    into an entry (rounding of x, U, V; n_b products and sums in t_b; the
    k_b products and sums of every block and the dense columns added into
    the row); and the error is not zero, so rounding does take place.
    (Every row's blocks cover all N columns, so c >= 2N: fp16 is checked on
    200 points.)"""
    if wp == F.FP32:
        _, O = small
    else:  # every row's chain is at least 2N operations: small N keeps c u < 1/2
        O = OB.build(W.points(200, 3, 96), W.INV_R, 1.0, 32, 1.0, 1, 1e-3, MASK)
    x = W.rhs(O.n, 1, "unit", 93)[:, 0]
    b = M.matvec(O, x)
    bw = M.matvec_wp(O, x, wp)
    xt = np.abs(x[O.perm])
    mag = np.zeros(O.n)
    chain = np.zeros(O.n)
    for blk in O.lowrank:
        rows = slice(blk.row_off, blk.row_off + blk.m)
        mag[rows] += np.abs(blk.Ud()) @ (np.abs(blk.Vd()).T @ xt[blk.col_off:blk.col_off + blk.n])
        chain[rows] += 2 * blk.k + 2 * blk.n
    for d in O.dense:
        rows = slice(d.row_off, d.row_off + d.m)
        mag[rows] += np.abs(d.D) @ xt[d.col_off:d.col_off + d.n]
        chain[rows] += 2 * d.n
    c = chain + 3
    u = U_WP[wp]
    assert np.all(c * u < 0.5)
    gamma = c * u / (1 - c * u)
    err = np.abs(bw - b)[O.perm]
    assert np.all(err <= gamma * mag)
    assert np.linalg.norm(bw - b) >= 0.01 * u * np.linalg.norm(b)


def test_backward_error_needs_working_precision_below_eps():
    """Section 5's experiment (1/r in 3-D, x uniform in (0,1), ell = L - 1):
    the relative backward error ||H x - b|| / (||H|| ||x||) follows eps in
    fp64 working precision and stays within Theorem 4.4's bound; in fp32
    (u = 2^-24) and fp16 (u = 2^-11) it levels off near u once eps is below
    u, within the bound while eps is large and above it once eps is well
    below u."""
    n = 2000
    pts = W.points(n, 3, 94)
    x = W.rhs(n, 1, "unit", 95)[:, 0]
    Hd = M.dense_h(pts, W.INV_R, 1.0)
    hx = Hd @ x
    denom = np.linalg.norm(Hd) * np.linalg.norm(x)
    L = tree_depth(n, 64)
    be, bound = {}, {}
    for eps in (1e-2, 1e-5, 1e-10):
        O = OB.build(pts, W.INV_R, 1.0, 64, 1.0, L - 1, eps, MASK)
        bound[eps] = BD.thm44_measured(O)
        for wp in (F.FP64, F.FP32, F.FP16):
            bw = M.matvec_wp(O, x, wp)
            assert np.all(np.isfinite(bw))
            be[eps, wp] = np.linalg.norm(hx - bw) / denom
    for eps in bound:
        assert be[eps, F.FP64] <= bound[eps]
    assert be[1e-2, F.FP32] <= bound[1e-2] and be[1e-5, F.FP32] <= bound[1e-5]
    assert be[1e-10, F.FP32] > 10 * bound[1e-10]
    assert be[1e-2, F.FP16] <= bound[1e-2]
    assert be[1e-5, F.FP16] > 2 * bound[1e-5] and be[1e-10, F.FP16] > 10 * bound[1e-10]
    # the plateau: below u the error no longer follows eps
    assert be[1e-10, F.FP16] == pytest.approx(be[1e-5, F.FP16], rel=0.2)
    assert U_WP[F.FP32] < be[1e-10, F.FP32] < 100 * U_WP[F.FP32]
    assert U_WP[F.FP16] < be[1e-10, F.FP16] < 100 * U_WP[F.FP16]
