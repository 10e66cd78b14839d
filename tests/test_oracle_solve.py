"""Conjugate gradients on the H_h product (oracle/solve.py): pinned against a
dense direct solve and against the finite termination of conjugate
gradients."""
import numpy as np
import pytest

import hh_workloads as W
from oracle import build as OB
from oracle import matvec as M
from oracle import solve as S


def test_cg_terminates_on_small_spd_system():
    """In exact arithmetic conjugate gradients solves an n x n SPD system in at
    most n steps; in floating point on a well-conditioned 30 x 30 system it
    reaches 1e-12 within n steps and matches the direct solve."""
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    A = Q @ np.diag(np.linspace(1.0, 10.0, 30)) @ Q.T
    b = rng.standard_normal(30)
    x, it, res = S.cg(None, b, rtol=1e-12, max_iter=100, apply=lambda v: A @ v)
    assert it <= 30 and res <= 1e-12
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)


@pytest.mark.parametrize("mask", [W.F64, W.F64 | W.F32 | W.F16 | W.BF16 | W.E4M3])
def test_cg_on_hh_matches_direct_solve(mask):
    """(H_hat + I) x = b for the SPD Gaussian kernel: the CG iterate agrees
    with the dense solve of the same (nearly symmetric) operator to the
    requested tolerance."""
    pts = W.points(1500, 3, 51)
    O = OB.build(pts, W.GAUSS, 0.05, 64, 1.0, 2, 1e-8, mask)
    b = W.rhs(1500, 1, "uniform", 52)[:, 0]
    x, it, res = S.cg(O, b, shift=1.0, rtol=1e-10, max_iter=500)
    assert res <= 1e-10 and 0 < it < 500
    A = M.dense_hhat(O) + np.eye(1500)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    assert np.linalg.norm(A @ x - b) <= 1e-8 * np.linalg.norm(b)


def test_cg_reports_breakdown_on_indefinite_operator():
    """p^T A p <= 0 (an indefinite operator) stops the iteration with an error
    instead of returning a meaningless iterate, as the library's solver does."""
    A = np.diag([1.0, -1.0])
    with pytest.raises(ValueError):
        S.cg(None, np.array([1.0, 1.0]), rtol=1e-12, max_iter=10, apply=lambda v: A @ v)
