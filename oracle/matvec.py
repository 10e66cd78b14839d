"""Algorithm 4: b = H_hat x, its transpose, and dense assemblies.

matvec   : b <- 0; for every admissible block b_I += U_hat (V_hat^T x_J);
           for every dense block b_I += H_IJ x_J.  All in float64 over the
           decoded stored factors, vectors permuted into tree order first and
           back afterwards.  Several right-hand sides are columns of x.
matvec_T : the transpose product x_bar_J += V_hat (U_hat^T y_bar_I) and
           x_bar_J += H_IJ^T y_bar_I (the backward of b = H_hat x).
dense_hhat / dense_h : the explicit matrices in the user's point order.

Parity: pinned by tests against the explicit dense H_hat (brute force), the
adjoint identity <y, H x> = <H^T y, x>, and against the exact kernel matrix
within the paper's bounds.
"""
from __future__ import annotations

import numpy as np

from .build import HMatrix
from .compress import kernel_entries


def _as2d(x):
    x = np.asarray(x, dtype=np.float64)
    return (x[:, None], True) if x.ndim == 1 else (x, False)


def matvec(H: HMatrix, x: np.ndarray) -> np.ndarray:
    x2, vec = _as2d(x)
    xt = x2[H.perm]
    bt = np.zeros_like(xt)
    for b in H.lowrank:
        if b.k == 0:
            continue
        t = b.Vd().T @ xt[b.col_off:b.col_off + b.n]
        bt[b.row_off:b.row_off + b.m] += b.Ud() @ t
    for d in H.dense:
        bt[d.row_off:d.row_off + d.m] += d.D @ xt[d.col_off:d.col_off + d.n]
    out = np.empty_like(bt)
    out[H.perm] = bt
    return out[:, 0] if vec else out


def matvec_T(H: HMatrix, y: np.ndarray) -> np.ndarray:
    y2, vec = _as2d(y)
    yt = y2[H.perm]
    xt = np.zeros_like(yt)
    for b in H.lowrank:
        if b.k == 0:
            continue
        t = b.Ud().T @ yt[b.row_off:b.row_off + b.m]
        xt[b.col_off:b.col_off + b.n] += b.Vd() @ t
    for d in H.dense:
        xt[d.col_off:d.col_off + d.n] += d.D.T @ yt[d.row_off:d.row_off + d.m]
    out = np.empty_like(xt)
    out[H.perm] = xt
    return out[:, 0] if vec else out


def dense_hhat(H: HMatrix) -> np.ndarray:
    """H_hat as an explicit N x N matrix in the user's point order."""
    A = np.zeros((H.n, H.n))
    for b in H.lowrank:
        A[b.row_off:b.row_off + b.m, b.col_off:b.col_off + b.n] += b.Ud() @ b.Vd().T
    for d in H.dense:
        A[d.row_off:d.row_off + d.m, d.col_off:d.col_off + d.n] += d.D
    out = np.empty_like(A)
    out[np.ix_(H.perm, H.perm)] = A
    return out


def dense_htilde(H: HMatrix) -> np.ndarray:
    """H~ (unrounded factors) as an explicit N x N matrix in the user's order."""
    A = np.zeros((H.n, H.n))
    for b in H.lowrank:
        A[b.row_off:b.row_off + b.m, b.col_off:b.col_off + b.n] += b.U @ b.V.T
    for d in H.dense:
        A[d.row_off:d.row_off + d.m, d.col_off:d.col_off + d.n] += d.D
    out = np.empty_like(A)
    out[np.ix_(H.perm, H.perm)] = A
    return out


def dense_h(points: np.ndarray, kernel: int, param: float) -> np.ndarray:
    """The exact kernel matrix H (Eq. 5.1) in the user's order."""
    return kernel_entries(kernel, param, points, points)


def h_rows_times(points: np.ndarray, kernel: int, param: float, rows: np.ndarray,
                 x: np.ndarray, chunk: int = 256) -> np.ndarray:
    """(H x)[rows] computed row by row from the kernel (brute force)."""
    x2, vec = _as2d(x)
    out = np.zeros((len(rows), x2.shape[1]))
    for s in range(0, len(rows), chunk):
        r = rows[s:s + chunk]
        out[s:s + len(r)] = kernel_entries(kernel, param, points[r], points) @ x2
    return out[:, 0] if vec else out
