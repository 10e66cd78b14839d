"""Algorithm 4: b = H_hat x, its transpose, and dense assemblies.

matvec   : b <- 0; for every admissible block b_I += U_hat (V_hat^T x_J);
           for every dense block b_I += H_IJ x_J.  All in float64 over the
           decoded stored factors, vectors permuted into tree order first and
           back afterwards.  Several right-hand sides are columns of x.
matvec_T : the transpose product x_bar_J += V_hat (U_hat^T y_bar_I) and
           x_bar_J += H_IJ^T y_bar_I (the backward of b = H_hat x).
matvec_wp: Algorithm 4 with every arithmetic operation in a working
           precision u (fp64, fp32 or fp16), the setting of the backward
           error experiment of Section 5 (the paper varies u to show that it
           must stay below about eps / N for Theorem 4.4 to hold): inputs
           and stored factors are rounded to u, each product and each sum of
           t_b = V^T x_J, of b_I += U t_b and of the dense blocks is rounded
           to u (NumPy's fp16 arithmetic rounds each operation's fp32 result,
           so a sum may be rounded twice), accumulated in the order of the
           loops below.
dense_hhat / dense_h : the explicit matrices in the user's point order.

Parity: pinned by tests against the explicit dense H_hat (brute force), the
adjoint identity <y, H x> = <H^T y, x>, and against the exact kernel matrix
within the paper's bounds; matvec_wp against matvec (u = fp64) and the
standard componentwise bound gamma_c |U||V|^T|x| of a computation with
paths of c operations in precision u (tests/test_oracle_working_precision.py).
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


WORKING_DTYPES = {0: np.float64, 1: np.float32, 2: np.float16}   # format codes FP64, FP32, FP16


def matvec_wp(H: HMatrix, x: np.ndarray, wp: int) -> np.ndarray:
    """b = H_hat x (one right-hand side) computed in working precision wp."""
    dt = WORKING_DTYPES[wp]
    xt = np.asarray(x, dtype=np.float64)[H.perm].astype(dt)
    bt = np.zeros(H.n, dtype=dt)
    for b in H.lowrank:
        if b.k == 0:
            continue
        U, V = b.Ud().astype(dt), b.Vd().astype(dt)
        xj = xt[b.col_off:b.col_off + b.n]
        t = np.zeros(b.k, dtype=dt)
        for r in range(b.n):                      # t = V^T x_J, one row at a time
            t = t + V[r] * xj[r]
        yi = bt[b.row_off:b.row_off + b.m]
        for c in range(b.k):                      # b_I += U t, one column at a time
            yi = yi + U[:, c] * t[c]
        bt[b.row_off:b.row_off + b.m] = yi
    for d in H.dense:
        D = d.D.astype(dt)
        xj = xt[d.col_off:d.col_off + d.n]
        yi = bt[d.row_off:d.row_off + d.m]
        for c in range(d.n):
            yi = yi + D[:, c] * xj[c]
        bt[d.row_off:d.row_off + d.m] = yi
    out = np.empty(H.n)
    out[H.perm] = bt.astype(np.float64)
    return out


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
