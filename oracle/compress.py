"""Kernel functions and LRcompression.

Kernel matrix (Eq. 5.1): H_ij = f(||x_i - x_j||_2), with H_ii = 0 when f is
singular at 0 (here: any r == 0 of a singular f gives 0).  Kernels of
Section 5 and the workload presets: exp(-r/p), 1/r, exp(-r^2/p), log r, 1/r^2.

LRcompression(H_IJ, eps) (Section 2.2, Eq. 2.1): returns U (|I| x p, columns
orthonormal) and V (|J| x p) with ||H_IJ - U V^T||_F <= eps ||H_IJ||_F.
The singular values Sigma go into V (reading R8), so ||U V^T||_F^2 =
trace(Sigma^2), the quantity Algorithm 5 accumulates.

  * small blocks (m*n <= DENSE_SVD_MAX): the truncated SVD of the dense block,
    as in the paper's experiments (Section 5): the smallest rank r whose
    discarded tail satisfies sqrt(sum_{i>r} s_i^2) <= eps sqrt(sum_i s_i^2);
  * larger blocks: ACA with partial pivoting (start row = the cluster's first
    index; stop once ||u_k|| ||v_k|| <= (eps/100) ||S_k||_F, with the running
    Frobenius estimate, has held on 3 consecutive steps), then QR of both
    factors, SVD of the k x k core and the same tail truncation at 0.99 eps, so
    that ACA's share and the truncation share add up to eps (reading R4).
    ACA's stopping test is a heuristic; the 1/100 share and the 3-step
    patience are what the dense-error tests need on touching clusters of
    singular kernels, where the plain eps/10 test stops early.

Parity: the dense path is the library SVD (pinned against the exact optimum
by Eckart-Young in tests); the ACA path is pinned by dense comparison of the
block error on sizes the test can form densely.
"""
from __future__ import annotations

import numpy as np

DENSE_SVD_MAX = 1 << 18
ACA_SHARE = 0.01
ACA_PATIENCE = 3

EXP, INV_R, GAUSS, LOG, INV_R2 = 0, 1, 2, 3, 4
SINGULAR = {INV_R, LOG, INV_R2}


def kernel_entries(kernel: int, param: float, xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    """Dense block f(||x_a - y_b||) for point sets xs (m, d) and ys (n, d)."""
    d2 = np.zeros((xs.shape[0], ys.shape[0]))
    for a in range(xs.shape[1]):
        diff = xs[:, a][:, None] - ys[:, a][None, :]
        d2 = d2 + diff * diff
    r = np.sqrt(d2)
    if kernel == EXP:
        return np.exp(-r / param)
    if kernel == GAUSS:
        return np.exp(-(r * r) / param)
    zero = r == 0.0
    rs = np.where(zero, 1.0, r)
    if kernel == INV_R:
        v = 1.0 / rs
    elif kernel == LOG:
        v = np.log(rs)
    elif kernel == INV_R2:
        v = 1.0 / (rs * rs)
    else:
        raise ValueError(kernel)
    return np.where(zero, 0.0, v)


def truncation_rank(s: np.ndarray, eps: float) -> int:
    """Smallest r with sqrt(sum_{i>=r} s_i^2) <= eps * sqrt(sum_i s_i^2)."""
    s2 = np.asarray(s, dtype=np.float64) ** 2
    total = float(np.sum(s2))
    if total == 0.0:
        return 0
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])   # tail[r] = sum_{i>=r}
    ok = np.nonzero(np.sqrt(tail) <= eps * np.sqrt(total))[0]
    return int(ok[0])


def svd_truncate(a: np.ndarray, eps: float):
    """Truncated SVD: (U orthonormal, V = Z Sigma, singular values kept)."""
    w, s, zt = np.linalg.svd(a, full_matrices=False)
    r = truncation_rank(s, eps)
    return w[:, :r].copy(), (zt[:r].T * s[:r]).copy(), s[:r].copy()


def aca(entry_row, entry_col, m: int, n: int, tol: float, patience: int = 3):
    """ACA with partial pivoting: A ~= U V^T, U (m,k) residual columns,
    V (n,k) residual rows divided by the pivot.  Stops once the rank-one
    update is below tol * ||S_k||_F on `patience` consecutive steps."""
    kmax = min(m, n)
    cap = min(kmax, 64)
    U = np.zeros((m, cap))
    V = np.zeros((n, cap))
    k = 0
    used = np.zeros(m, dtype=bool)
    i = 0
    norm2 = 0.0
    calm = 0
    while k < kmax:
        row = entry_row(i) - V[:, :k] @ U[i, :k]
        used[i] = True
        j = int(np.argmax(np.abs(row)))
        piv = row[j]
        if piv == 0.0:
            free = np.nonzero(~used)[0]
            if free.size == 0:
                break
            i = int(free[0])
            continue
        v = row / piv
        u = entry_col(j) - U[:, :k] @ V[j, :k]
        cross = float(np.dot(U[:, :k].T @ u, V[:, :k].T @ v)) if k else 0.0
        uu, vv = float(np.dot(u, u)), float(np.dot(v, v))
        norm2 = norm2 + 2.0 * cross + uu * vv
        if k == cap:
            cap = min(kmax, 2 * cap)
            U = np.concatenate([U, np.zeros((m, cap - k))], axis=1)
            V = np.concatenate([V, np.zeros((n, cap - k))], axis=1)
        U[:, k] = u
        V[:, k] = v
        k += 1
        if np.sqrt(uu) * np.sqrt(vv) <= tol * np.sqrt(max(norm2, 0.0)):
            calm += 1
            if calm >= patience:
                break
        else:
            calm = 0
        if np.all(used):
            break
        i = int(np.argmax(np.where(used, -1.0, np.abs(u))))
    return U[:, :k].copy(), V[:, :k].copy()


def recompress(U: np.ndarray, V: np.ndarray, eps: float):
    """QR of both factors, SVD of the core, tail truncation at eps."""
    if U.shape[1] == 0:
        return U, V, np.zeros(0)
    qu, ru = np.linalg.qr(U)
    qv, rv = np.linalg.qr(V)
    w, s, zt = np.linalg.svd(ru @ rv.T)
    r = truncation_rank(s, eps)
    return qu @ w[:, :r], (qv @ zt[:r].T) * s[:r], s[:r].copy()


def lr_compress(kernel: int, param: float, xs: np.ndarray, ys: np.ndarray, eps: float):
    """LRcompression of the block f(xs, ys): (U, V, singular values)."""
    m, n = xs.shape[0], ys.shape[0]
    if m * n <= DENSE_SVD_MAX:
        return svd_truncate(kernel_entries(kernel, param, xs, ys), eps)
    U, V = aca(lambda i: kernel_entries(kernel, param, xs[i:i + 1], ys)[0],
               lambda j: kernel_entries(kernel, param, xs, ys[j:j + 1])[:, 0],
               m, n, ACA_SHARE * eps, ACA_PATIENCE)
    return recompress(U, V, (1.0 - ACA_SHARE) * eps)
