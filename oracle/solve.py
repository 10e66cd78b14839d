"""Conjugate gradients on the H_h product: the fast iterative solver that
the paper notes the product enables (Section 5, end).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Hestenes-Stiefel conjugate gradients for (H_hat + shift I) x = b with H_hat
applied by Algorithm 4 (matvec.py), in float64, stopping when the recursively
updated residual satisfies ||r_k|| <= rtol ||b||:
    r_0 = b - (H_hat + shift I) x_0,  p_0 = r_0
    alpha_k = (r_k . r_k) / (p_k . (H_hat + shift I) p_k)
    x_{k+1} = x_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k (H_hat + shift I) p_k
    p_{k+1} = r_{k+1} + ((r_{k+1} . r_{k+1}) / (r_k . r_k)) p_k

Parity: pinned in tests/test_oracle_solve.py against a dense direct solve of
the same operator and against the exact arithmetic property of conjugate
gradients on a small system (convergence within n steps).
"""
from __future__ import annotations

import numpy as np

from . import matvec as M


def cg(H, b: np.ndarray, shift: float = 0.0, rtol: float = 1e-8, max_iter: int = 1000,
       x0: np.ndarray | None = None, apply=None) -> tuple[np.ndarray, int, float]:
    """Returns (x, iterations, ||r|| / ||b||).  apply(v) overrides the operator
    (default: M.matvec(H, v) + shift v)."""
    op = apply if apply is not None else (lambda v: M.matvec(H, v) + shift * v)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - op(x)
    p = r.copy()
    bnorm = float(np.sqrt(b @ b))
    rr = float(r @ r)
    it = 0
    while it < max_iter and np.sqrt(rr) > rtol * bnorm:
        q = op(p)
        pq = float(p @ q)
        if not pq > 0.0:
            raise ValueError("conjugate gradients broke down: p^T A p <= 0")
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, (float(np.sqrt(rr)) / bnorm if bnorm > 0 else 0.0)
