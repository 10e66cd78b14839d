"""Error bounds of Section 4.

Lemma 3.1:    ||H - H~|| <= eps ||H||.
Theorem 4.2:  ||H - H_hat|| <~ (2 sqrt(l C' + C'' + (L - l) C''') + 1) eps ||H||,
              here with the measured sparsity constants of the built
              partition (reading R3): (2 sqrt(sum_l C_sp(l)) + 1) eps.
Per-block a-posteriori form of Eq. 4.3: ||H~_IJ - H_hat_IJ|| <=
              (2 + sqrt(p) u) u ||H~_IJ||, summed in squares, plus eps.
Theorem 4.4:  backward error ||Delta H|| <= 2 (2 sqrt(...) + 1) eps ||H||;
              metric ||H x - b|| / (||H|| ||x||) (Section 5.3).

Parity: closed forms; checked numerically against dense matrices in tests.
"""
from __future__ import annotations

import math

from . import formats as F
from .build import HMatrix
from .partition import sparsity_closed_form


def thm42_paper(d: int, eta: float, ell: int, L: int, eps: float) -> float:
    c1, c2, c3 = sparsity_closed_form(d, eta)
    return (2.0 * math.sqrt(ell * c1 + c2 + (L - ell) * c3) + 1.0) * eps


def thm42_measured(H: HMatrix) -> float:
    return (2.0 * math.sqrt(sum(H.csp())) + 1.0) * H.tol


def thm44_measured(H: HMatrix) -> float:
    return 2.0 * thm42_measured(H)


def aposteriori_rounding(H: HMatrix) -> float:
    """sqrt(sum_b ((2 + sqrt(p_b) u_b) u_b ||H~_b||)^2) / ||H~||  (Eq. 4.3 summed)."""
    s = 0.0
    for b in H.lowrank:
        if b.fmt == F.FP64:
            continue
        u = F.UNIT_ROUNDOFF[b.fmt]
        s += ((2.0 + math.sqrt(b.k) * u) * u * b.norm) ** 2
    return math.sqrt(s) / H.norm_Ht
