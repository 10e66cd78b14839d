"""H_h construction (Algorithm 1), Frobenius norms (Algorithm 5) and the
adaptive mixed precision representation (Algorithm 3).

Steps, in the paper's order:
 1. cluster tree and the hybrid partition (Algorithm 1's three loops and the
    dense leaf diagonal), see tree.py / partition.py;
 2. LRcompression of every admissible block to eps (Algorithm 1);
 3. ||H~_IJ||^2 = trace(Sigma^2) of each compressed block and
    ||H~||^2 = sum of those plus the squared norms of the dense blocks
    (Algorithm 5; with ell == L the leaf neighbours are added densely);
 4. xi = ||H~_IJ|| / ||H~|| and u_IJ = max{u_bar in {u} U U_set :
    u_bar <= eps / (2^{dl/2} xi)} (Eq. 4.6 / Algorithm 3), where the factor
    2^{dl/2} is the square root of the number of clusters at level l, i.e.
    2^{l/2} for the binary tree (reading R2);
 5. with ell == L, a leaf neighbour block is kept low rank only when that
    pays off in its assigned format, p (m + n) b / 64 < m n (Section 4.3,
    special case of Algorithm 3); otherwise it stays dense in fp64;
 6. U and V stored in the assigned format with power-of-two block scales
    (formats.py); dense diagonal blocks stay in fp64 (working precision).

Storage (Eqs. 2.6, 3.3-3.6, Section 5.2 bit count): a low-rank block costs
p (m + n) b / 64 words of fp64, a dense block m n.

Parity: pinned by tests (Lemma 3.1 on dense N, Algorithm 5 identity, the
worked example of Section 4.3, monotonicity of the rule, eps <= 1e-10 gives
only fp64, storage criterion S_s - S_h = S_1 - S_2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import formats as F
from .compress import kernel_entries, lr_compress
from .partition import KIND_NBR, Partition, measured_csp, partition
from .tree import Tree, build_tree, build_tree_2d


@dataclass
class LRBlock:
    level: int
    kind: int
    i: int
    j: int
    row_off: int
    m: int
    col_off: int
    n: int
    U: np.ndarray            # H~ factor, float64 (|I| x p), orthonormal columns
    V: np.ndarray            # H~ factor, float64 (|J| x p), carries Sigma
    sv: np.ndarray           # kept singular values
    norm: float              # ||H~_IJ||_F = sqrt(trace(Sigma^2))
    fmt: int = F.FP64
    exp_u: int = 0
    exp_v: int = 0
    Us: np.ndarray = None    # stored values (exactly representable in fmt)
    Vs: np.ndarray = None

    @property
    def k(self) -> int:
        return int((self.U if self.U is not None else self.Us).shape[1])

    def Ud(self) -> np.ndarray:
        """decoded U = stored * 2^exp_u"""
        return np.ldexp(self.Us, self.exp_u)

    def Vd(self) -> np.ndarray:
        return np.ldexp(self.Vs, self.exp_v)


@dataclass
class DenseBlock:
    level: int
    i: int
    j: int
    row_off: int
    m: int
    col_off: int
    n: int
    D: np.ndarray            # float64 (m x n)


@dataclass
class HMatrix:
    n: int
    dim: int
    kernel: int
    kernel_param: float
    leaf_size: int
    eta: float
    ell: int
    tol: float
    fmt_mask: int
    points: np.ndarray
    tree: Tree
    lowrank: list = field(default_factory=list)
    dense: list = field(default_factory=list)
    norm_Ht: float = 0.0

    @property
    def L(self) -> int:
        return self.tree.L

    @property
    def perm(self) -> np.ndarray:
        return self.tree.perm

    def csp(self) -> list[int]:
        return measured_csp([(b.level, b.i) for b in self.lowrank], self.L)

    def storage(self, uniform_fp64: bool = False) -> float:
        """Storage in fp64 words: sum p(m+n) b/64 + sum m n."""
        s = 0.0
        for b in self.lowrank:
            bits = 64 if uniform_fp64 else F.BITS[b.fmt]
            s += b.k * (b.m + b.n) * bits / 64.0
        for d in self.dense:
            s += d.m * d.n
        return s

    def count_by_format(self) -> dict:
        out = {f: 0 for f in F.NAMES}
        for b in self.lowrank:
            out[b.fmt] += 1
        return out


# fmt_mask bit 5: the rule takes Table 1's printed u = 2.5e-1 for the 8-bit
# format (formats.choose_format's q43_rule); bits 0-4 select the formats
RULE_Q43 = 1 << 5


def allowed_formats(fmt_mask: int) -> list[int]:
    return [f for f in (F.FP32, F.FP16, F.BF16, F.E4M3) if fmt_mask & (1 << f)]


def level_factor(level: int) -> float:
    """sqrt of the number of clusters at level l of the binary tree: 2^{l/2}."""
    return math.sqrt(math.ldexp(1.0, level))


def lowrank_pays_off(p: int, m: int, n: int, bits: int) -> bool:
    """Section 4.3: a neighbour block is stored low rank when p (m + n) b / 64 < m n."""
    return p * (m + n) * bits / 64.0 < m * n


def block_tau(tol: float, level: int, norm_b: float, norm_all: float) -> float:
    """eps / (2^{l/2} xi) with xi = ||H~_IJ|| / ||H~|| (Eq. 4.6)."""
    xi = norm_b / norm_all
    if xi == 0.0:
        return math.inf
    return tol / (level_factor(level) * xi)


def build(points: np.ndarray, kernel: int, kernel_param: float, leaf_size: int,
          eta: float, ell: int, tol: float, fmt_mask: int, tree_kind: str = "kd") -> HMatrix:
    """tree_kind "kd": binary KD bisection; "2d": the balanced 2^d-tree, with
    ell given in its tree levels (-1: floor(L/2)) and stored as the binary
    level d ell, like every block level (so 2^{l/2} of the rule is the
    paper's 2^{d l'/2} at tree level l')."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n, dim = pts.shape
    if tree_kind == "2d":
        tree = build_tree_2d(pts, leaf_size)
    elif tree_kind == "kd":
        tree = build_tree(pts, leaf_size)
    else:
        raise ValueError("tree_kind must be 'kd' or '2d'")
    L = tree.L
    if ell < 0:
        ell = (L // tree.step) // 2
    ell *= tree.step
    part: Partition = partition(tree, eta, ell)
    tp = pts[tree.perm]                              # points in tree order
    H = HMatrix(n=n, dim=dim, kernel=kernel, kernel_param=kernel_param, leaf_size=leaf_size,
                eta=eta, ell=ell, tol=tol, fmt_mask=fmt_mask, points=pts, tree=tree)

    # Algorithm 1: compress every admissible block; dense blocks at the leaves
    for (l, i, j, kind) in part.lowrank:
        ro, m = tree.rng(l, i)
        co, nn = tree.rng(l, j)
        U, V, s = lr_compress(kernel, kernel_param, tp[ro:ro + m], tp[co:co + nn], tol)
        H.lowrank.append(LRBlock(l, kind, i, j, ro, m, co, nn, U, V, s,
                                 float(np.sqrt(np.sum(s * s)))))
    nbr_candidates = []  # indices into H.dense
    for (l, i, j, kind) in part.dense:
        ro, m = tree.rng(l, i)
        co, nn = tree.rng(l, j)
        D = kernel_entries(kernel, kernel_param, tp[ro:ro + m], tp[co:co + nn])
        H.dense.append(DenseBlock(l, i, j, ro, m, co, nn, D))
        if kind == KIND_NBR:
            nbr_candidates.append(len(H.dense) - 1)

    # Algorithm 5: ||H~||^2 from the singular values and the dense blocks
    norm2 = sum(b.norm ** 2 for b in H.lowrank) + sum(float(np.sum(d.D * d.D)) for d in H.dense)
    H.norm_Ht = math.sqrt(norm2)

    # Algorithm 3: precision of every admissible block
    allowed = allowed_formats(fmt_mask)
    q43 = bool(fmt_mask & RULE_Q43)
    for b in H.lowrank:
        b.fmt = F.choose_format(block_tau(tol, b.level, b.norm, H.norm_Ht), allowed, q43)

    # Section 4.3 special case (ell == L): compress a leaf neighbour when it pays off
    if ell == L and nbr_candidates:
        nbr_set = set(nbr_candidates)
        keep = []
        for idx, d in enumerate(H.dense):
            if idx not in nbr_set:
                keep.append(d)
                continue
            U, V, s = lr_compress(kernel, kernel_param, tp[d.row_off:d.row_off + d.m],
                                  tp[d.col_off:d.col_off + d.n], tol)
            nb = float(np.sqrt(np.sum(s * s)))
            f = F.choose_format(block_tau(tol, d.level, nb, H.norm_Ht), allowed, q43)
            if lowrank_pays_off(U.shape[1], d.m, d.n, F.BITS[f]):
                H.lowrank.append(LRBlock(d.level, KIND_NBR, d.i, d.j, d.row_off, d.m,
                                         d.col_off, d.n, U, V, s, nb, fmt=f))
            else:
                keep.append(d)
        H.dense = keep

    # store the factors in their formats
    for b in H.lowrank:
        b.Us, b.exp_u = F.quantize_factor(b.U, b.fmt)
        b.Vs, b.exp_v = F.quantize_factor(b.V, b.fmt)
    return H
