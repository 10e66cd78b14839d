"""Per-leaf-cluster parity for the GPU tests.

A whole-vector relative error dilutes a mistake confined to one leaf cluster
(a wrong cluster offset, a dropped block row) by about the square root of the
number of clusters.  These helpers compare the rows of every nonempty leaf
cluster of the matrix's own cluster tree separately (over all columns), so
that such a mistake meets the full tolerance.  Rows are in the caller's point
order; a leaf cluster's rows are perm[off:off + size] of its tree range.

The scale of cluster I is max(||ref_I||, ||ref|| sqrt(|I| / N)): its own norm,
floored at its share of the whole vector's norm.  The floor matters where the
product cancels: for a smooth kernel and a zero-mean right-hand side, y is a
smooth random field, and a cluster on one of its zero crossings has a small
||y_I|| but the same absolute rounding error (fp32 accumulation is accurate
relative to |A| |x|, not to |A x|) as its neighbours.  A localized mistake
is at least the size of the cluster's own contributions, far above either
scale times the tolerance.

Tolerance per cluster: the fp64 path's 1e-12 as is (its double-float
arithmetic sits near 1e-14); for the fp32-accumulating path twice the
whole-vector 1e-6 (cluster_tol), because the largest of hundreds of cluster
errors exceeds the whole vector's root-mean-square error (measured: 1.002e-6
on one cluster of a 2,048-point H_s matrix with e4m3 blocks whose whole
vector met 1e-6).  A dilution factor sqrt(N / |I|) of 4 to 30 on these
matrices is what the per-cluster check removes.
"""

import numpy as np


def cluster_tol(tol):
    """Per-cluster tolerance for a whole-vector tolerance tol."""
    return tol if tol < 1e-9 else 2.0 * tol


def leaf_rows(O):
    """Caller-order row indices of each nonempty leaf cluster of an oracle
    matrix (built by the oracle or read from a library file)."""
    t = O.tree
    out = []
    for i in range(1 << t.L):
        off, size = t.rng(t.L, i)
        if size > 0:
            out.append(np.asarray(O.perm[off:off + size]))
    return out


def cluster_errors(y, ref, O):
    """||y_I - ref_I|| / max(||ref_I||, ||ref|| sqrt(|I| / N)) for every leaf
    cluster I (Frobenius over the columns); with an all-zero reference the
    product must match exactly (error 0, else inf)."""
    y2 = np.asarray(y).reshape(len(y), -1)
    r2 = np.asarray(ref).reshape(len(ref), -1)
    total, n = float(np.linalg.norm(r2)), r2.shape[0]
    errs = []
    for rows in leaf_rows(O):
        nr = max(float(np.linalg.norm(r2[rows])), total * np.sqrt(len(rows) / n))
        ne = float(np.linalg.norm(y2[rows] - r2[rows]))
        errs.append(ne / nr if nr > 0 else (0.0 if ne == 0 else np.inf))
    return np.array(errs)


def assert_clusters(y, ref, O, tol, extra=None):
    """Every leaf cluster I meets ||y_I - ref_I|| <= cluster_tol(tol) * (its
    scale) (+ ||extra_I|| when an additive allowance of y's shape is given);
    tol is the whole-vector tolerance of the comparison."""
    tol = cluster_tol(tol)
    if extra is None:
        e = cluster_errors(y, ref, O)
        worst = int(np.argmax(e))
        assert e[worst] <= tol, f"leaf cluster {worst}: relative error {e[worst]:.3e} > {tol:.1e}"
        return
    y2 = np.asarray(y).reshape(len(y), -1)
    r2 = np.asarray(ref).reshape(len(ref), -1)
    x2 = np.asarray(extra).reshape(len(extra), -1)
    total, n = float(np.linalg.norm(r2)), r2.shape[0]
    for c, rows in enumerate(leaf_rows(O)):
        err = float(np.linalg.norm(y2[rows] - r2[rows]))
        scale = max(float(np.linalg.norm(r2[rows])), total * np.sqrt(len(rows) / n))
        bound = tol * scale + float(np.linalg.norm(x2[rows]))
        assert err <= bound, f"leaf cluster {c}: error {err:.3e} > bound {bound:.3e}"
