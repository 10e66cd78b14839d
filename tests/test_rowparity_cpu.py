"""The per-leaf-cluster comparison of the GPU tests (tests/rowparity.py) on
the CPU: a mistake planted in the oracle (one low-rank block dropped) shows
up in the cluster errors undiluted, while the whole-vector error shrinks by
about the square root of the number of clusters; rounding-level differences
pass at their own scale."""
import copy

import numpy as np

import hh_workloads as W
from oracle import build as OB
from oracle import matvec as M
from rowparity import cluster_errors


def test_cluster_errors_see_a_dropped_block_undiluted():
    pts = W.points(4096, 3, 71)
    O = OB.build(pts, W.INV_R, 1.0, 32, 1.0, 3, 1e-6, W.F64)
    x = W.rhs(4096, 1, "uniform", 72)[:, 0]
    ref = M.matvec(O, x)
    # the smallest block of the finest weak level: one leaf-pair block
    b = min((b for b in O.lowrank if b.level == O.L), key=lambda b: b.m * b.n)
    bad = copy.copy(O)
    bad.lowrank = [c for c in O.lowrank if c is not b]
    y = M.matvec(bad, x)
    whole = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    per = cluster_errors(y, ref, O)
    assert per.max() >= 5 * whole               # about sqrt(128 clusters) / sqrt(clusters hit)
    assert np.count_nonzero(per > 0) == 1       # only the block's row cluster moved
    tiny = ref * (1 + 1e-13)
    assert cluster_errors(tiny, ref, O).max() <= 2e-13
