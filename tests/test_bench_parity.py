"""bench.py's parity field: the product against the oracle's Algorithm 4 on
the rows of sampled leaf clusters (blocks restricted to those rows), checked
on CPU against the oracle's own full product."""
import numpy as np

import bench
import hh_workloads as W
from oracle import build as OB
from oracle import hhfile
from oracle import matvec as M


def test_rows_check_against_full_product(tmp_path):
    O = OB.build(W.points(3000, 3, 5), W.INV_R, 1.0, 64, 1.0, 2, 1e-6, W.F64 | W.F32 | W.F16 | W.BF16)
    path = str(tmp_path / "p.hhm")
    hhfile.write(O, path)
    G = hhfile.read(path)
    x = W.rhs(3000, 1, "uniform", 6)[:, 0]
    y = M.matvec(G, x)
    r = bench.oracle_rows_check(G, x, y)
    assert r["rel_err"] <= 1e-15 and r["leaf_clusters"] == 8 and r["rows"] > 0
    # every leaf: the sampled rows cover the product
    r = bench.oracle_rows_check(G, x, y * (1 + 1e-7), leaves=1 << G.tree.L)
    assert r["rows"] == 3000 and abs(r["rel_err"] - 1e-7) <= 1e-12
    # an error in one leaf cluster's rows is seen when that leaf is sampled
    leaf = (1 << G.tree.L) - 1 + 3
    yp = y.copy()
    yp[G.perm[int(G.tree.off[leaf]):int(G.tree.off[leaf] + G.tree.size[leaf])]] += 1.0
    assert bench.oracle_rows_check(G, x, yp, leaves=1 << G.tree.L)["rel_err"] > 1e-4


def test_rows_check_many_columns(tmp_path):
    O = OB.build(W.points(2000, 3, 7), W.GAUSS, 0.05, 64, 1.0, 2, 1e-6, W.F64 | W.F32 | W.BF16 | W.E4M3)
    path = str(tmp_path / "m.hhm")
    hhfile.write(O, path)
    G = hhfile.read(path)
    X = W.rhs(2000, 5, "normal", 8)
    Y = M.matvec(G, X)
    assert bench.oracle_rows_check(G, X, Y)["rel_err"] <= 1e-15
    Yp = Y.copy()
    Yp[:, 3] *= 1 + 1e-6
    r = bench.oracle_rows_check(G, X, Yp, leaves=1 << G.tree.L)
    assert r["rows"] == 2000 and 0 < r["rel_err"] < 1e-6

