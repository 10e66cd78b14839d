"""GPU parity of the row-sharded product's shards (hh_shard) on one GPU.

The shards of 2 and 3 ranks run one after another on cuda:0 (no collective,
no kernel waits on another); their products are assembled the way
paper_2604_09147_gb300.dist assembles them (each shard's own rows of y; the
sum of the transposed parts) and compared with the oracle's product of the
whole matrix, in tree order, whole vector and per leaf cluster: 1, 4 and 32
columns (the 32-column product takes the tensor-core and CUDA-core kernels on
blocks cut at range boundaries), and a uniform-fp64 matrix at 1e-12.
"""
import numpy as np
import pytest

import hh_workloads as W
from oracle import hhfile
from oracle import matvec as M
from rowparity import assert_clusters
from test_gpu_tc import abs_product

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ALL = W.F64 | W.F32 | W.F16 | W.BF16 | W.E4M3


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_09147_gb300 import build as b
    b.build()
    import paper_2604_09147_gb300 as pkg
    return pkg


def _tree(O):
    """An oracle matrix's copy whose point order is the tree order (to apply
    the per-cluster check to tree-order vectors)."""
    import copy
    T = copy.copy(O)
    T.tree = copy.copy(O.tree)
    T.tree.perm = np.arange(O.n)
    return T


@pytest.mark.parametrize("mask,tol", [(ALL, 1e-6), (W.F64, 1e-12)])
def test_shards_assemble_the_product(P, tmp_path, mask, tol):
    n = 20000
    H = P.HMatrix.build(W.points(n, 3, 805), W.INV_R, 1.0, 64, 1.0, -1, 1e-5, mask, device=0)
    path = str(tmp_path / "h.hhm")
    H.save(path)
    G = hhfile.read(path)
    T = _tree(G)
    perm = G.perm
    for nr in (1, 4, 32):
        X = W.rhs(n, nr, "normal", 806 + nr)
        ref = M.matvec(G, X)[perm]
        ref_t = M.matvec_T(G, X)[perm]
        Xt = torch.from_numpy(np.ascontiguousarray(X[perm].T)).cuda().t()
        for world in (2, 3):
            b = H.shard_plan(world)
            y = np.zeros_like(ref)
            xb = np.zeros_like(ref_t)
            for r in range(world):
                S = H.shard(b[r], b[r + 1], 0)
                yr = S.matvec(Xt).cpu().numpy()
                assert not np.any(yr[:b[r]]) and not np.any(yr[b[r + 1]:])   # rows outside stay zero
                y[b[r]:b[r + 1]] = yr[b[r]:b[r + 1]]
                yb = torch.zeros_like(Xt)
                yb[b[r]:b[r + 1]] = Xt[b[r]:b[r + 1]]
                xb += S.matvec(yb, transpose=True).cpu().numpy()
                S.sync_status()
            # 32 columns: the tensor-core allowance of tests/test_gpu_tc.py over
            # the whole matrix's eligible blocks (cut blocks take the CUDA cores)
            tc = nr >= 32 and mask != W.F64
            ea = abs_product(G, X, False)[perm] if tc else np.zeros_like(ref)
            et = abs_product(G, X, True)[perm] if tc else np.zeros_like(ref_t)
            assert np.linalg.norm(y - ref) <= tol * np.linalg.norm(ref) + np.linalg.norm(ea)
            assert np.linalg.norm(xb - ref_t) <= tol * np.linalg.norm(ref_t) + np.linalg.norm(et)
            assert_clusters(y, ref, T, tol, extra=ea if tc else None)
            assert_clusters(xb, ref_t, T, tol, extra=et if tc else None)
