"""GPU parity: the CUDA path through the C-ABI against the oracle.

Tolerances:
  * fp64-stored factors and dense blocks are computed in fp64 on the GPU:
    ||y_gpu - y_oracle|| / ||y_oracle|| <= 1e-12 over the same stored factors.
  * 32/16/8-bit factors are computed with fp32 accumulation (input rounded to
    fp32, products and sums in fp32, fp64 scatter):
    ||y_gpu - y_oracle|| / ||y_oracle|| <= 1e-6 over the same stored factors,
    and against the exact kernel matrix the backward error
    ||H x - y|| / (||H|| ||x||) stays within Theorem 4.4's bound + 1e-6.
The oracle either builds the matrix itself and writes the file the library
loads (hh_load), or reads the file the library's host builder wrote.
"""
import os

import numpy as np
import pytest

import hh_workloads as W
from rowparity import assert_clusters
from oracle import build as OB
from oracle.compress import kernel_entries
from oracle import hhfile
from oracle import matvec as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ALL = W.F64 | W.F32 | W.F16 | W.BF16 | W.E4M3
CACHE = os.environ.get("HH_CACHE_DIR", "/tmp/hh_cache")
TOL64, TOL32 = 1e-12, 1e-6


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_09147_gb300 import build as b
    b.build()
    import paper_2604_09147_gb300 as pkg
    return pkg


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def oracle_pair(P, tmp_path, pts, kernel, param, leaf, ell, tol, mask):
    O = OB.build(pts, kernel, param, leaf, 1.0, ell, tol, mask)
    path = str(tmp_path / "o.hhm")
    hhfile.write(O, path)
    return O, P.HMatrix.load(path, 0)


def check_against(P, H, O, x, tol):
    """Forward and transposed product against the oracle: the whole vector
    and every leaf cluster's rows at the same relative tolerance."""
    y = H.matvec(gpu(x)).cpu().numpy()
    ref = M.matvec(O, x)
    assert rel(y, ref) <= tol
    assert_clusters(y, ref, O, tol)
    z = H.matvec(gpu(x), transpose=True).cpu().numpy()
    ref = M.matvec_T(O, x)
    assert rel(z, ref) <= tol
    assert_clusters(z, ref, O, tol)
    H.sync_status()


def test_fp64_path_matches_oracle_file(P, tmp_path):
    c = W.CONFIGS["plain_small"]
    pts = W.config_points("plain_small")
    O, H = oracle_pair(P, tmp_path, pts, c["kernel"], c["kernel_param"], c["leaf"], c["ell"], c["tol"], W.F64)
    x = W.config_rhs("plain_small")
    check_against(P, H, O, x[:, 0], TOL64)
    # several right-hand sides with a leading dimension larger than n
    for nrhs in (2, 3, 4, 5, 8):
        xs = W.rhs(len(pts), nrhs, "uniform", 100 + nrhs)
        buf = torch.zeros((nrhs, len(pts) + 7), dtype=torch.float64, device="cuda")
        buf[:, :len(pts)] = gpu(xs.T)
        xv = buf.t()[:len(pts)]
        assert xv.stride(1) == len(pts) + 7
        y = H.matvec(xv).cpu().numpy()
        assert rel(y, M.matvec(O, xs)) <= TOL64
        assert_clusters(y, M.matvec(O, xs), O, TOL64)


@pytest.mark.parametrize("n,dim,kernel,param,ell,tol,nfmt", [(8192, 3, W.GAUSS, 0.01, 4, 1e-3, 3),
                                                             (6000, 3, W.INV_R, 1.0, 3, 1e-2, 1),
                                                             (5000, 2, W.LOG, 1.0, 3, 1e-4, 2)])
def test_adaptive_formats_match_oracle_file(P, tmp_path, n, dim, kernel, param, ell, tol, nfmt):
    pts = W.points(n, dim, 5)
    O, H = oracle_pair(P, tmp_path, pts, kernel, param, 64, ell, tol, ALL)
    used = {b.fmt for b in O.lowrank}
    assert len(used) >= nfmt
    x = W.rhs(n, 1, "uniform", 6)[:, 0]
    check_against(P, H, O, x, TOL32)
    xs = W.rhs(n, 4, "normal", 7)
    y4 = H.matvec(gpu(xs)).cpu().numpy()
    assert rel(y4, M.matvec(O, xs)) <= TOL32
    assert_clusters(y4, M.matvec(O, xs), O, TOL32)


@pytest.mark.parametrize("dim,kernel", [(3, W.INV_R), (2, W.LOG)])
def test_sphere_surface_points(P, tmp_path, dim, kernel):
    """The paper's second particle set (points on the unit sphere / circle):
    single, several and 32 columns (the tensor-core path), forward and
    transposed, against the oracle over the same stored factors."""
    n = 6144
    pts = W.sphere_points(n, dim, 15)
    O, H = oracle_pair(P, tmp_path, pts, kernel, 1.0, 64, 4, 1e-5, ALL)
    x = W.rhs(n, 1, "uniform", 16)[:, 0]
    check_against(P, H, O, x, TOL32)
    xs = W.rhs(n, 4, "normal", 17)
    assert rel(H.matvec(gpu(xs)).cpu().numpy(), M.matvec(O, xs)) <= TOL32
    # 32 columns: tensor-core blocks bounded as in tests/test_gpu_tc.py
    X = W.rhs(n, 32, "normal", 18)
    Y = H.matvec(torch.from_numpy(np.ascontiguousarray(X.T)).cuda().t()).cpu().numpy()
    H.sync_status()
    ref = M.matvec(O, X)
    xt = np.abs(X[O.perm])
    ab = np.zeros_like(xt)
    for b in O.lowrank:
        if b.k > 0 and b.fmt in (1, 2, 3, 4) and b.row_off % 16 == 0 and b.col_off % 16 == 0:
            w = 2.0 ** -20 if b.fmt == 1 else 2.0 ** -12
            ab[b.row_off:b.row_off + b.m] += w * (np.abs(b.Ud()) @ (np.abs(b.Vd()).T @ xt[b.col_off:b.col_off + b.n]))
    abu = np.empty_like(ab)
    abu[O.perm] = ab
    assert np.linalg.norm(Y - ref) <= TOL32 * np.linalg.norm(ref) + np.linalg.norm(abu)


@pytest.mark.parametrize("dim,kernel", [(2, W.LOG), (3, W.INV_R)])
def test_2d_tree_matrices(P, tmp_path, dim, kernel):
    """Matrices on the balanced 2^d-tree (cells of any size, some empty)
    through the same kernels: 1, 4 and 32 columns, forward and transposed."""
    import math
    n = 5000
    pts = W.points(n, dim, 19) * 2 - 1
    O = OB.build(pts, kernel, 1.0, 32, math.sqrt(dim), 1, 1e-5, ALL, tree_kind="2d")
    path = str(tmp_path / "t2d.hhm")
    hhfile.write(O, path)
    H = P.HMatrix.load(path, 0)
    assert H.info()["tree_step"] == dim
    check_against(P, H, O, W.rhs(n, 1, "uniform", 20)[:, 0], TOL32)
    xs = W.rhs(n, 4, "normal", 21)
    assert rel(H.matvec(gpu(xs)).cpu().numpy(), M.matvec(O, xs)) <= TOL32
    X = W.rhs(n, 32, "normal", 22)
    for tr in (False, True):
        Y = H.matvec(torch.from_numpy(np.ascontiguousarray(X.T)).cuda().t(), transpose=tr).cpu().numpy()
        H.sync_status()
        ref = M.matvec_T(O, X) if tr else M.matvec(O, X)
        assert rel(Y, ref) <= 1e-5


@pytest.mark.parametrize("n,dim,leaf,ell,mask", [
    (50, 2, 64, -1, W.F64),            # one dense block (L = 0)
    (5000, 3, 128, 3, ALL),            # ragged cluster sizes
    (3001, 2, 64, 0, W.F64 | W.F32),   # HODLR (ell = 0), odd n
    (2048, 2, 64, 5, ALL),             # H_s (ell = L) with neighbour blocks
    (129, 3, 128, 1, W.F64),           # two leaves of 64 / 65 points
])
def test_edge_cases(P, tmp_path, n, dim, leaf, ell, mask):
    pts = W.points(n, dim, 8)
    kernel = W.EXP if dim == 2 else W.INV_R
    O, H = oracle_pair(P, tmp_path, pts, kernel, 1.0, leaf, ell, 1e-4, mask)
    x = W.rhs(n, 1, "uniform", 9)[:, 0]
    tol = TOL64 if mask == W.F64 else TOL32
    check_against(P, H, O, x, tol)
    assert np.all(H.matvec(torch.zeros(n, dtype=torch.float64, device="cuda")).cpu().numpy() == 0)


def test_library_builder_plain_small(P, tmp_path):
    """hh_build on the plain small workload; oracle reads the saved factors."""
    c = W.CONFIGS["plain_small"]
    pts = W.config_points("plain_small")
    H = P.HMatrix.build(pts, c["kernel"], c["kernel_param"], c["leaf"], c["eta"], c["ell"], c["tol"], c["fmts"], device=0)
    path = str(tmp_path / "b.hhm")
    H.save(path)
    G = hhfile.read(path)
    x = W.config_rhs("plain_small")[:, 0]
    y = H.matvec(gpu(x)).cpu().numpy()
    assert rel(y, M.matvec(G, x)) <= TOL64
    Hd = M.dense_h(pts, c["kernel"], c["kernel_param"])
    bx = Hd @ x
    inf = H.info()
    assert np.linalg.norm(bx - y) / (np.linalg.norm(Hd) * np.linalg.norm(x)) <= inf["bound_thm44"]
    assert rel(y, bx) <= 50 * c["tol"]


@pytest.fixture(scope="module")
def adaptive_65k(P):
    c = W.CONFIGS["adaptive_65k"]
    pts = W.config_points("adaptive_65k")
    H64 = P.HMatrix.build_cached(pts, CACHE, c["kernel"], c["kernel_param"], c["leaf"], c["eta"], c["ell"],
                                 c["tol"], W.F64, device=0)
    Ham = H64.reencode(c["fmts"], 0)
    return c, pts, H64, Ham


def test_full_size_adaptive_65k(P, adaptive_65k, tmp_path):
    """Full size, bench launch configuration: both layouts against the oracle
    over the same stored factors, and the backward error on sampled rows."""
    c, pts, H64, Ham = adaptive_65k
    x = W.config_rhs("adaptive_65k")[:, 0]
    for H, tol in ((H64, TOL64), (Ham, TOL32)):
        path = str(tmp_path / "f.hhm")
        H.save(path)
        G = hhfile.read(path)
        y = H.matvec(gpu(x)).cpu().numpy()
        yo = M.matvec(G, x)
        assert rel(y, yo) <= tol
        assert_clusters(y, yo, G, tol)
        z = H.matvec(gpu(x), transpose=True).cpu().numpy()
        zo = M.matvec_T(G, x)
        assert rel(z, zo) <= tol
        assert_clusters(z, zo, G, tol)
        del G
    # backward error against the exact kernel on 1024 sampled rows
    rows = np.random.default_rng(0).choice(len(pts), 1024, replace=False)
    y = Ham.matvec(gpu(x)).cpu().numpy()
    bx = M.h_rows_times(pts, c["kernel"], c["kernel_param"], rows, x)
    # ||H||_F estimated from the same rows (unbiased for uniform sampling)
    hn = 0.0
    for s in range(0, len(rows), 128):
        blk = kernel_entries(c["kernel"], c["kernel_param"], pts[rows[s:s + 128]], pts)
        hn += float(np.sum(blk * blk))
    hn = np.sqrt(hn * len(pts) / len(rows))
    be = np.linalg.norm(bx - y[rows]) * np.sqrt(len(pts) / len(rows)) / (hn * np.linalg.norm(x))
    assert be <= Ham.info()["bound_thm44"] + 1e-6


def test_autograd_backward_is_transpose(P, tmp_path):
    pts = W.points(4000, 3, 12)
    O, H = oracle_pair(P, tmp_path, pts, W.EXP, 1.0, 64, 3, 1e-5, W.F64 | W.F32 | W.BF16)
    x = gpu(W.rhs(4000, 1, "uniform", 1)[:, 0]).requires_grad_(True)
    ybar = W.rhs(4000, 1, "normal", 2)[:, 0]
    y = P.hh_apply(H, x)
    y.backward(gpu(ybar))
    assert rel(x.grad.cpu().numpy(), M.matvec_T(O, ybar)) <= TOL32
    # adjoint identity on 16 random directions
    for k in range(16):
        d = W.rhs(4000, 1, "uniform", 50 + k)[:, 0]
        lhs = float(np.dot(ybar, H.matvec(gpu(d)).cpu().numpy()))
        rhs = float(np.dot(H.matvec(gpu(ybar), transpose=True).cpu().numpy(), d))
        assert abs(lhs - rhs) <= 1e-6 * abs(lhs) + 1e-12


def test_autograd_matches_central_differences(P, tmp_path):
    """The product is linear, so a central difference of L(x) = <ybar, A_h x>
    with any step is <ybar, A_h d> up to rounding.  On a uniform-fp64 matrix
    (fp64-class arithmetic, within 1e-12 of the oracle) with h = 1e-3 the
    rounding is about 1e-12 ||ybar|| ||y|| / h; the hand-written backward
    <A_h^T ybar, d> must agree to 1e-7 ||ybar|| ||y|| on 8 directions (about
    6e-6 of the derivative itself for these random vectors)."""
    pts = W.points(4000, 3, 13)
    _, H = oracle_pair(P, tmp_path, pts, W.EXP, 1.0, 64, 3, 1e-8, W.F64)
    x = gpu(W.rhs(4000, 1, "uniform", 3)[:, 0]).requires_grad_(True)
    ybar = gpu(W.rhs(4000, 1, "normal", 4)[:, 0])
    torch.dot(ybar, P.hh_apply(H, x)).backward()
    g = x.grad.detach()
    x0 = x.detach()
    scale = float(ybar.norm()) * float(H.matvec(x0).norm())
    h = 1e-3
    for k in range(8):
        d = gpu(W.rhs(4000, 1, "uniform", 60 + k)[:, 0])
        lp = float(torch.dot(ybar, H.matvec(x0 + h * d)))
        lm = float(torch.dot(ybar, H.matvec(x0 - h * d)))
        assert abs((lp - lm) / (2 * h) - float(torch.dot(g, d))) <= 1e-7 * scale


def test_host_api_and_batched(P, tmp_path):
    mats, xs, oracles = [], [], []
    for i, n in enumerate((2100, 3333, 1500)):
        pts = W.points(n, 2 + i % 2, 20 + i)
        O, H = oracle_pair(P, tmp_path, pts, W.EXP if i % 2 == 0 else W.INV_R, 1.0, 64, -1, 1e-6,
                           W.F64 | W.F32 | W.F16 | W.BF16)
        mats.append(H)
        oracles.append(O)
        xs.append(W.rhs(n, 1, "uniform", 30 + i)[:, 0])
    ys = P.matvec_batched(mats, [gpu(x) for x in xs])
    for H, O, x, y in zip(mats, oracles, xs, ys):
        assert rel(y.cpu().numpy(), M.matvec(O, x)) <= TOL32
        assert rel(H.matvec_host(x), M.matvec(O, x)) <= TOL32
        out = torch.empty(len(x), dtype=torch.float64, pin_memory=True).numpy()
        assert H.matvec_host(x, out=out) is out and rel(out, M.matvec(O, x)) <= TOL32
        assert rel(H.matvec_ws(gpu(x)).cpu().numpy(), M.matvec(O, x)) <= TOL32
        H.sync_status()
    with pytest.raises(ValueError):
        mats[0].matvec_host(xs[0], out=np.empty(len(xs[0]) + 1))


def test_batch_one_launch_sequence_and_graph(P, tmp_path):
    """Uneven batch (2-D exp and 3-D 1/r, sizes that are not multiples of the
    leaf size) through one persistent kernel and through a captured CUDA
    graph, forward and transposed, against the oracle per matrix; and the
    same batch through the four-launch sequence (HH_BATCH_LAUNCHES=4)."""
    specs = [(3000, 2, W.EXP, 64), (5184, 3, W.INV_R, 128), (2100, 2, W.EXP, 64), (7777, 3, W.INV_R, 128),
             (4096, 2, W.EXP, 64), (2500, 3, W.INV_R, 64)]
    mats, oracles, xs = [], [], []
    for i, (n, dim, kern, leaf) in enumerate(specs):
        H = P.HMatrix.build(W.points(n, dim, 9100 + i), kernel=kern, kernel_param=1.0, leaf_size=leaf, eta=1.0,
                            switch_level=-1, tol=1e-6, fmt_mask=W.F64 | W.F32 | W.F16 | W.BF16, device=0)
        path = str(tmp_path / f"b{i}.hhm")
        H.save(path)
        mats.append(H)
        oracles.append(hhfile.read(path))
        xs.append(W.rhs(n, 1, "uniform", 9200 + i)[:, 0])
    B = P.HBatch(mats)
    assert B.offsets == list(np.cumsum([0] + [s[0] for s in specs]))
    x = gpu(np.concatenate(xs))
    for tr in (False, True):
        y1 = B.matvec(x, transpose=tr).cpu().numpy()
        y2 = B.matvec(x, transpose=tr, graph=True).cpu().numpy()
        y3 = B.matvec(x, transpose=tr, graph=True).cpu().numpy()  # replay
        mats[0].sync_status()
        for i, O in enumerate(oracles):
            a, b = B.offsets[i], B.offsets[i + 1]
            ref = M.matvec_T(O, xs[i]) if tr else M.matvec(O, xs[i])
            assert rel(y1[a:b], ref) <= TOL32
            assert_clusters(y1[a:b], ref, O, TOL32)
        # replays agree up to the order of the fp64 atomic additions
        assert rel(y3, y2) <= 1e-12
        assert rel(y2, y1) <= 1e-12
    # the persistent cooperative kernel (default) against the four-launch sequence
    os.environ["HH_BATCH_LAUNCHES"] = "4"
    try:
        B4 = P.HBatch(mats)
    finally:
        del os.environ["HH_BATCH_LAUNCHES"]
    for tr in (False, True):
        yp = B.matvec(x, transpose=tr, graph=True).cpu().numpy()
        y4 = B4.matvec(x, transpose=tr, graph=True).cpu().numpy()
        assert rel(y4, yp) <= 1e-12
        assert rel(B4.matvec(x, transpose=tr).cpu().numpy(), yp) <= 1e-12
    B4.close()
    B.close()


def test_batch_fp64_matrices_match_at_1e12(P, tmp_path):
    """A batch of uniform-fp64 matrices keeps the fp64 path's 1e-12."""
    mats, oracles, xs = [], [], []
    for i, n in enumerate((1500, 3333, 2048)):
        O = OB.build(W.points(n, 2, 9300 + i), W.EXP, 1.0, 64, 1.0, -1, 1e-8, W.F64)
        path = str(tmp_path / f"f{i}.hhm")
        hhfile.write(O, path)
        mats.append(P.HMatrix.load(path, 0))
        oracles.append(O)
        xs.append(W.rhs(n, 1, "uniform", 9400 + i)[:, 0])
    B = P.HBatch(mats)
    y = B.matvec(gpu(np.concatenate(xs)), graph=True).cpu().numpy()
    for i, O in enumerate(oracles):
        a, b = B.offsets[i], B.offsets[i + 1]
        assert rel(y[a:b], M.matvec(O, xs[i])) <= TOL64
        assert_clusters(y[a:b], M.matvec(O, xs[i]), O, TOL64)
    B.close()


def test_autotune_keeps_results(P):
    """hh_autotune changes launch parameters only: the products before and
    after agree up to rounding, and the choices are reported."""
    H = P.HMatrix.build(W.points(6000, 3, 9500), kernel=W.GAUSS, kernel_param=0.05, leaf_size=64, eta=1.0,
                        switch_level=-1, tol=1e-5, fmt_mask=ALL, device=0)
    x1 = gpu(W.rhs(6000, 1, "uniform", 9501)[:, 0])
    xm = gpu(np.ascontiguousarray(W.rhs(6000, 40, "normal", 9502).T)).t()
    before = [H.matvec(x1).cpu().numpy(), H.matvec(x1, transpose=True).cpu().numpy(), H.matvec(xm).cpu().numpy()]
    info0 = H.info()
    assert info0["tuned"] == 0 and info0["split_positions"] == 8192
    choice = H.autotune(40)
    info = H.info()
    assert info["tuned"] == 1 and choice["split_positions"] in (1024, 2048, 4096, 8192, 16384, 32768, 65536)
    assert all(1 <= c <= 16 for c in choice["blocks_per_sm"])
    after = [H.matvec(x1).cpu().numpy(), H.matvec(x1, transpose=True).cpu().numpy(), H.matvec(xm).cpu().numpy()]
    H.sync_status()
    for a, b in zip(before, after):
        assert rel(b, a) <= 1e-6
