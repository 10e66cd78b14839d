"""GPU parity of the many-right-hand-side path (hh_matvec / hh_matvec_T with
nrhs >= 32) against the oracle, on the stored factors the library's builder
wrote.

The tensor cores take the low-rank blocks stored in fp32, fp16, bf16 and e4m3
whose clusters start at multiples of 16; every other block (fp64, dense, and
unaligned clusters) takes the CUDA cores, which meet 1e-6 relative on their
own.  A tensor-core product carries the slicing of its operands and the
tensor core's truncating fp32 accumulation: fp32 blocks are sliced exactly
(three bf16 slices of factor and input) and their accumulators are drained
into round-to-nearest registers every 16 terms, so their error stays near
fp32's unit roundoff; 16- and 8-bit blocks keep two input slices and one
accumulator per tile (about 2^-17 of their product).  The bound checked is

    ||Y_gpu - Y_oracle||_F <= 1e-6 ||Y_oracle||_F
                              + 2^-20 || sum_{fp32 b} |U_b| (|V_b|^T |X_J|) ||_F
                              + 2^-12 || sum_{16/8-bit b} |U_b| (|V_b|^T |X_J|) ||_F,

sums over the tensor-core blocks: 16 units of fp32 roundoff for fp32 blocks,
half the unit roundoff of fp16 (the most precise 16-bit format) for the
others, i.e. below the rounding error their storage already carries.  On one
case the backward error against the exact kernel matrix is checked against
Theorem 4.4's bound + 1e-6, column by column.
"""
import numpy as np
import pytest

import hh_workloads as W
from rowparity import assert_clusters
from oracle import hhfile
from oracle import matvec as M
from oracle.compress import kernel_entries

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-6


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_09147_gb300 import build as b
    b.build()
    import paper_2604_09147_gb300 as pkg
    return pkg


# (name, n, dim, kernel, kernel_param, leaf, switch level, tol, formats)
CASES = {
    # fp16, bf16 and e4m3 blocks on the tensor cores next to fp32 blocks on the
    # streaming passes
    "gauss_all": (8192, 3, W.GAUSS, 0.05, 64, 4, 1e-5, 31),
    # fp16 and bf16 blocks only
    "invr_16bit": (8192, 3, W.INV_R, 1.0, 64, 3, 1e-3, 31),
    # n = 5184: clusters below level 2 do not start at multiples of 16, so most
    # blocks stay on the streaming passes next to the tensor-core ones
    "invr_mixed": (5184, 3, W.INV_R, 1.0, 64, 3, 1e-3, 31),
    # the multi-RHS workload's kernel and formats at n = 8192
    "gauss_narrow": (8192, 3, W.GAUSS, 0.01, 128, 5, 1e-6, W.F64 | W.F32 | W.BF16 | W.E4M3),
}

_built = {}


def case(P, tmp_path_factory, name):
    if name not in _built:
        n, dim, kern, par, leaf, ell, tol, mask = CASES[name]
        pts = W.points(n, dim, 500 + n)
        H = P.HMatrix.build(pts, kernel=kern, kernel_param=par, leaf_size=leaf, eta=1.0, switch_level=ell,
                            tol=tol, fmt_mask=mask, device=0)
        path = str(tmp_path_factory.mktemp("tc") / f"{name}.hhm")
        H.save(path)
        _built[name] = (H, hhfile.read(path))
    return _built[name]


def tc_blocks(O):
    """The blocks the library's tensor-core path takes (its eligibility rule)."""
    return [b for b in O.lowrank
            if b.k > 0 and b.fmt in (1, 2, 3, 4) and b.row_off % 16 == 0 and b.col_off % 16 == 0]


def abs_product(O, x, transpose):
    """2^-20 sum over the fp32 tensor-core blocks plus 2^-12 sum over the 16/8-bit
    ones of |U_b| (|V_b|^T |x_J|) (or the transpose), user order."""
    xt = np.abs(x[O.perm])
    out = np.zeros_like(xt)
    for b in tc_blocks(O):
        U, V = np.abs(b.Ud()), np.abs(b.Vd())
        w = 2.0 ** -20 if b.fmt == 1 else 2.0 ** -12
        if transpose:
            out[b.col_off:b.col_off + b.n] += w * (V @ (U.T @ xt[b.row_off:b.row_off + b.m]))
        else:
            out[b.row_off:b.row_off + b.m] += w * (U @ (V.T @ xt[b.col_off:b.col_off + b.n]))
    res = np.empty_like(out)
    res[O.perm] = out
    return res


def check(H, O, nrhs, transpose, seed):
    n = H.n
    x = W.rhs(n, nrhs, "normal", seed)
    xg = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()  # column-major (n, nrhs)
    y = H.matvec(xg, transpose=transpose).cpu().numpy()
    H.sync_status()
    ref = M.matvec_T(O, x) if transpose else M.matvec(O, x)
    assert y.shape == ref.shape
    ab = abs_product(O, x, transpose)
    d = y - ref
    assert np.linalg.norm(d) <= TOL * np.linalg.norm(ref) + np.linalg.norm(ab)
    assert_clusters(y, ref, O, TOL, extra=ab)          # the same bound per leaf cluster
    for c in range(nrhs):
        assert np.linalg.norm(d[:, c]) <= TOL * np.linalg.norm(ref[:, c]) + np.linalg.norm(ab[:, c])
    return x, y


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nrhs", [32, 128])
def test_tc_matches_oracle(P, tmp_path_factory, name, nrhs):
    H, O = case(P, tmp_path_factory, name)
    assert H.info()["tc_blocks"] == len(tc_blocks(O)) > 0
    check(H, O, nrhs, False, 7000 + nrhs)
    check(H, O, nrhs, True, 7100 + nrhs)


def test_tc_backward_error_within_theorem_4_4(P, tmp_path_factory):
    """||H x_c - y_c|| / (||H||_F ||x_c||) <= Theorem 4.4's bound + 1e-6 for every
    column, H the exact kernel matrix."""
    H, O = case(P, tmp_path_factory, "gauss_all")
    n, dim, kern, par = CASES["gauss_all"][:4]
    x, y = check(H, O, 32, False, 7600)
    hx = np.zeros_like(x)
    fro2 = 0.0
    for s in range(0, n, 512):
        blk = kernel_entries(kern, par, O.points[s:s + 512], O.points)
        hx[s:s + 512] = blk @ x
        fro2 += float(np.sum(blk * blk))
    be = np.linalg.norm(hx - y, axis=0) / (np.sqrt(fro2) * np.linalg.norm(x, axis=0))
    assert be.max() <= H.info()["bound_thm44"] + 1e-6


@pytest.mark.parametrize("name", ["gauss_all", "gauss_narrow"])
@pytest.mark.parametrize("nrhs", [5, 8, 16, 17])
def test_tc_few_columns(P, tmp_path_factory, name, nrhs):
    """5 to 31 columns take the many-column sequence too (hh_matvec switches
    at 5): fewer right-hand sides than one 16-row MMA block, and 8 columns as
    in the many-right-hand-side workload, against the oracle per column and
    per leaf cluster, forward and transposed."""
    H, O = case(P, tmp_path_factory, name)
    check(H, O, nrhs, False, 7400 + nrhs)
    check(H, O, nrhs, True, 7500 + nrhs)
    assert min(H.info()["tc_panel_bytes"]) > 0            # both directions went through the tensor cores


@pytest.mark.parametrize("nrhs", [33, 47, 200])
def test_tc_ragged_rhs_counts(P, tmp_path_factory, nrhs):
    """nrhs not a multiple of 16 (padded right-hand sides must stay zero) and
    nrhs > 128 (two launch sequences)."""
    H, O = case(P, tmp_path_factory, "gauss_all")
    check(H, O, nrhs, False, 7200 + nrhs)
    check(H, O, nrhs, True, 7300 + nrhs)


def test_tc_split_groups(P, tmp_path_factory, monkeypatch):
    """Phase-1 items of 64 positions: every group of the matrix is split, and
    the CTA that arrives last adds the partial sums."""
    n, dim, kern, par, leaf, ell, tol, mask = CASES["gauss_narrow"]
    monkeypatch.setenv("HH_TC_SPLIT_POSITIONS", "64")
    pts = W.points(n, dim, 500 + n)
    H = P.HMatrix.build(pts, kernel=kern, kernel_param=par, leaf_size=leaf, eta=1.0, switch_level=ell,
                        tol=tol, fmt_mask=mask, device=0)
    path = str(tmp_path_factory.mktemp("tcs") / "split.hhm")
    H.save(path)
    O = hhfile.read(path)
    for nrhs, tr in ((32, False), (128, True), (48, False)):
        check(H, O, nrhs, tr, 7700 + nrhs)
        check(H, O, nrhs, tr, 7800 + nrhs)  # counters were reset by the previous call


def test_tc_panels_packed_per_direction(P, tmp_path_factory):
    """A fresh handle holds no tensor-core panels; the first tensor-core
    product in a direction packs that direction's panels (reported by
    hh_info), and later products reuse them."""
    _, O = case(P, tmp_path_factory, "gauss_narrow")
    path = str(tmp_path_factory.mktemp("panels") / "m.hhm")
    hhfile.write(O, path)
    H = P.HMatrix.load(path, 0)
    assert H.info()["tc_panel_bytes"] == [0, 0]
    check(H, O, 32, False, 7900)
    fwd = H.info()["tc_panel_bytes"]
    assert fwd[0] > 0 and fwd[1] == 0
    check(H, O, 32, True, 7901)
    both = H.info()["tc_panel_bytes"]
    assert both[0] == fwd[0] and both[1] > 0
    check(H, O, 48, False, 7902)
    check(H, O, 48, True, 7903)
    assert H.info()["tc_panel_bytes"] == both


def test_tc_agrees_with_streaming_path(P, tmp_path_factory):
    """The same product through the tensor cores (one call with 32 columns) and
    through the streaming passes (eight calls with 4 columns)."""
    H, O = case(P, tmp_path_factory, "gauss_all")
    x = W.rhs(H.n, 32, "uniform", 7400)
    xg = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()
    y_tc = H.matvec(xg).cpu().numpy()
    y_st = np.concatenate([H.matvec(xg[:, 4 * i:4 * i + 4]).cpu().numpy() for i in range(8)], axis=1)
    H.sync_status()
    ab = abs_product(O, x, False)
    assert np.linalg.norm(y_tc - y_st) <= 2 * TOL * np.linalg.norm(y_st) + np.linalg.norm(ab)


def test_tc_autograd_multi_rhs(P, tmp_path_factory):
    """Forward and backward of the differentiable product with 64 columns."""
    H, O = case(P, tmp_path_factory, "invr_16bit")
    x = W.rhs(H.n, 64, "uniform", 7500)
    ybar = W.rhs(H.n, 64, "normal", 7501)
    xt = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t().requires_grad_(True)
    y = P.hh_apply(H, xt)
    y.backward(torch.from_numpy(np.ascontiguousarray(ybar.T)).cuda().t())
    ref_y, ref_g = M.matvec(O, x), M.matvec_T(O, ybar)
    ab_y, ab_g = abs_product(O, x, False), abs_product(O, ybar, True)
    assert np.linalg.norm(y.detach().cpu().numpy() - ref_y) <= TOL * np.linalg.norm(ref_y) + np.linalg.norm(ab_y)
    assert np.linalg.norm(xt.grad.cpu().numpy() - ref_g) <= TOL * np.linalg.norm(ref_g) + np.linalg.norm(ab_g)


@pytest.mark.parametrize("nrhs", [5, 8, 32, 40, 128])
def test_many_rhs_fp64_matrix(P, tmp_path, nrhs):
    """Uniform fp64 storage with many right-hand sides: the fp64 low-rank blocks
    take the streaming passes in chunks of 4 columns and the dense blocks the
    pair-of-fp32 kernel; the fp64 path's 1e-12 holds for every column."""
    from oracle import build as OB
    c = W.CONFIGS["plain_small"]
    pts = W.config_points("plain_small")
    O = OB.build(pts, c["kernel"], c["kernel_param"], c["leaf"], 1.0, c["ell"], c["tol"], W.F64)
    path = str(tmp_path / "p.hhm")
    hhfile.write(O, path)
    H = P.HMatrix.load(path, 0)
    for tr in (False, True):
        x = W.rhs(len(pts), nrhs, "uniform", 7900 + nrhs + tr)
        xg = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()
        y = H.matvec(xg, transpose=tr).cpu().numpy()
        H.sync_status()
        ref = M.matvec_T(O, x) if tr else M.matvec(O, x)
        cols = np.linalg.norm(y - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert cols.max() <= 1e-12, cols.max()


@pytest.mark.parametrize("n,leaf", [(100, 128), (700, 64), (1, 64)])
def test_many_rhs_tiny_matrices(P, tmp_path, n, leaf):
    """Matrices with no low-rank block (a single dense block, or one point)
    and one that is mostly dense: the many-column sequence with empty
    tensor-core and CUDA-core tables."""
    from oracle import build as OB
    pts = W.points(n, 2, 7700 + n)
    O = OB.build(pts, W.EXP, 1.0, leaf, 1.0, -1, 1e-6, 31)
    path = str(tmp_path / "t.hhm")
    hhfile.write(O, path)
    H = P.HMatrix.load(path, 0)
    x = W.rhs(n, 33, "uniform", 7800 + n)
    xg = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()
    for tr in (False, True):
        y = H.matvec(xg, transpose=tr).cpu().numpy()
        H.sync_status()
        ref = M.matvec_T(O, x) if tr else M.matvec(O, x)
        ab = abs_product(O, x, tr)
        assert np.linalg.norm(y - ref) <= TOL * np.linalg.norm(ref) + np.linalg.norm(ab)


@pytest.mark.parametrize("leaf,ell", [(64, 5), (256, 1)])
def test_many_rhs_dense_entries_fp64(P, tmp_path, leaf, ell):
    """The dense blocks on the tensor cores where several entries meet the same
    output rows: with the switch level at the leaves (2,048 points, leaf 64,
    L = 5) the leaf neighbours stay dense, so a row has several dense blocks;
    with leaf 256 every block is split over two entries of 128 contracted
    positions.  The later entries load and add, the first one stores.  The
    input's magnitude varies by 2^40 over positions and columns, so the
    exponents of the digits (one per row, one per right-hand side and entry)
    are exercised; the fp64 path's 1e-12 holds for every column."""
    from oracle import build as OB
    n = 2048
    pts = W.points(n, 2, 9100 + leaf)
    O = OB.build(pts, W.EXP, 1.0, leaf, 1.0, ell, 1e-10, W.F64)
    assert any(d.row_off != d.col_off for d in O.dense) or max(d.m for d in O.dense) > 128
    path = str(tmp_path / "d.hhm")
    hhfile.write(O, path)
    H = P.HMatrix.load(path, 0)
    # hh_info's count of the tensor-core dense work: per 128-row tile, each
    # dense block meeting it, in entries of at most 128 contracted positions,
    # 128 x 16 operand elements per k-step of 16 positions
    ksteps = 0
    for d in O.dense:
        tiles = range(d.row_off // 128, (d.row_off + d.m - 1) // 128 + 1)
        ksteps += len(tiles) * sum((min(128, d.n - k0) + 15) // 16 for k0 in range(0, d.n, 128))
    assert H.info()["dense_tc_elems"] == ksteps * 128 * 16
    nrhs = 40
    p = np.arange(n)[:, None]
    j = np.arange(nrhs)[None, :]
    x = W.rhs(n, nrhs, "uniform", 9200 + leaf) * 2.0 ** (((p * 37 + j * 11) % 41) - 20)
    xg = torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()
    for tr in (False, True):
        y = H.matvec(xg, transpose=tr).cpu().numpy()
        H.sync_status()
        ref = M.matvec_T(O, x) if tr else M.matvec(O, x)
        cols = np.linalg.norm(y - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert cols.max() <= 1e-12, cols.max()
