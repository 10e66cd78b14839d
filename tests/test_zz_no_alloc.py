"""GPU test of hh_matvec_noalloc, the product that allocates nothing.

Callers that cannot allocate device memory at call time (a framework that
owns all device memory, a loop that must not pay cudaMalloc's implicit
synchronisation) use this entry point; its scratch is a fixed array inside
the library.  The test calls it through the C-ABI twice in a row, forward and
transposed, and compares with hh_matvec on the same matrix; checks that the
device's free memory is the same before and after the calls; and checks that
a matrix too large for the fixed array is rejected with HH_EINVAL.  It builds
its own matrices, so it passes alone in a fresh process as well as after
other tests.
"""
import ctypes

import numpy as np
import pytest

import hh_workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-6          # the adaptive-path tolerance of the other GPU tests


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_09147_gb300 import build as b
    b.build()
    import paper_2604_09147_gb300 as pkg
    return pkg


def _entry(P):
    lib = ctypes.CDLL(P.LIB_PATH)
    f = lib.hh_matvec_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.hh_last_error.restype = ctypes.c_char_p
    lib.hh_last_error.argtypes = []
    return lib, f


def test_noalloc_matches_matvec_twice(P):
    lib, f = _entry(P)
    pts = W.points(12000, 3, 31)
    H = P.HMatrix.build(pts, W.GAUSS, 0.02, 64, 1.0, 4, 1e-4, W.F64 | W.F32 | W.F16 | W.BF16 | W.E4M3,
                        device=0)
    n = H.n
    st = torch.cuda.current_stream().cuda_stream
    xs = [[torch.from_numpy(W.rhs(n, 1, "uniform", 40 + 2 * trial + tr)[:, 0].copy()).cuda() for trial in range(2)]
          for tr in (0, 1)]
    refs = [[H.matvec(xs[tr][t], transpose=bool(tr)) for t in range(2)] for tr in (0, 1)]
    ys = [[torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)] for _ in (0, 1)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for tr in (0, 1):
        for t in range(2):
            rc = f(H._h, tr, xs[tr][t].data_ptr(), ys[tr][t].data_ptr(), st)
            assert rc == 0, lib.hh_last_error().decode()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0          # nothing was allocated
    for tr in (0, 1):
        for t in range(2):
            a, b = ys[tr][t].cpu().numpy(), refs[tr][t].cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL
    H.sync_status()


def test_noalloc_rejects_matrix_beyond_its_scratch(P, tmp_path):
    """A 1,048,576-point matrix needs about 40 MB of scratch, more than the
    32 MiB array: the call fails with HH_EINVAL and says so.  The matrix is
    one cluster with no blocks (its product is zero), written with the
    oracle's file writer, so that nothing large has to be built."""
    from oracle import hhfile
    from oracle.build import HMatrix as OM
    from oracle.tree import Tree
    lib, f = _entry(P)
    n = 1 << 20
    pts = W.points(n, 3, 32)
    tree = Tree(L=0, perm=np.arange(n, dtype=np.int64), off=np.zeros(1, np.int64),
                size=np.array([n], np.int64), lo=pts.min(axis=0)[None, :], hi=pts.max(axis=0)[None, :])
    O = OM(n=n, dim=3, kernel=W.EXP, kernel_param=1.0, leaf_size=n, eta=1.0, ell=0, tol=1e-6,
           fmt_mask=W.F64, points=pts, tree=tree, norm_Ht=1.0)
    path = str(tmp_path / "empty.hhm")
    hhfile.write(O, path)
    H = P.HMatrix.load(path, 0)
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    rc = f(H._h, 0, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == P.HH_EINVAL
    assert b"bytes of scratch" in lib.hh_last_error()
    assert torch.count_nonzero(H.matvec(x)).item() == 0     # the ordinary product still runs
