"""GPU test of hh_matvec_noalloc, the product that allocates nothing.

Callers that cannot allocate device memory at call time (a framework that
owns all device memory, a loop that must not pay cudaMalloc's implicit
synchronisation) use this entry point; its scratch is a fixed array inside
the library.  The test calls it through the C-ABI twice in a row, forward and
transposed, and compares with hh_matvec on the same matrix.  It builds its own
matrix, so it passes alone in a fresh process as well as after other tests.
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


def test_noalloc_matches_matvec_twice(P):
    lib = ctypes.CDLL(P.LIB_PATH)
    f = lib.hh_matvec_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    pts = W.points(12000, 3, 31)
    H = P.HMatrix.build(pts, W.GAUSS, 0.02, 64, 1.0, 4, 1e-4, W.F64 | W.F32 | W.F16 | W.BF16 | W.E4M3,
                        device=0)
    n = H.n
    st = torch.cuda.current_stream().cuda_stream
    for transpose in (0, 1):
        for trial in range(2):
            x = torch.from_numpy(W.rhs(n, 1, "uniform", 40 + 2 * trial + transpose)[:, 0].copy()).cuda()
            ref = H.matvec(x, transpose=bool(transpose))
            y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            rc = f(H._h, transpose, x.data_ptr(), y.data_ptr(), st)
            assert rc == 0, lib.hh_last_error
            torch.cuda.synchronize()
            a, b = y.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL
    H.sync_status()
