"""The differentiation workload's matrix family at the largest size whose host
construction fits a routine GPU test run (about a minute and a half on 8-16
host cores): N = 131,072 points U[0,1]^3, exp(-r), leaf 128, eta 1, switch
level floor(L/2) (the rule the 1,048,576-point workload's level 6 follows:
L = 10 gives 5), tol 1e-6, adaptive {fp64, fp32, bf16} re-encoded from the
uniform-fp64 build of the same compression.

Checked through torch.autograd (forward y = A_h x, hand-written backward
x_bar = A_h^T y_bar, x ~ U(-1,1), y_bar ~ N(0,1)):
  * y and x_bar against the oracle's Algorithm 4 and its transpose over the
    same stored factors, whole vector and every leaf cluster, 1e-6 relative;
  * the adjoint identity <y_bar, A_h d> = <A_h^T y_bar, d> on 16 seeded
    directions, 1e-6 relative;
  * central differences with step 1e-6 of L(x) = <y_bar, A x> on the
    uniform-fp64 matrix (fp64-class arithmetic: the products' rounding, about
    1e-14 ||y_bar|| ||y|| with random signs, divided by the 2e-6 of the
    difference) against the backward, 16 directions, within
    1e-6 ||y_bar|| ||y||.
The 1,048,576-point size itself runs in tests/test_gpu_scale.py (opt-in).
"""
import os

import numpy as np
import pytest

import hh_workloads as W
from oracle import hhfile
from oracle import matvec as M
from rowparity import assert_clusters

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
CACHE = os.environ.get("HH_CACHE_DIR", "/tmp/hh_cache")
N = 131072
TOL = 1e-6


@pytest.fixture(scope="module")
def mats(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_09147_gb300 import build as b
    b.build()
    import paper_2604_09147_gb300 as P
    c = W.CONFIGS["autograd_1m"]
    pts = W.points(N, 3, 1234 + c["id"])
    H64 = P.HMatrix.build_cached(pts, CACHE, c["kernel"], c["kernel_param"], c["leaf"], c["eta"], -1, c["tol"],
                                 W.F64, device=0)
    Ham = H64.reencode(c["fmts"], 0)
    path = str(tmp_path_factory.mktemp("exp") / "amp.hhm")
    Ham.save(path)
    return P, H64, Ham, hhfile.read(path)


def test_exp_131k_autograd_against_oracle_rows(mats):
    P, H64, Ham, G = mats
    assert Ham.info()["ell"] == Ham.info()["L"] // 2
    x = torch.from_numpy(W.rhs(N, 1, "uniform", 5201)[:, 0].copy()).cuda().requires_grad_(True)
    ybar = W.rhs(N, 1, "normal", 5202)[:, 0]
    y = P.hh_apply(Ham, x)
    y.backward(torch.from_numpy(ybar.copy()).cuda())
    Ham.sync_status()
    xs = x.detach().cpu().numpy()
    yo, xo = M.matvec(G, xs), M.matvec_T(G, ybar)
    yg, xg = y.detach().cpu().numpy(), x.grad.cpu().numpy()
    assert np.linalg.norm(yg - yo) <= TOL * np.linalg.norm(yo)
    assert np.linalg.norm(xg - xo) <= TOL * np.linalg.norm(xo)
    assert_clusters(yg, yo, G, TOL)
    assert_clusters(xg, xo, G, TOL)


def test_exp_131k_adjoint_16_directions(mats):
    P, H64, Ham, G = mats
    ybar = torch.from_numpy(W.rhs(N, 1, "normal", 5203)[:, 0].copy()).cuda()
    xbar = Ham.matvec(ybar, transpose=True)
    D = torch.from_numpy(np.ascontiguousarray(W.rhs(N, 16, "uniform", 5204).T)).cuda().t()
    AD = Ham.matvec(D)
    Ham.sync_status()
    lhs = (ybar[:, None] * AD).sum(0).cpu().numpy()
    rhs = (xbar[:, None] * D).sum(0).cpu().numpy()
    scale = ybar.norm().item() * AD.norm(dim=0).cpu().numpy()
    assert np.max(np.abs(lhs - rhs) / scale) <= TOL


def test_exp_131k_central_differences_fp64(mats):
    P, H64, Ham, G = mats
    x = torch.from_numpy(W.rhs(N, 1, "uniform", 5205)[:, 0].copy()).cuda().requires_grad_(True)
    ybar = torch.from_numpy(W.rhs(N, 1, "normal", 5206)[:, 0].copy()).cuda()
    torch.dot(ybar, P.hh_apply(H64, x)).backward()
    g = x.grad.detach()
    x0 = x.detach()
    scale = float(ybar.norm()) * float(H64.matvec(x0).norm())
    h = 1e-6
    for k in range(16):
        d = torch.from_numpy(W.rhs(N, 1, "uniform", 5300 + k)[:, 0].copy()).cuda()
        lp = float(torch.dot(ybar, H64.matvec(x0 + h * d)))
        lm = float(torch.dot(ybar, H64.matvec(x0 - h * d)))
        assert abs((lp - lm) / (2 * h) - float(torch.dot(g, d))) <= 1e-6 * scale
    H64.sync_status()
