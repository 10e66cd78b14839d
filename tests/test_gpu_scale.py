"""Full-size checks that need minutes of host construction: opt in with
HH_SCALE_TESTS=1.

The differentiation workload at scale: N = 1,048,576 points U[0,1]^3,
exp(-r), leaf 128, eta 1, switch level 6, tol 1e-6, adaptive {fp64, fp32,
bf16}; forward y = A_h x for x ~ U(-1,1) and the hand-written backward
x_bar = A_h^T y_bar for y_bar ~ N(0,1) through torch.autograd.  Checked:
  * the adjoint identity <y_bar, A_h d> = <A_h^T y_bar, d> for 16 seeded
    directions d (the operator is linear, so this is the exact form of a
    finite-difference test), within 1e-6 relative;
  * 256 sampled entries of y and of x_bar against the exact kernel matrix
    (kernel symmetric, so row i of H is column i), their error relative to
    ||H~||_F (Algorithm 5) times the vector norm, scaled to the full length,
    within Theorem 4.4's bound + 1e-6.
"""
import os

import numpy as np
import pytest

import hh_workloads as W
from oracle.compress import kernel_entries

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")
CACHE = os.environ.get("HH_CACHE_DIR", "/tmp/hh_cache")


@pytest.fixture(scope="module")
def P():
    if os.environ.get("HH_SCALE_TESTS") != "1":
        pytest.skip("full-size checks: set HH_SCALE_TESTS=1")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_09147_gb300 import build as b
    b.build()
    import paper_2604_09147_gb300 as pkg
    return pkg


def test_autograd_1m_adjoint_and_sampled_rows(P):
    c = W.CONFIGS["autograd_1m"]
    pts = W.config_points("autograd_1m")
    H = P.HMatrix.build_cached(pts, CACHE, c["kernel"], c["kernel_param"], c["leaf"], c["eta"], c["ell"], c["tol"],
                               c["fmts"], device=0)
    n = len(pts)
    info = H.info()
    x = torch.from_numpy(W.config_rhs("autograd_1m")[:, 0].copy()).cuda().requires_grad_(True)
    ybar = torch.from_numpy(W.rhs(n, 1, "normal", 4205)[:, 0].copy()).cuda()
    y = P.hh_apply(H, x)
    y.backward(ybar)
    xbar = x.grad.detach()
    H.sync_status()
    # adjoint identity on 16 directions
    D = torch.from_numpy(np.ascontiguousarray(W.rhs(n, 16, "normal", 4206).T)).cuda().t()
    AD = H.matvec(D)
    lhs = (ybar[:, None] * AD).sum(0).cpu().numpy()
    rhs = (xbar[:, None] * D).sum(0).cpu().numpy()
    scale = ybar.norm().item() * AD.norm(dim=0).cpu().numpy()
    assert np.max(np.abs(lhs - rhs) / scale) <= 1e-6
    # sampled rows of the exact kernel matrix
    rng = np.random.default_rng(4207)
    S = rng.choice(n, 256, replace=False)
    xs, ys, yg, xg = x.detach().cpu().numpy(), ybar.cpu().numpy(), y.detach().cpu().numpy(), xbar.cpu().numpy()
    hx, hty = np.zeros(len(S)), np.zeros(len(S))
    for k in range(0, len(S), 32):
        blk = kernel_entries(c["kernel"], c["kernel_param"], pts[S[k:k + 32]], pts)
        hx[k:k + 32] = blk @ xs
        hty[k:k + 32] = blk @ ys
    frac = np.sqrt(n / len(S))
    be_y = frac * np.linalg.norm(hx - yg[S]) / (info["norm_ht"] * np.linalg.norm(xs))
    be_x = frac * np.linalg.norm(hty - xg[S]) / (info["norm_ht"] * np.linalg.norm(ys))
    bound = info["bound_thm44"] + 1e-6
    assert be_y <= bound and be_x <= bound, (be_y, be_x, bound)
