"""Seeded synthetic inputs for the H_h matrix-vector product.

This module holds no arithmetic of the method: it only draws point clouds,
right-hand sides and the workload presets (sizes, kernels, tolerances) that
both the CUDA path and the CPU oracle consume.  Points follow the paper's
experimental set-up (Section 5): N particles uniform in a hypercube (the
presets use the unit hypercube [0,1]^d).  Every draw uses numpy's Philox
counter-based generator with an explicit seed.

Kernel ids (the order of the C-ABI enum ``hh_kernel``):
    0  exp(-r/p)            (Matern, p = kernel_param)
    1  1/r,   K(x,x) = 0    (3-D single-layer Laplace)
    2  exp(-r^2/p)          (Gaussian, p = kernel_param)
    3  log r, K(x,x) = 0    (2-D single-layer Laplace)
    4  1/r^2, K(x,x) = 0
Format bits (``hh_fmt_mask``): fp64=1, fp32=2, fp16=4, bf16=8, e4m3=16.
"""
from __future__ import annotations

import math

import numpy as np

EXP, INV_R, GAUSS, LOG, INV_R2 = 0, 1, 2, 3, 4
F64, F32, F16, BF16, E4M3 = 1, 2, 4, 8, 16
RULE_Q43 = 32  # fmt_mask option: the rule uses Table 1's u = 2.5e-1 for the 8-bit format

# Workload presets.  Seeds: points 1234 + id, vectors 42 + id.
CONFIGS = {
    # 2-D exp(-r), N=4,096, leaf 64, eta 1, switch level 3, tol 1e-8, uniform fp64.
    "plain_small": dict(id=1, n=4096, dim=2, kernel=EXP, kernel_param=1.0, leaf=64,
                        eta=1.0, ell=3, tol=1e-8, fmts=F64, rhs="uniform"),
    # 3-D 1/r, N=65,536, leaf 128, eta 1, switch level 4, tol 1e-6, {fp64,fp32,fp16,bf16}.
    "adaptive_65k": dict(id=2, n=65536, dim=3, kernel=INV_R, kernel_param=1.0, leaf=128,
                         eta=1.0, ell=4, tol=1e-6, fmts=F64 | F32 | F16 | BF16, rhs="uniform"),
    # 3-D Gaussian exp(-r^2/0.01), N=262,144, leaf 128, switch level 5, tol 1e-6,
    # {fp64,fp32,bf16,e4m3}; nrhs in {1,8,32,128}, N(0,1) right-hand sides.
    "multirhs_262k": dict(id=3, n=262144, dim=3, kernel=GAUSS, kernel_param=0.01, leaf=128,
                          eta=1.0, ell=5, tol=1e-6, fmts=F64 | F32 | BF16 | E4M3, rhs="normal"),
    # 3-D exp(-r), N=1,048,576, leaf 128, switch level 6, tol 1e-6, {fp64,fp32,bf16}.
    "autograd_1m": dict(id=5, n=1048576, dim=3, kernel=EXP, kernel_param=1.0, leaf=128,
                        eta=1.0, ell=6, tol=1e-6, fmts=F64 | F32 | BF16, rhs="uniform"),
}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def points(n: int, dim: int, seed: int) -> np.ndarray:
    """N points uniform in [0,1]^dim, float64, row-major (n, dim)."""
    return _rng(seed).random((int(n), int(dim)))


def sphere_points(n: int, dim: int, seed: int) -> np.ndarray:
    """N points on the surface of the unit hypersphere in R^dim (the paper's
    second particle set, Section 5), uniform on the surface: normalized
    standard normal vectors.  float64, row-major (n, dim)."""
    g = _rng(seed).standard_normal((int(n), int(dim)))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def rhs(n: int, nrhs: int, dist: str, seed: int) -> np.ndarray:
    """Right-hand sides, float64, column-major (n, nrhs) as a Fortran-ordered array.

    dist: "uniform" -> U(-1,1); "unit" -> U(0,1); "normal" -> N(0,1).
    """
    g = _rng(seed)
    if dist == "uniform":
        x = g.uniform(-1.0, 1.0, size=(nrhs, n))
    elif dist == "unit":
        x = g.random((nrhs, n))
    elif dist == "normal":
        x = g.standard_normal((nrhs, n))
    else:
        raise ValueError(dist)
    return np.asfortranarray(x.T)


def config_points(name: str, n: int | None = None) -> np.ndarray:
    c = CONFIGS[name]
    return points(c["n"] if n is None else n, c["dim"], 1234 + c["id"])


def config_rhs(name: str, nrhs: int = 1, n: int | None = None) -> np.ndarray:
    c = CONFIGS[name]
    return rhs(c["n"] if n is None else n, nrhs, c["rhs"], 42 + c["id"])


def uneven_batch(count: int = 64, seed: int = 1238, nmin: int = 2048, nmax: int = 131072):
    """The uneven batch of independent matrices: N log-uniform in [nmin, nmax]
    (the preset: [2,048, 131,072]).

    Even index: 2-D exp(-r), leaf 64.  Odd index: 3-D 1/r, leaf 128.  eta 1,
    tol 1e-6, adaptive {fp64, fp32, fp16, bf16}, switch level -1 (floor(L/2)).
    Returns a list of dicts with the build parameters and the points.
    """
    g = _rng(seed)
    ns = np.exp(g.uniform(math.log(nmin), math.log(nmax), size=count)).astype(np.int64)
    out = []
    for i, n in enumerate(ns):
        if i % 2 == 0:
            p = dict(dim=2, kernel=EXP, kernel_param=1.0, leaf=64)
        else:
            p = dict(dim=3, kernel=INV_R, kernel_param=1.0, leaf=128)
        p.update(n=int(n), eta=1.0, ell=-1, tol=1e-6, fmts=F64 | F32 | F16 | BF16)
        p["points"] = points(int(n), p["dim"], seed * 1000 + i)
        p["x"] = rhs(int(n), 1, "uniform", seed * 1000 + 500 + i)
        out.append(p)
    return out
