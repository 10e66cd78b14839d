"""GB300 H_h-matrix library: Python binding of the C-ABI in include/hh.h.

Argument marshalling only: every step of the product runs in libhh.so's
sm_103a kernels; PyTorch supplies device memory and the current CUDA stream.
The library must have been built (``python -m paper_2604_09147_gb300.build``);
the first call into it raises ImportError when libhh.so is missing.

    H = HMatrix.build(points, kernel=INV_R, leaf_size=128, eta=1.0,
                      switch_level=4, tol=1e-6, fmt_mask=F64 | F32 | F16 | BF16)
    y = H @ x                     # x: float64 CUDA tensor (n,) or (n, nrhs)
    y = hh_apply(H, x)            # differentiable: backward is A_h^T ybar
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhh.so")

EXP, INV_R, GAUSS, LOG, INV_R2 = 0, 1, 2, 3, 4
F64, F32, F16, BF16, E4M3 = 1, 2, 4, 8, 16
RULE_Q43 = 32  # fmt_mask option: the rule uses Table 1's u = 2.5e-1 for the 8-bit format
FMT_NAMES = ("fp64", "fp32", "fp16", "bf16", "e4m3")
HH_OK, HH_EINVAL, HH_ENOMEM, HH_ECUDA, HH_ETIMEOUT, HH_ENOTSUP, HH_EIO, HH_EDEVICE = 0, -1, -2, -3, -4, -5, -6, -7
MAX_LEVELS = 48


class HHError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hh error {code}: {msg}")
        self.code = code


class _Info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("dim", ctypes.c_int32), ("L", ctypes.c_int32), ("ell", ctypes.c_int32),
        ("leaf_size", ctypes.c_int32), ("kernel", ctypes.c_int32), ("device", ctypes.c_int32),
        ("eta", ctypes.c_double), ("tol", ctypes.c_double), ("kernel_param", ctypes.c_double),
        ("n_lowrank", ctypes.c_int64), ("n_dense", ctypes.c_int64),
        ("blocks_per_fmt", ctypes.c_int64 * 5), ("factor_bytes_per_fmt", ctypes.c_int64 * 5),
        ("dense_bytes", ctypes.c_int64), ("u_bytes", ctypes.c_int64), ("v_bytes", ctypes.c_int64),
        ("max_rank", ctypes.c_int64),
        ("storage_amp", ctypes.c_double), ("storage_fp64", ctypes.c_double),
        ("bytes_per_matvec", ctypes.c_double), ("flops_per_matvec", ctypes.c_double),
        ("norm_ht", ctypes.c_double), ("csp", ctypes.c_int32 * MAX_LEVELS),
        ("bound_thm42", ctypes.c_double), ("bound_thm44", ctypes.c_double),
        ("bound_rounding", ctypes.c_double), ("build_seconds", ctypes.c_double),
        ("tc_blocks", ctypes.c_int64), ("tc_factor_bytes", ctypes.c_int64),
        ("tc_u_elems", ctypes.c_int64), ("tc_v_elems", ctypes.c_int64),
        ("mr_u_elems", ctypes.c_int64), ("mr_v_elems", ctypes.c_int64), ("dense_elems", ctypes.c_int64),
        ("tuned", ctypes.c_int32), ("split_positions", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32 * 4),
        ("tc_panel_bytes", ctypes.c_int64 * 2), ("tree_step", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("build_device", ctypes.c_int32), ("pad2_", ctypes.c_int32), ("build_fallback", ctypes.c_int64),
        ("build_device_seconds", ctypes.c_double), ("stream_depth", ctypes.c_int32 * 4),
        ("item_bytes", ctypes.c_int64), ("dense_tc_elems", ctypes.c_int64),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2604_09147_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    c = ctypes
    P, I64, I32, U32, U64, D = c.c_void_p, c.c_int64, c.c_int, c.c_uint32, c.c_uint64, c.c_double
    sig = {
        "hh_build": (I32, [P, I64, I32, I32, D, I32, D, I32, D, U32, U64, I32, c.POINTER(P)]),
        "hh_build_ex": (I32, [P, I64, I32, I32, D, I32, D, I32, D, U32, U64, I32, I32, c.POINTER(P)]),
        "hh_build_dev": (I32, [P, I64, I32, I32, D, I32, D, I32, D, U32, U64, I32, I32, c.POINTER(P)]),
        "hh_optimal_switch_level_dev": (I32, [P, I64, I32, I32, D, I32, D, D, U32, U64, I32, I32, c.POINTER(I32),
                                              c.POINTER(I32), c.POINTER(D)]),
        "hh_load": (I32, [c.c_char_p, I32, c.POINTER(P)]),
        "hh_reencode": (I32, [P, U32, I32, c.POINTER(P)]),
        "hh_optimal_switch_level": (I32, [P, I64, I32, I32, D, I32, D, D, U32, U64, I32, c.POINTER(I32),
                                          c.POINTER(I32), c.POINTER(D)]),
        "hh_save": (I32, [P, c.c_char_p]),
        "hh_shard_plan": (I32, [P, I32, c.POINTER(I64)]),
        "hh_shard": (I32, [P, I64, I64, I32, c.POINTER(P)]),
        "hh_info": (I32, [P, c.POINTER(_Info)]),
        "hh_perm": (I32, [P, P]),
        "hh_matvec": (I32, [P, P, P, I32, I64, I64, P]),
        "hh_matvec_T": (I32, [P, P, P, I32, I64, I64, P]),
        "hh_workspace_bytes": (I32, [P, c.POINTER(c.c_size_t)]),
        "hh_solve_cg": (I32, [P, P, P, D, D, I32, c.POINTER(I32), c.POINTER(D), P]),
        "hh_matvec_ws": (I32, [P, I32, P, P, I32, I64, I64, P, c.c_size_t, P]),
        "hh_matvec_host": (I32, [P, I32, P, P, I32, P]),
        "hh_matvec_timed": (I32, [P, I32, P, P, I32, I64, I64, P, c.POINTER(c.c_float)]),
        "hh_matvec_stages": (I32, [P, I32, P, P, I32, I64, I64, P, c.POINTER(c.c_float)]),
        "hh_autotune": (I32, [P, I32]),
        "hh_matvec_batched": (I32, [c.POINTER(P), I32, c.POINTER(P), c.POINTER(P), P]),
        "hh_batch_create": (I32, [c.POINTER(P), I32, c.POINTER(P)]),
        "hh_batch_offsets": (I32, [P, c.POINTER(I64)]),
        "hh_batch_matvec": (I32, [P, I32, P, P, P]),
        "hh_batch_matvec_graph": (I32, [P, I32, P, P, P]),
        "hh_batch_free": (None, [P]),
        "hh_sync_status": (I32, [P, P]),
        "hh_free": (None, [P]),
        "hh_last_error": (c.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_LIB = None


def _L():
    """The loaded library (loaded on first use; raises if it was not built)."""
    global _LIB
    if _LIB is None:
        _LIB = _load()
    return _LIB


def _check(rc: int):
    if rc != HH_OK:
        raise HHError(rc, _L().hh_last_error().decode(errors="replace"))


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _as_colmajor(x: torch.Tensor, n: int):
    """(view, nrhs, ld, was_vector) of x as a column-major float64 matrix."""
    if x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError("x must be a float64 CUDA tensor")
    if x.dim() == 1:
        if x.shape[0] != n:
            raise ValueError(f"x has {x.shape[0]} rows, expected {n}")
        return x.contiguous(), 1, n, True
    if x.dim() != 2 or x.shape[0] != n:
        raise ValueError(f"x must have shape ({n},) or ({n}, nrhs)")
    if x.stride(0) == 1 and x.stride(1) >= n:
        return x, x.shape[1], x.stride(1), False
    xc = x.t().contiguous().t()
    return xc, x.shape[1], n, False


class HMatrix:
    """A built H_h matrix on one GPU (or host only with device=-1)."""

    def __init__(self, handle: int, device: int):
        self._h = ctypes.c_void_p(handle)
        self.device = device
        inf = self.info()
        self.n = inf["n"]
        self._ws = None

    # -- construction -------------------------------------------------------
    @classmethod
    def build(cls, points, kernel: int = INV_R, kernel_param: float = 1.0, leaf_size: int = 128,
              eta: float = 1.0, switch_level: int = -1, tol: float = 1e-6, fmt_mask: int = F64 | F32 | F16 | BF16,
              seed: int = 0, device: int | None = None, tree: str = "kd",
              construct_on_device: bool = False) -> "HMatrix":
        """hh_build_ex; tree "kd" (binary KD bisection) or "2d" (the balanced
        2^d-tree, switch_level in its levels).  construct_on_device: the
        blocks' compression runs on `device` (hh_build_dev)."""
        pts = np.ascontiguousarray(points.cpu().numpy() if isinstance(points, torch.Tensor) else points,
                                   dtype=np.float64)
        if pts.ndim != 2:
            raise ValueError("points must be (n, dim)")
        if tree not in ("kd", "2d"):
            raise ValueError("tree must be 'kd' or '2d'")
        if device is None:
            device = torch.cuda.current_device() if torch.cuda.is_available() else -1
        out = ctypes.c_void_p()
        fn = _L().hh_build_dev if construct_on_device else _L().hh_build_ex
        _check(fn(pts.ctypes.data, pts.shape[0], pts.shape[1], kernel, kernel_param, leaf_size,
                  eta, switch_level, tol, fmt_mask, seed, 1 if tree == "2d" else 0, device, ctypes.byref(out)))
        return cls(out.value, device)

    @classmethod
    def build_cached(cls, points, cache_dir: str, kernel: int = INV_R, kernel_param: float = 1.0,
                     leaf_size: int = 128, eta: float = 1.0, switch_level: int = -1, tol: float = 1e-6,
                     fmt_mask: int = F64 | F32 | F16 | BF16, seed: int = 0,
                     device: int | None = None) -> "HMatrix":
        """hh_build, checkpointed: the matrix is saved under cache_dir keyed by
        a hash of the points and parameters and loaded from there next time."""
        import hashlib
        pts = np.ascontiguousarray(points.cpu().numpy() if isinstance(points, torch.Tensor) else points,
                                   dtype=np.float64)
        key = hashlib.sha256(pts.tobytes() + repr((kernel, kernel_param, leaf_size, eta, switch_level, tol,
                                                   fmt_mask, seed, 1)).encode()).hexdigest()[:24]
        path = os.path.join(cache_dir, f"hh_{key}.hhm")
        if os.path.exists(path):
            return cls.load(path, device)
        H = cls.build(pts, kernel, kernel_param, leaf_size, eta, switch_level, tol, fmt_mask, seed, device)
        os.makedirs(cache_dir, exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        H.save(tmp)
        os.replace(tmp, path)
        return H

    @classmethod
    def load(cls, path: str, device: int | None = None) -> "HMatrix":
        if device is None:
            device = torch.cuda.current_device() if torch.cuda.is_available() else -1
        out = ctypes.c_void_p()
        _check(_L().hh_load(os.fsencode(path), device, ctypes.byref(out)))
        return cls(out.value, device)

    def reencode(self, fmt_mask: int, device: int | None = None) -> "HMatrix":
        """Algorithm 3 again with another format set (source must be uniform fp64)."""
        if device is None:
            device = self.device
        out = ctypes.c_void_p()
        _check(_L().hh_reencode(self._h, fmt_mask, device, ctypes.byref(out)))
        return HMatrix(out.value, device)

    def save(self, path: str) -> None:
        _check(_L().hh_save(self._h, os.fsencode(path)))

    # -- several GPUs ------------------------------------------------------
    def shard_plan(self, nranks: int) -> list[int]:
        """hh_shard_plan: tree-position bounds of the block rows of nranks ranks."""
        b = (ctypes.c_int64 * (nranks + 1))()
        _check(_L().hh_shard_plan(self._h, int(nranks), b))
        return [int(v) for v in b]

    def shard(self, p0: int, p1: int, device: int | None = None) -> "HMatrix":
        """hh_shard: the block rows [p0, p1) as a matrix whose vectors are in
        tree order (see paper_2604_09147_gb300.dist for the collectives)."""
        if device is None:
            device = self.device
        out = ctypes.c_void_p()
        _check(_L().hh_shard(self._h, int(p0), int(p1), device, ctypes.byref(out)))
        return HMatrix(out.value, device)

    def close(self) -> None:
        if self._h is not None and self._h.value:
            _L().hh_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- queries -----------------------------------------------------------
    def info(self) -> dict:
        s = _Info()
        _check(_L().hh_info(self._h, ctypes.byref(s)))
        d = {name: getattr(s, name) for name, _ in _Info._fields_}
        d["blocks_per_fmt"] = {FMT_NAMES[i]: int(s.blocks_per_fmt[i]) for i in range(5)}
        d["factor_bytes_per_fmt"] = {FMT_NAMES[i]: int(s.factor_bytes_per_fmt[i]) for i in range(5)}
        d["csp"] = [int(s.csp[i]) for i in range(s.L + 1)]
        d["blocks_per_sm"] = [int(v) for v in s.blocks_per_sm]
        d["tc_panel_bytes"] = [int(v) for v in s.tc_panel_bytes]
        d["stream_depth"] = [int(v) for v in s.stream_depth]
        return d

    def autotune(self, nrhs_many: int = 0) -> dict:
        """Time candidate launch parameters on the device and keep the fastest
        (streaming CTAs per SM; with nrhs_many > 0 the many-column item split)."""
        _check(_L().hh_autotune(self._h, int(nrhs_many)))
        i = self.info()
        return {"blocks_per_sm": i["blocks_per_sm"], "stream_depth": i["stream_depth"],
                "item_bytes": i["item_bytes"], "split_positions": i["split_positions"]}

    def perm(self) -> np.ndarray:
        p = np.empty(self.n, dtype=np.int32)
        _check(_L().hh_perm(self._h, p.ctypes.data))
        return p

    def workspace_bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(_L().hh_workspace_bytes(self._h, ctypes.byref(b)))
        return int(b.value)

    # -- products ----------------------------------------------------------
    def matvec(self, x: torch.Tensor, transpose: bool = False, out: torch.Tensor | None = None) -> torch.Tensor:
        """y = A_h x (or A_h^T x) on the current CUDA stream."""
        xv, nrhs, ldx, vec = _as_colmajor(x, self.n)
        if out is None:
            out = torch.empty((self.n,) if vec else (nrhs, self.n), dtype=torch.float64, device=x.device)
            yv = out if vec else out.t()
        else:
            yv = out
        ldy = self.n if vec else yv.stride(1)
        if not vec and yv.stride(0) != 1:
            raise ValueError("out must be column-major (stride(0) == 1)")
        f = _L().hh_matvec_T if transpose else _L().hh_matvec
        _check(f(self._h, xv.data_ptr(), yv.data_ptr(), nrhs, ldx, ldy, _stream_ptr(x.device)))
        return yv

    def __matmul__(self, x: torch.Tensor) -> torch.Tensor:
        return self.matvec(x)

    def matvec_ws(self, x: torch.Tensor, transpose: bool = False) -> torch.Tensor:
        """Product with a workspace from torch's allocator (safe on any stream)."""
        xv, nrhs, ldx, vec = _as_colmajor(x, self.n)
        nb = self.workspace_bytes()
        ws = torch.empty(nb + 256, dtype=torch.uint8, device=x.device)
        base = (ws.data_ptr() + 255) // 256 * 256
        out = torch.empty((nrhs, self.n), dtype=torch.float64, device=x.device).t()
        _check(_L().hh_matvec_ws(self._h, 1 if transpose else 0, xv.data_ptr(), out.data_ptr(), nrhs, ldx,
                                 self.n, base, nb, _stream_ptr(x.device)))
        return out[:, 0] if vec else out

    def matvec_host(self, x: np.ndarray, transpose: bool = False, out: np.ndarray | None = None) -> np.ndarray:
        """End-to-end product from host memory (copies inside the call).  out:
        an optional column-major float64 array of x's shape to write into
        (page-locked memory, e.g. a pinned torch tensor's numpy view, lets the
        device-to-host copy run at full speed)."""
        xa = np.asfortranarray(x, dtype=np.float64)
        nrhs = 1 if xa.ndim == 1 else xa.shape[1]
        if out is None:
            y = np.empty_like(xa, order="F")
        else:
            if out.shape != xa.shape or out.dtype != np.float64 or not out.flags.f_contiguous:
                raise ValueError("out must be a column-major float64 array of x's shape")
            y = out
        st = _stream_ptr(self.device) if self.device >= 0 else 0
        _check(_L().hh_matvec_host(self._h, 1 if transpose else 0, xa.ctypes.data, y.ctypes.data, nrhs, st))
        return y

    def matvec_timed(self, x: torch.Tensor, y: torch.Tensor, transpose: bool = False) -> list:
        """One product with per-launch CUDA-event times in ms (synchronises):
        [prep, phase 1, phase 2, finish]."""
        xv, nrhs, ldx, vec = _as_colmajor(x, self.n)
        ms = (ctypes.c_float * 4)()
        ldy = self.n if y.dim() == 1 else y.stride(1)
        _check(_L().hh_matvec_timed(self._h, 1 if transpose else 0, xv.data_ptr(), y.data_ptr(), nrhs, ldx, ldy,
                                    _stream_ptr(x.device), ms))
        return [float(v) for v in ms]

    def matvec_stages(self, x: torch.Tensor, y: torch.Tensor, transpose: bool = False) -> list:
        """One product of up to 128 columns through the many-right-hand-side
        sequence with per-launch CUDA-event times in ms (synchronises):
        [input images, dense blocks, fp64 streaming passes, CUDA-core phase 1,
        tensor-core phase 1, CUDA-core phase 2, tensor-core phase 2, finish]."""
        xv, nrhs, ldx, vec = _as_colmajor(x, self.n)
        ms = (ctypes.c_float * 8)()
        ldy = self.n if y.dim() == 1 else y.stride(1)
        _check(_L().hh_matvec_stages(self._h, 1 if transpose else 0, xv.data_ptr(), y.data_ptr(), nrhs, ldx, ldy,
                                     _stream_ptr(x.device), ms))
        return [float(v) for v in ms]

    def solve_cg(self, b: torch.Tensor, shift: float = 0.0, rtol: float = 1e-8, max_iter: int = 1000,
                 x0: torch.Tensor | None = None) -> tuple:
        """hh_solve_cg: conjugate gradients for (A_h + shift I) x = b on the
        device; returns (x, iterations, final relative residual)."""
        if b.dim() != 1 or b.shape[0] != self.n or b.dtype != torch.float64 or not b.is_cuda:
            raise ValueError("b must be a cuda float64 vector of length n")
        b = b.contiguous()
        x = torch.zeros_like(b) if x0 is None else x0.detach().clone().contiguous()
        it, res = ctypes.c_int(), ctypes.c_double()
        _check(_L().hh_solve_cg(self._h, b.data_ptr(), x.data_ptr(), float(shift), float(rtol), int(max_iter),
                                ctypes.byref(it), ctypes.byref(res), _stream_ptr(b.device)))
        return x, it.value, res.value

    def sync_status(self) -> None:
        _check(_L().hh_sync_status(self._h, _stream_ptr(self.device)))


def optimal_switch_level(points, kernel: int = INV_R, kernel_param: float = 1.0, leaf_size: int = 128,
                         eta: float = 1.0, tol: float = 1e-6, fmt_mask: int = F64 | F32 | F16 | BF16,
                         seed: int = 0, tree: str = "kd", device: int = -1) -> tuple:
    """Algorithm 2 (hh_optimal_switch_level): the switching level with the
    largest storage gain over the H_s matrix.  Returns (ell*, L, {level: gain})
    with gain = S_s - S_h(level) in fp64 words for every level evaluated
    (tree levels; tree "kd" or "2d").  device >= 0: the compressions of the
    evaluated levels run on that GPU (hh_optimal_switch_level_dev)."""
    pts = np.ascontiguousarray(points.cpu().numpy() if isinstance(points, torch.Tensor) else points,
                               dtype=np.float64)
    if pts.ndim != 2:
        raise ValueError("points must be (n, dim)")
    ell, depth = ctypes.c_int(), ctypes.c_int()
    g = (ctypes.c_double * MAX_LEVELS)()
    _check(_L().hh_optimal_switch_level_dev(pts.ctypes.data, pts.shape[0], pts.shape[1], kernel, kernel_param,
                                            leaf_size, eta, tol, fmt_mask, seed, 1 if tree == "2d" else 0,
                                            int(device), ctypes.byref(ell), ctypes.byref(depth), g))
    gains = {l: float(g[l]) for l in range(depth.value + 1) if not np.isnan(g[l])}
    return ell.value, depth.value, gains


def matvec_batched(mats: list, xs: list) -> list:
    """y_i = A_i x_i for independent matrices (one RHS each) in one call."""
    n = len(mats)
    ys = [torch.empty_like(x) for x in xs]
    hs = (ctypes.c_void_p * n)(*[m._h.value for m in mats])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
    _check(_L().hh_matvec_batched(hs, n, xp, yp, _stream_ptr(xs[0].device) if n else 0))
    return ys


class HBatch:
    """Independent matrices (one right-hand side each) multiplied in one launch
    sequence over concatenated vectors: matrix i's vector is
    x[offsets[i]:offsets[i+1]] in its own point order.  The matrices must stay
    open while the batch exists."""

    def __init__(self, mats: list):
        self.mats = list(mats)
        hs = (ctypes.c_void_p * len(mats))(*[m._h.value for m in mats])
        out = ctypes.c_void_p()
        _check(_L().hh_batch_create(hs, len(mats), ctypes.byref(out)))
        self._b = out
        offs = (ctypes.c_int64 * (len(mats) + 1))()
        _check(_L().hh_batch_offsets(self._b, offs))
        self.offsets = [int(v) for v in offs]
        self.device = mats[0].device

    def matvec(self, x: torch.Tensor, transpose: bool = False, out: torch.Tensor | None = None,
               graph: bool = False) -> torch.Tensor:
        """y = blockdiag(A_i) x (graph=True: replay a captured CUDA graph)."""
        if x.dtype != torch.float64 or not x.is_cuda or x.dim() != 1 or not x.is_contiguous() \
                or x.numel() != self.offsets[-1]:
            raise ValueError("x must be a contiguous float64 CUDA vector of the concatenated size")
        y = torch.empty_like(x) if out is None else out
        f = _L().hh_batch_matvec_graph if graph else _L().hh_batch_matvec
        _check(f(self._b, 1 if transpose else 0, x.data_ptr(), y.data_ptr(), _stream_ptr(x.device)))
        return y

    def close(self) -> None:
        if getattr(self, "_b", None) and self._b.value:
            _L().hh_batch_free(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HhMatvec(torch.autograd.Function):
    """y = A_h x with the hand-written backward x_bar = A_h^T y_bar."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, H: HMatrix) -> torch.Tensor:
        ctx.H = H
        return H.matvec(x)

    @staticmethod
    def backward(ctx, ybar: torch.Tensor):
        return ctx.H.matvec(ybar.contiguous() if ybar.dim() == 1 else ybar, transpose=True), None


def hh_apply(H: HMatrix, x: torch.Tensor) -> torch.Tensor:
    return HhMatvec.apply(x, H)
