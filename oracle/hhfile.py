"""Serialized H_h file: the input both the oracle and the CUDA path consume.

Little-endian layout (version 1):
  magic      8 bytes  b"HHMATv01"
  ints       int64[16]: N, dim, L, ell, leaf_size, kernel, n_lr, n_dense,
                        fmt_mask, arena_bytes, dense_elems, n_nodes, seed,
                        step, 0, 0
             (step: binary levels per tree level, 1 for the KD tree, d for
             the 2^d-tree; 0 is read as 1.  L, ell and block levels are
             binary levels.)
  reals      float64[8]: eta, tol, kernel_param, ||H~||_F, 0, 0, 0, 0
  points     float64[N * dim]   (user order, row-major)
  perm       int32[N]           (perm[p] = user index of tree position p)
  nodes      n_nodes x {int64 off, int64 size, float64 lo[dim], float64 hi[dim]}
  lowrank    n_lr x {int32 level, kind, i, j; int64 row_off, m, col_off, n;
                     int32 k, fmt, exp_u, exp_v; int64 u_off, v_off, ldu, ldv;
                     float64 norm}                                   (104 bytes)
  dense      n_dense x {int32 level, i, j, 0; int64 row_off, m, col_off, n, d_off}
  arena      uint8[arena_bytes]: every factor column-major in its format,
             u_off / v_off multiples of 16 bytes, ld * element size a
             multiple of 16 bytes, rows m..ld-1 of each column zero
  dense data float64[dense_elems]: each dense block column-major, ld = m

Decoded factor value = stored value * 2^exp.  This module reads and writes
the format with NumPy only.
"""
from __future__ import annotations

import numpy as np

from . import formats as F
from .build import DenseBlock, HMatrix, LRBlock
from .tree import Tree

MAGIC = b"HHMATv01"
LR_DT = np.dtype([("level", "<i4"), ("kind", "<i4"), ("i", "<i4"), ("j", "<i4"),
                  ("row_off", "<i8"), ("m", "<i8"), ("col_off", "<i8"), ("n", "<i8"),
                  ("k", "<i4"), ("fmt", "<i4"), ("exp_u", "<i4"), ("exp_v", "<i4"),
                  ("u_off", "<i8"), ("v_off", "<i8"), ("ldu", "<i8"), ("ldv", "<i8"),
                  ("norm", "<f8")])
DN_DT = np.dtype([("level", "<i4"), ("i", "<i4"), ("j", "<i4"), ("pad", "<i4"),
                  ("row_off", "<i8"), ("m", "<i8"), ("col_off", "<i8"), ("n", "<i8"),
                  ("d_off", "<i8")])
assert LR_DT.itemsize == 104 and DN_DT.itemsize == 56


def _node_dt(dim):
    return np.dtype([("off", "<i8"), ("size", "<i8"), ("lo", "<f8", (dim,)), ("hi", "<f8", (dim,))])


def _ld(rows: int, fmt: int) -> int:
    per = 16 // F.BYTES[fmt]
    return -(-rows // per) * per


def write(H: HMatrix, path: str, seed: int = 0) -> None:
    t = H.tree
    nn = len(t.off)
    lr = np.zeros(len(H.lowrank), dtype=LR_DT)
    chunks = []
    pos = 0

    def put(stored, fmt):
        nonlocal pos
        rows, k = stored.shape
        ld = _ld(rows, fmt)
        buf = np.zeros((k, ld), dtype=np.float64)
        buf[:, :rows] = stored.T
        raw = F.encode_bits(buf.reshape(-1), fmt).tobytes()
        off = pos
        pad = (-len(raw)) % 256
        chunks.append(raw + b"\0" * pad)
        pos += len(raw) + pad
        return off, ld

    for idx, b in enumerate(H.lowrank):
        u_off, ldu = put(b.Us, b.fmt)
        v_off, ldv = put(b.Vs, b.fmt)
        lr[idx] = (b.level, b.kind, b.i, b.j, b.row_off, b.m, b.col_off, b.n, b.k, b.fmt,
                   b.exp_u, b.exp_v, u_off, v_off, ldu, ldv, b.norm)
    dn = np.zeros(len(H.dense), dtype=DN_DT)
    dparts = []
    dpos = 0
    for idx, d in enumerate(H.dense):
        dn[idx] = (d.level, d.i, d.j, 0, d.row_off, d.m, d.col_off, d.n, dpos)
        dparts.append(np.asfortranarray(d.D).reshape(-1, order="F"))
        dpos += d.m * d.n
    nodes = np.zeros(nn, dtype=_node_dt(H.dim))
    nodes["off"], nodes["size"], nodes["lo"], nodes["hi"] = t.off, t.size, t.lo, t.hi
    ints = np.array([H.n, H.dim, t.L, H.ell, H.leaf_size, H.kernel, len(lr), len(dn),
                     H.fmt_mask, pos, dpos, nn, seed, t.step, 0, 0], dtype="<i8")
    reals = np.array([H.eta, H.tol, H.kernel_param, H.norm_Ht, 0, 0, 0, 0], dtype="<f8")
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(ints.tobytes())
        f.write(reals.tobytes())
        f.write(np.ascontiguousarray(H.points, dtype="<f8").tobytes())
        f.write(t.perm.astype("<i4").tobytes())
        f.write(nodes.tobytes())
        f.write(lr.tobytes())
        f.write(dn.tobytes())
        for c in chunks:
            f.write(c)
        for p in dparts:
            f.write(p.astype("<f8").tobytes())


def read(path: str) -> HMatrix:
    """Read a file into an HMatrix whose factors hold the stored values
    (H~ factors U, V are not part of the file and are left as None)."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != MAGIC:
        raise ValueError("not an H_h file")
    p = 8
    ints = np.frombuffer(data, "<i8", 16, p); p += 128
    reals = np.frombuffer(data, "<f8", 8, p); p += 64
    n, dim, L, ell, leaf, kernel, nlr, ndn, mask, abytes, delems, nn = (int(v) for v in ints[:12])
    pts = np.frombuffer(data, "<f8", n * dim, p).reshape(n, dim).copy(); p += 8 * n * dim
    perm = np.frombuffer(data, "<i4", n, p).astype(np.int64); p += 4 * n
    ndt = _node_dt(dim)
    nodes = np.frombuffer(data, ndt, nn, p); p += ndt.itemsize * nn
    lr = np.frombuffer(data, LR_DT, nlr, p); p += LR_DT.itemsize * nlr
    dn = np.frombuffer(data, DN_DT, ndn, p); p += DN_DT.itemsize * ndn
    arena = np.frombuffer(data, np.uint8, abytes, p); p += abytes
    dd = np.frombuffer(data, "<f8", delems, p); p += 8 * delems
    if p != len(data):
        raise ValueError("trailing or missing bytes in H_h file")
    tree = Tree(L=L, perm=perm, off=nodes["off"].astype(np.int64), size=nodes["size"].astype(np.int64),
                lo=np.array(nodes["lo"]), hi=np.array(nodes["hi"]), step=max(1, int(ints[13])))
    H = HMatrix(n=n, dim=dim, kernel=kernel, kernel_param=float(reals[2]), leaf_size=leaf,
                eta=float(reals[0]), ell=ell, tol=float(reals[1]), fmt_mask=mask, points=pts,
                tree=tree, norm_Ht=float(reals[3]))

    def get(off, ld, rows, k, fmt):
        sz = F.BYTES[fmt]
        if off % 16 or (ld * sz) % 16 or ld < rows or off + ld * k * sz > abytes:
            raise ValueError("bad factor layout")
        raw = arena[off:off + ld * k * sz]
        vals = F.decode_bits(raw.copy(), fmt).reshape(k, ld)
        return np.ascontiguousarray(vals[:, :rows].T)

    for r in lr:
        fmt, k = int(r["fmt"]), int(r["k"])
        Us = get(int(r["u_off"]), int(r["ldu"]), int(r["m"]), k, fmt)
        Vs = get(int(r["v_off"]), int(r["ldv"]), int(r["n"]), k, fmt)
        H.lowrank.append(LRBlock(int(r["level"]), int(r["kind"]), int(r["i"]), int(r["j"]),
                                 int(r["row_off"]), int(r["m"]), int(r["col_off"]), int(r["n"]),
                                 None, None, None, float(r["norm"]), fmt, int(r["exp_u"]),
                                 int(r["exp_v"]), Us, Vs))
    for r in dn:
        m, nc, o = int(r["m"]), int(r["n"]), int(r["d_off"])
        D = dd[o:o + m * nc].reshape(nc, m).T.copy()
        H.dense.append(DenseBlock(int(r["level"]), int(r["i"]), int(r["j"]), int(r["row_off"]),
                                  m, int(r["col_off"]), nc, D))
    return H
