"""The row-sharded product on CPU ranks (gloo), world sizes 2 and 3.

Each rank takes its range of block rows from the library's hh_shard_plan,
its shard from hh_shard (host only), and computes that shard's product with
the ORACLE (Algorithm 4 over the shard's stored factors, read back from the
file hh_save writes); paper_2604_09147_gb300.dist supplies the all-gather of
x and the reduce-scatter of the transpose's parts.  The assembled y = A_h x
and x_bar = A_h^T y_bar must equal the oracle's product of the whole matrix
element by element (up to the order of floating-point additions).  No GPU is
involved: this checks the ownership split, the shards' contents and the
collectives' plumbing.
"""
import os
import socket

import numpy as np
import pytest

import hh_workloads as W

torch = pytest.importorskip("torch")
ALL = W.F64 | W.F32 | W.F16 | W.BF16 | W.E4M3


class OracleShard:
    """The oracle's Algorithm 4 over a shard's factors (tree order)."""

    def __init__(self, H, p0, p1, path):
        from oracle import hhfile
        H.shard(p0, p1, device=-1).save(path)
        self.G = hhfile.read(path)
        assert np.array_equal(self.G.perm, np.arange(H.n))

    def matvec(self, x, transpose=False):
        from oracle import matvec as M
        xn = x.numpy()
        return torch.from_numpy(M.matvec_T(self.G, xn) if transpose else M.matvec(self.G, xn))


def _rank_main(rank, world, port, path, tmp, x, ybar, y_ref, xb_ref):
    import torch.distributed as dist

    import paper_2604_09147_gb300 as P
    from paper_2604_09147_gb300.dist import RowSharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        H = P.HMatrix.load(path, device=-1)
        b = H.shard_plan(world)
        assert b[0] == 0 and b[-1] == H.n and all(u <= v for u, v in zip(b, b[1:]))
        local = OracleShard(H, b[rank], b[rank + 1], os.path.join(tmp, f"shard{rank}.hhm"))
        rs = RowSharded(H, local=local)
        y = rs.gather(rs.matvec(rs.scatter(torch.from_numpy(x)))).numpy()
        xb = rs.gather(rs.matvec_T(rs.scatter(torch.from_numpy(ybar)))).numpy()
        for got, ref in ((y, y_ref), (xb, xb_ref)):
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max()), \
                float(np.abs(got - ref).max() / np.abs(ref).max())
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_row_sharded_product_matches_oracle(tmp_path, world):
    import torch.multiprocessing as mp

    from oracle import build as OB
    from oracle import hhfile
    from oracle import matvec as M
    n = 3000
    O = OB.build(W.points(n, 3, 801), W.INV_R, 1.0, 64, 1.0, 3, 1e-5, ALL)
    path = str(tmp_path / "full.hhm")
    hhfile.write(O, path)
    x = W.rhs(n, 1, "uniform", 802)[:, 0]
    ybar = W.rhs(n, 1, "normal", 803)[:, 0]
    mp.spawn(_rank_main, args=(world, _free_port(), path, str(tmp_path), x, ybar, M.matvec(O, x),
                               M.matvec_T(O, ybar)), nprocs=world, join=True)


def test_shard_plan_balances_and_respects_clusters():
    """The ranges are unions of clusters and their costs are balanced to
    within one cluster's cost of the mean."""
    import paper_2604_09147_gb300 as P
    H = P.HMatrix.build(W.points(20000, 3, 804), W.INV_R, 1.0, 64, 1.0, -1, 1e-5, ALL, device=-1)
    path = "/tmp/hh_shard_plan_test.hhm"
    H.save(path)
    from oracle import hhfile
    G = hhfile.read(path)
    os.remove(path)
    for world in (2, 3, 4, 8):
        b = H.shard_plan(world)
        L = G.tree.L
        starts = {int(G.tree.off[(1 << L) - 1 + i]) for i in range(1 << L)} | {H.n}
        assert all(v in starts for v in b)
        # bytes streamed per range: U rows inside + row share of V + dense
        cost = np.zeros(world)
        sz = {0: 8, 1: 4, 2: 2, 3: 2, 4: 1}
        for blk in G.lowrank:
            for r in range(world):
                lo, hi = max(blk.row_off, b[r]), min(blk.row_off + blk.m, b[r + 1])
                if hi > lo:
                    cost[r] += (hi - lo) * blk.k * sz[blk.fmt] * (1 + blk.n / blk.m)
        for d in G.dense:
            r = int(np.searchsorted(b, d.row_off, side="right") - 1)
            cost[r] += 8.0 * d.m * d.n
        assert cost.max() <= 1.35 * cost.mean(), (world, cost / cost.mean())
