"""The H_h product with its block rows split over the ranks of a
torch.distributed process group (one GPU per rank).

Algorithm 4's block rows are independent: rank r owns the tree positions
[bounds[r], bounds[r+1]) of hh_shard_plan and holds the shard of those block
rows (hh_shard), whose vectors are in tree order.  Vectors are distributed by
the same ranges: a rank holds x_tree[p0:p1], the entries of x at the tree
positions it owns (scatter / gather convert from and to the caller's order).

    forward    y = A_h x:     all-gather x (8 N bytes), y_tree = shard(x_tree),
                              keep rows [p0, p1) (no reduction);
    transpose  x_bar = A_h^T y_bar: y_bar zero outside [p0, p1),
                              x_part = shard^T(y_bar), reduce-scatter of the
                              parts (8 N bytes), keep rows [p0, p1).

Ranges of unequal length travel padded to the longest one.  The collectives
are torch.distributed's (NCCL between GPUs, gloo on CPU); this module does no
arithmetic of the method: the products run in the shard's kernels, or in any
object with the same ``matvec(x, transpose=...)`` method.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


class RowSharded:
    def __init__(self, H, group=None, local=None, device=None):
        """H: the whole matrix (host-only handles suffice); local: the rank's
        product on its tree-order block rows (default: H.shard(p0, p1) on
        `device`, which defaults to H's)."""
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.n = H.n
        self.bounds = H.shard_plan(self.world)
        self.p0, self.p1 = self.bounds[self.rank], self.bounds[self.rank + 1]
        self.width = max(b - a for a, b in zip(self.bounds, self.bounds[1:]))
        self.perm = torch.from_numpy(H.perm().astype("int64"))  # tree position -> caller index
        self.local = local if local is not None else H.shard(self.p0, self.p1, device)

    # -- distribution of vectors ------------------------------------------------
    def scatter(self, x_user: torch.Tensor) -> torch.Tensor:
        """This rank's entries of a caller-order vector: x[perm[p0:p1]]."""
        return x_user[self.perm[self.p0:self.p1].to(x_user.device)]

    def gather(self, v_local: torch.Tensor) -> torch.Tensor:
        """The whole caller-order vector from every rank's entries."""
        vt = self._all_gather(v_local)
        out = torch.empty_like(vt)
        out[self.perm.to(vt.device)] = vt
        return out

    def _all_gather(self, v_local: torch.Tensor) -> torch.Tensor:
        pad = torch.zeros(self.width, dtype=v_local.dtype, device=v_local.device)
        pad[:v_local.shape[0]] = v_local
        buf = torch.empty(self.world * self.width, dtype=v_local.dtype, device=v_local.device)
        dist.all_gather_into_tensor(buf, pad, group=self.group)
        return torch.cat([buf[r * self.width:r * self.width + (b - a)]
                          for r, (a, b) in enumerate(zip(self.bounds, self.bounds[1:]))])

    def _reduce_scatter(self, v_full: torch.Tensor) -> torch.Tensor:
        buf = torch.zeros(self.world * self.width, dtype=v_full.dtype, device=v_full.device)
        for r, (a, b) in enumerate(zip(self.bounds, self.bounds[1:])):
            buf[r * self.width:r * self.width + (b - a)] = v_full[a:b]
        out = torch.empty(self.width, dtype=v_full.dtype, device=v_full.device)
        dist.reduce_scatter_tensor(out, buf, group=self.group)
        return out[:self.p1 - self.p0]

    # -- products ----------------------------------------------------------------
    def matvec(self, x_local: torch.Tensor) -> torch.Tensor:
        """Rows [p0, p1) (tree order) of A_h x, from this rank's x entries."""
        y = self.local.matvec(self._all_gather(x_local))
        return y[self.p0:self.p1]

    def matvec_T(self, ybar_local: torch.Tensor) -> torch.Tensor:
        """Rows [p0, p1) (tree order) of A_h^T y_bar, from this rank's y_bar entries."""
        yb = torch.zeros(self.n, dtype=ybar_local.dtype, device=ybar_local.device)
        yb[self.p0:self.p1] = ybar_local
        return self._reduce_scatter(self.local.matvec(yb, transpose=True))
