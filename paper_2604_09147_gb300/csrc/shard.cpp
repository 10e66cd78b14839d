// Row-block ownership of the H_h product on several GPUs, and the matrix of
// one owner's block rows.
//
// Algorithm 4 computes b_I = sum over the blocks (I, J) of block row I, and
// block rows are independent: the rows of b split into contiguous ranges of
// tree positions, one per rank, and each rank needs only the blocks whose row
// cluster meets its range, all of x (one all-gather) and, for the transpose,
// its own rows of y_bar, with the contributions to x_bar summed over ranks
// (one reduce-scatter).
//
// shard_plan: the ranges are unions of consecutive clusters of a tree level
// l0 = min(L, ceil(log2 nranks) + 3) (eight clusters per rank or more), cut
// where the running cost crosses r / nranks of the total.  The cost of a
// cluster is the factor and dense bytes its rows stream: per block row
// segment |rows in c| k sz of U plus the share |rows in c| / m of V's n k sz
// (a block that spans several ranges is cut by rows, and every owner reads
// all of its V), plus 8 m n per dense block.
//
// make_shard: the rows [p0, p1) of every block that meets them, with U cut
// to those rows and V kept whole, compacted into a new arena; dense blocks
// inside the range; the points in tree order and the identity permutation,
// so that a shard's input and output vectors are in tree order.
#include <algorithm>
#include <cstring>
#include <stdexcept>

#include "hh_host.h"

namespace hh {

namespace {

int64_t ld_rows(int64_t rows, int fmt) {
  const int64_t per = 16 / fmt_bytes(fmt);
  return (rows + per - 1) / per * per;
}

int64_t align256(int64_t v) { return (v + 255) / 256 * 256; }

}  // namespace

void shard_plan(const HostMatrix& h, int nranks, std::vector<int64_t>& bounds) {
  if (nranks < 1) throw std::invalid_argument("nranks must be >= 1");
  bounds.assign(static_cast<size_t>(nranks) + 1, 0);
  bounds[nranks] = h.n;
  if (nranks == 1) return;
  int lg = 0;
  while ((1 << lg) < nranks) ++lg;
  const int l0 = std::min<int>(h.L, lg + 3);
  const int64_t nc = int64_t(1) << l0;
  const int64_t base = nc - 1;  // heap index of cluster 0 at level l0
  std::vector<double> cost(static_cast<size_t>(nc), 0.0);
  // cluster of level l0 holding tree position p (clusters are consecutive ranges)
  auto cluster_of = [&](int64_t p) {
    int64_t lo = 0, hi = nc - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) / 2;
      if (h.node_off[base + mid] <= p) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };
  for (const LRBlock& b : h.lr) {
    if (b.k == 0 || b.m == 0) continue;
    const double sz = fmt_bytes(b.fmt);
    for (int64_t c = cluster_of(b.row_off); c < nc; ++c) {
      const int64_t co = h.node_off[base + c], cs = h.node_size[base + c];
      const int64_t r0 = std::max(co, b.row_off), r1 = std::min(co + cs, b.row_off + b.m);
      if (co >= b.row_off + b.m) break;
      if (r1 <= r0) continue;
      const double rows = double(r1 - r0);
      cost[c] += rows * b.k * sz + double(b.n) * b.k * sz * rows / double(b.m);
    }
  }
  for (const DenseBlock& d : h.dense)
    if (d.m > 0) cost[cluster_of(d.row_off)] += 8.0 * double(d.m) * double(d.n);
  double total = 0.0;
  for (double c : cost) total += c;
  // cut before the first cluster whose running cost reaches r / nranks of the
  // total (or the nearer boundary of the two around that point)
  std::vector<int64_t> cut(static_cast<size_t>(nranks) + 1, 0);
  cut[nranks] = nc;
  double run = 0.0;
  int64_t c = 0;
  for (int r = 1; r < nranks; ++r) {
    const double target = total * r / nranks;
    while (c < nc && run + cost[c] <= target) run += cost[c++];
    int64_t at = c;
    if (c < nc && (run + cost[c]) - target < target - run) at = c + 1;  // closer after this cluster
    at = std::max(at, cut[r - 1]);
    cut[r] = std::min<int64_t>(at, nc);
  }
  for (int r = 1; r < nranks; ++r)
    bounds[r] = cut[r] >= nc ? h.n : h.node_off[base + cut[r]];
}

void make_shard(const HostMatrix& src, int64_t p0, int64_t p1, HostMatrix& out) {
  if (p0 < 0 || p1 < p0 || p1 > src.n) throw std::invalid_argument("shard range outside [0, n]");
  out = HostMatrix();
  out.n = src.n;
  out.dim = src.dim;
  out.L = src.L;
  out.ell = src.ell;
  out.leaf = src.leaf;
  out.kernel = src.kernel;
  out.step = src.step;
  out.eta = src.eta;
  out.tol = src.tol;
  out.kparam = src.kparam;
  out.norm_ht = src.norm_ht;
  out.fmt_mask = src.fmt_mask;
  out.seed = src.seed;
  out.points.resize(src.points.size());
  for (int64_t p = 0; p < src.n; ++p)
    std::memcpy(&out.points[p * src.dim], &src.points[int64_t(src.perm[p]) * src.dim], sizeof(double) * src.dim);
  out.perm.resize(static_cast<size_t>(src.n));
  for (int64_t p = 0; p < src.n; ++p) out.perm[p] = static_cast<int32_t>(p);
  out.node_off = src.node_off;
  out.node_size = src.node_size;
  out.node_lo = src.node_lo;
  out.node_hi = src.node_hi;
  // low-rank blocks: U cut to the owned rows, V whole
  int64_t pos = 0;
  for (const LRBlock& b : src.lr) {
    const int64_t r0 = std::max(b.row_off, p0), r1 = std::min(b.row_off + b.m, p1);
    if (r1 <= r0) continue;
    LRBlock B = b;
    B.row_off = r0;
    B.m = r1 - r0;
    B.ldu = ld_rows(B.m, b.fmt);
    B.ldv = b.ldv;
    const int64_t sz = fmt_bytes(b.fmt);
    B.u_off = pos;
    pos += align256(B.ldu * b.k * sz);
    B.v_off = pos;
    pos += align256(B.ldv * b.k * sz);
    out.lr.push_back(B);
  }
  out.arena.assign(static_cast<size_t>(pos), 0);
  size_t q = 0;
  for (const LRBlock& b : src.lr) {
    const int64_t r0 = std::max(b.row_off, p0), r1 = std::min(b.row_off + b.m, p1);
    if (r1 <= r0) continue;
    const LRBlock& B = out.lr[q++];
    const int64_t sz = fmt_bytes(b.fmt);
    for (int64_t c = 0; c < b.k; ++c)
      std::memcpy(&out.arena[B.u_off + c * B.ldu * sz], &src.arena[b.u_off + (c * b.ldu + (r0 - b.row_off)) * sz],
                  static_cast<size_t>(B.m * sz));
    if (b.k > 0)
      std::memcpy(&out.arena[B.v_off], &src.arena[b.v_off], static_cast<size_t>(b.ldv * b.k * sz));
  }
  // dense blocks: whole inside the range (ranges end at cluster boundaries)
  int64_t dpos = 0;
  for (const DenseBlock& d : src.dense) {
    if (d.row_off + d.m <= p0 || d.row_off >= p1) continue;
    if (d.row_off < p0 || d.row_off + d.m > p1)
      throw std::invalid_argument("shard range cuts a dense block (bounds must be cluster boundaries)");
    DenseBlock D = d;
    D.d_off = dpos;
    dpos += d.m * d.n;
    out.dense.push_back(D);
  }
  out.dense_data.resize(static_cast<size_t>(dpos));
  size_t di = 0;
  for (const DenseBlock& d : src.dense) {
    if (d.row_off + d.m <= p0 || d.row_off >= p1) continue;
    std::memcpy(&out.dense_data[out.dense[di++].d_off], &src.dense_data[d.d_off],
                sizeof(double) * static_cast<size_t>(d.m * d.n));
  }
}

}  // namespace hh
