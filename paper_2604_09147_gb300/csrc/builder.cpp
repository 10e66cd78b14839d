// Host builder of the H_h matrix: cluster tree, hybrid partition
// (Algorithm 1), LRcompression, Frobenius norms (Algorithm 5), adaptive
// precision assignment (Algorithm 3) and the format-grouped factor arena.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <numeric>
#include <stdexcept>
#include <thread>
#include <tuple>

#include "construct.h"
#include "hh_host.h"
#include "linalg.h"

namespace hh {

int fmt_bytes(int fmt) {
  static const int b[NFMT] = {8, 4, 2, 2, 1};
  return b[fmt];
}
int fmt_bits(int fmt) { return 8 * fmt_bytes(fmt); }
double unit_roundoff(int fmt) {
  // u = 2^-(mantissa bits + 1) (Table 1; 2^-4 for the 1-4-3 format)
  static const double u[NFMT] = {0x1p-53, 0x1p-24, 0x1p-11, 0x1p-8, 0x1p-4};
  return u[fmt];
}

namespace {

// ---------------------------------------------------------------- kernels
// Eq. 5.1: H_ij = f(|x_i - x_j|), f(0) = 0 for the singular kernels.
inline double kernel_value(int kernel, double p, double r) {
  switch (kernel) {
    case 0: return std::exp(-r / p);
    case 1: return r == 0.0 ? 0.0 : 1.0 / r;
    case 2: return std::exp(-(r * r) / p);
    case 3: return r == 0.0 ? 0.0 : std::log(r);
    default: return r == 0.0 ? 0.0 : 1.0 / (r * r);
  }
}

struct Geometry {
  const double* pts;  // tree-ordered points, n x dim
  int dim;
  int kernel;
  double p;
  double entry(int64_t a, int64_t b) const {
    const double* x = pts + a * dim;
    const double* y = pts + b * dim;
    double s = 0.0;
    for (int d = 0; d < dim; ++d) {
      double t = x[d] - y[d];
      s = s + t * t;
    }
    return kernel_value(kernel, p, std::sqrt(s));
  }
};

// -------------------------------------------------------------------- tree
int tree_depth(int64_t n, int64_t leaf) {
  int L = 0;
  while ((n + (int64_t(1) << L) - 1) >> L > leaf) ++L;
  return L;
}

void build_tree(const double* pts, int64_t n, int dim, int leaf, HostMatrix& h) {
  const int L = tree_depth(n, leaf);
  const int64_t nn = (int64_t(2) << L) - 1;
  h.L = L;
  h.node_off.assign(nn, 0);
  h.node_size.assign(nn, 0);
  h.node_lo.assign(nn * dim, 0.0);
  h.node_hi.assign(nn * dim, 0.0);
  std::vector<int64_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  h.node_size[0] = n;
  for (int64_t node = 0; node < nn; ++node) {
    const int64_t o = h.node_off[node], s = h.node_size[node];
    double* lo = &h.node_lo[node * dim];
    double* hi = &h.node_hi[node * dim];
    if (s > 0) {
      for (int d = 0; d < dim; ++d) lo[d] = hi[d] = pts[perm[o] * dim + d];
      for (int64_t q = o; q < o + s; ++q)
        for (int d = 0; d < dim; ++d) {
          double v = pts[perm[q] * dim + d];
          lo[d] = std::min(lo[d], v);
          hi[d] = std::max(hi[d], v);
        }
    }
    int level = 63 - __builtin_clzll(static_cast<unsigned long long>(node + 1));
    if (level == L) continue;
    int axis = 0;
    double best = hi[0] - lo[0];
    for (int d = 1; d < dim; ++d)
      if (hi[d] - lo[d] > best) {
        best = hi[d] - lo[d];
        axis = d;
      }
    std::sort(perm.begin() + o, perm.begin() + o + s, [&](int64_t a, int64_t b) {
      double ca = pts[a * dim + axis], cb = pts[b * dim + axis];
      return ca < cb || (ca == cb && a < b);
    });
    const int64_t half = s / 2;
    h.node_off[2 * node + 1] = o;
    h.node_size[2 * node + 1] = half;
    h.node_off[2 * node + 2] = o + half;
    h.node_size[2 * node + 2] = s - half;
  }
  h.perm.resize(n);
  for (int64_t q = 0; q < n; ++q) h.perm[q] = static_cast<int32_t>(perm[q]);
}

// The balanced 2^d-tree (Section 2.1) held in the same heap: binary level b
// splits its cell at the midpoint of axis b mod dim (a point goes up when its
// coordinate is >= the midpoint; each half keeps its parent's order), so
// 2^d-tree level l is binary level dim * l.  The root cell is the smallest
// axis-aligned hypercube around the points; the depth is the smallest l2
// with ceil(n / 2^{dim l2}) <= leaf.  Cells may be empty.  A cluster's
// geometry (node_lo / node_hi) is its cell, the hypercube of Section 2.1's
// analysis.
void build_tree_2d(const double* pts, int64_t n, int dim, int leaf, HostMatrix& h) {
  int l2 = 0;
  while (dim * l2 < 46 && ((n + (int64_t(1) << (dim * l2)) - 1) >> (dim * l2)) > leaf) ++l2;
  const int L = dim * l2;
  const int64_t nn = (int64_t(2) << L) - 1;
  h.L = L;
  h.step = dim;
  h.node_off.assign(nn, 0);
  h.node_size.assign(nn, 0);
  h.node_lo.assign(nn * dim, 0.0);
  h.node_hi.assign(nn * dim, 0.0);
  std::vector<double>& clo = h.node_lo;  // cells
  std::vector<double>& chi = h.node_hi;
  double half = 0.0;
  std::vector<double> mn(dim), mx(dim);
  for (int d = 0; d < dim; ++d) mn[d] = mx[d] = pts[d];
  for (int64_t q = 0; q < n; ++q)
    for (int d = 0; d < dim; ++d) {
      mn[d] = std::min(mn[d], pts[q * dim + d]);
      mx[d] = std::max(mx[d], pts[q * dim + d]);
    }
  for (int d = 0; d < dim; ++d) half = std::max(half, mx[d] - mn[d]);
  half = 0.5 * half;
  for (int d = 0; d < dim; ++d) {
    const double c = 0.5 * (mn[d] + mx[d]);
    clo[d] = c - half;
    chi[d] = c + half;
  }
  std::vector<int64_t> perm(n), tmp(n);
  std::iota(perm.begin(), perm.end(), 0);
  h.node_size[0] = n;
  for (int64_t node = 0; node < nn; ++node) {
    const int64_t o = h.node_off[node], s = h.node_size[node];
    const int level = 63 - __builtin_clzll(static_cast<unsigned long long>(node + 1));
    if (level == L) continue;
    const int axis = level % dim;
    const double mid = 0.5 * (clo[node * dim + axis] + chi[node * dim + axis]);
    int64_t lower = 0;
    for (int64_t q = o; q < o + s; ++q)
      if (pts[perm[q] * dim + axis] < mid) tmp[o + lower++] = perm[q];
    int64_t up = o + lower;
    for (int64_t q = o; q < o + s; ++q)
      if (!(pts[perm[q] * dim + axis] < mid)) tmp[up++] = perm[q];
    for (int64_t q = o; q < o + s; ++q) perm[q] = tmp[q];
    for (int c = 1; c <= 2; ++c)
      for (int d = 0; d < dim; ++d) {
        clo[(2 * node + c) * dim + d] = clo[node * dim + d];
        chi[(2 * node + c) * dim + d] = chi[node * dim + d];
      }
    chi[(2 * node + 1) * dim + axis] = mid;
    clo[(2 * node + 2) * dim + axis] = mid;
    h.node_off[2 * node + 1] = o;
    h.node_size[2 * node + 1] = lower;
    h.node_off[2 * node + 2] = o + lower;
    h.node_size[2 * node + 2] = s - lower;
  }
  h.perm.resize(n);
  for (int64_t q = 0; q < n; ++q) h.perm[q] = static_cast<int32_t>(perm[q]);
}

// --------------------------------------------------------------- partition
double box_diam(const HostMatrix& h, int64_t node) {
  double s = 0.0;
  for (int d = 0; d < h.dim; ++d) {
    double e = h.node_hi[node * h.dim + d] - h.node_lo[node * h.dim + d];
    s = s + e * e;
  }
  return std::sqrt(s);
}

double box_dist(const HostMatrix& h, int64_t a, int64_t b) {
  double s = 0.0;
  for (int d = 0; d < h.dim; ++d) {
    double g1 = h.node_lo[b * h.dim + d] - h.node_hi[a * h.dim + d];
    double g2 = h.node_lo[a * h.dim + d] - h.node_hi[b * h.dim + d];
    double g = std::max(0.0, std::max(g1, g2));
    s = s + g * g;
  }
  return std::sqrt(s);
}

// Eq. 2.2, inclusive.  On the 2^d-tree the clusters are congruent cells and,
// at eta = sqrt(d), cells one cell apart meet the condition with equality
// (admissible in the closed forms of Eqs. 2.3 and 2.5); rounding decides
// such a tie either way, so there the comparison carries a relative slack
// of 1e-12.
bool adm_s(const HostMatrix& h, int64_t a, int64_t b, double eta) {
  double rhs = eta * box_dist(h, a, b);
  if (h.step > 1) rhs = rhs * (1.0 + 1e-12);
  return std::min(box_diam(h, a), box_diam(h, b)) <= rhs;
}

struct Pair {
  int level, i, j, kind;  // kind: LR kinds, or -1 diagonal dense / KIND_NBR dense candidate
};

// On a 2^d-tree (h.step = dim) a pair is refined into the 2^d x 2^d pairs of
// its clusters' children step binary levels down, and pairs with an empty
// cluster are dropped.
void hybrid_partition(const HostMatrix& h, double eta, int ell, std::vector<Pair>& lr,
                      std::vector<Pair>& dense) {
  const int L = h.L, step = h.step;
  std::vector<Pair> stack{{0, 0, 0, 0}};
  while (!stack.empty()) {
    Pair p = stack.back();
    stack.pop_back();
    const int l = p.level;
    const int64_t ni = (int64_t(1) << l) - 1 + p.i, nj = (int64_t(1) << l) - 1 + p.j;
    if (step > 1 && (h.node_size[ni] == 0 || h.node_size[nj] == 0)) continue;
    if (l >= 1) {
      if (l <= ell && adm_s(h, ni, nj, eta)) {
        lr.push_back({l, p.i, p.j, KIND_STD});
        continue;
      }
      if (l == ell && ell < L && p.i != p.j) {
        lr.push_back({l, p.i, p.j, KIND_FINER});
        continue;
      }
      if (l > ell && p.i != p.j) {
        lr.push_back({l, p.i, p.j, KIND_WEAK});
        continue;
      }
    }
    if (l == L) {
      dense.push_back({l, p.i, p.j, p.i == p.j ? -1 : KIND_NBR});
      continue;
    }
    const int c = 1 << step;
    for (int a = c - 1; a >= 0; --a)
      for (int b = c - 1; b >= 0; --b) stack.push_back({l + step, c * p.i + a, c * p.j + b, 0});
  }
}

// ------------------------------------------------------------- compression
struct Compressed {
  la::Mat U, V;
  std::vector<double> s;
};

// Compressions already computed, keyed by (level, i, j).  A block's
// compression depends only on its two clusters and tol, so builds of the same
// points, tree and tol with different switching levels (Algorithm 2) share
// them.
using CompressionCache = std::map<std::tuple<int, int, int>, std::shared_ptr<const Compressed>>;

constexpr int64_t kDenseMax = int64_t(1) << 18;
constexpr double kAcaShare = 0.01;
constexpr int kAcaPatience = 3;

// LRcompression to eps (Eq. 2.1): U orthonormal, V = Z Sigma.
//
// Both paths first reach an approximation A ~= Q M^T with Q orthonormal and
// a small k-column factor, then take the left singular vectors W of a k x k
// matrix by one-sided Jacobi and truncate: U = Q-side times W_r and
// V = M-side times W_r, whose columns have norms sigma_1..sigma_r.
void compress_block(const Geometry& g, int64_t r0, int64_t m, int64_t c0, int64_t n, double eps,
                    Compressed& out) {
  auto empty = [&]() {
    out.U = la::Mat(m, 0);
    out.V = la::Mat(n, 0);
    out.s.clear();
  };
  if (m * n <= kDenseMax) {
    // dense block: column-pivoted QR to eps/100 (exact trailing norm), A ~=
    // Ub R with Ub orthonormal.  With R^T = Qb Rb, the left singular vectors
    // of R are those of Rb^T, and A ~= (Ub W_r)(R^T W_r)^T.
    la::Mat A(m, n);
    for (int64_t c = 0; c < n; ++c)
      for (int64_t r = 0; r < m; ++r) A(r, c) = g.entry(r0 + r, c0 + c);
    la::Mat Ub, R;
    la::cpqr_trunc(std::move(A), kAcaShare * eps, Ub, R);
    const int64_t k = R.m;
    if (k == 0) return empty();
    la::Mat Rt(n, k);  // R^T, n >= k
    for (int64_t i = 0; i < k; ++i)
      for (int64_t c = 0; c < n; ++c) Rt(c, i) = R(i, c);
    la::Mat F = Rt;
    std::vector<double> tau;
    la::qr_factor(F, tau);
    la::Mat Rb = la::qr_r(F), RbT(k, k);
    for (int64_t c = 0; c < k; ++c)
      for (int64_t r = 0; r < k; ++r) RbT(r, c) = Rb(c, r);
    la::Mat W;
    std::vector<double> s;
    la::svd_left(RbT, W, s);
    const int r = la::trunc_rank(s, (1.0 - kAcaShare) * eps);
    out.s.assign(s.begin(), s.begin() + r);
    out.U = la::Mat(m, r);
    out.V = la::Mat(n, r);
    la::gemm(m, r, k, 1.0, Ub.a.data(), 1, m, W.a.data(), 1, k, out.U.a.data(), m);
    la::gemm(n, r, k, 1.0, Rt.a.data(), 1, n, W.a.data(), 1, k, out.V.a.data(), n);
    return;
  }
  la::Mat U, V;
  la::aca([&](int64_t i, double* o) { for (int64_t c = 0; c < n; ++c) o[c] = g.entry(r0 + i, c0 + c); },
          [&](int64_t j, double* o) { for (int64_t r = 0; r < m; ++r) o[r] = g.entry(r0 + r, c0 + j); },
          m, n, kAcaShare * eps, kAcaPatience, U, V);
  const int64_t k = U.n;
  if (k == 0) return empty();
  // A ~= Qu T Qv^T with T = Ru Rv^T.  Left singular vectors of T, QR
  // preconditioned for the Jacobi sweeps: T = Q1 R1 (column pivoting, R1
  // graded), R1^T = Q2 R2, so T = Q1 R2^T Q2^T and the left singular vectors
  // of T are Q1 times those of R2^T, whose columns are nearly orthogonal.
  // Then U = Qu (Q1 W_r) and V = Qv (T^T Q1 W_r).
  std::vector<double> tu, tv;
  la::qr_factor(U, tu);
  la::qr_factor(V, tv);
  la::Mat Ru = la::qr_r(U), Rv = la::qr_r(V), T(k, k);
  la::gemm(k, k, k, 1.0, Ru.a.data(), 1, k, Rv.a.data(), k, 1, T.a.data(), k);
  la::Mat Q1, R1;
  la::cpqr_trunc(T, 0.0, Q1, R1);
  const int64_t k1 = R1.m;
  if (k1 == 0) return empty();
  la::Mat F(k, k1);  // R1^T
  for (int64_t i = 0; i < k1; ++i)
    for (int64_t c = 0; c < k; ++c) F(c, i) = R1(i, c);
  std::vector<double> t2;
  la::qr_factor(F, t2);
  la::Mat R2 = la::qr_r(F), X(k1, k1);
  for (int64_t c = 0; c < k1; ++c)
    for (int64_t r = 0; r <= c; ++r) X(c, r) = R2(r, c);
  la::Mat W;
  std::vector<double> s;
  la::svd_left(X, W, s);
  const int r = la::trunc_rank(s, (1.0 - kAcaShare) * eps);
  out.s.assign(s.begin(), s.begin() + r);
  la::Mat Wt(k, r), Y(k, r);
  la::gemm(k, r, k1, 1.0, Q1.a.data(), 1, k, W.a.data(), 1, k1, Wt.a.data(), k);
  la::gemm(k, r, k, 1.0, T.a.data(), k, 1, Wt.a.data(), 1, k, Y.a.data(), k);
  la::qr_apply_q(U, tu, Wt, out.U);
  la::qr_apply_q(V, tv, Y, out.V);
}

// ----------------------------------------------------------------- formats
struct FmtSpec {
  int mbits, emin;
  double vmax, target;
};
FmtSpec fmt_spec(int fmt) {
  switch (fmt) {
    case F64: return {52, -1022, 1.7976931348623157e308, 1.0};
    case F32: return {23, -126, 3.4028234663852886e38, 1.0};
    case F16: return {10, -14, 65504.0, 65504.0};
    case BF16: return {7, -126, 3.3895313892515355e38, 1.0};
    default: return {3, -6, 448.0, 448.0};
  }
}

// round-to-nearest-even of v into fmt (subnormals kept); exact in double
double round_to(double v, int fmt) {
  if (fmt == F64 || v == 0.0) return v;
  FmtSpec sp = fmt_spec(fmt);
  int E;
  std::frexp(v, &E);
  int e = std::max(E - 1, sp.emin);
  double q = std::ldexp(1.0, e - sp.mbits);
  double r = std::nearbyint(v / q) * q;
  if (std::fabs(r) > sp.vmax) throw std::runtime_error("factor value exceeds format range");
  return r;
}

// power-of-two scale: every factor's largest magnitude lands in (t/2, t],
// t = the format's maximum for fp16 / e4m3, 1 for fp32 / bf16 / fp64
int scale_exponent(double maxabs, int fmt) {
  if (maxabs == 0.0) return 0;
  const double t = fmt_spec(fmt).target;
  int E;
  std::frexp(maxabs / t, &E);
  int e = E;
  while (std::ldexp(maxabs, -e) > t) ++e;
  while (std::ldexp(maxabs, -(e - 1)) <= t) --e;
  return e;
}

void store_value(uint8_t* dst, double r, int fmt) {
  switch (fmt) {
    case F64: std::memcpy(dst, &r, 8); return;
    case F32: {
      float f = static_cast<float>(r);
      std::memcpy(dst, &f, 4);
      return;
    }
    case BF16: {
      float f = static_cast<float>(r);
      uint32_t w;
      std::memcpy(&w, &f, 4);
      uint16_t b = static_cast<uint16_t>(w >> 16);
      std::memcpy(dst, &b, 2);
      return;
    }
    case F16: {
      uint16_t s = std::signbit(r) ? 0x8000 : 0;
      double a = std::fabs(r);
      uint16_t bits;
      if (a < 0x1p-14) {
        bits = static_cast<uint16_t>(std::lrint(a / 0x1p-24));
      } else {
        int E;
        std::frexp(a, &E);
        int e = E - 1;
        uint16_t mant = static_cast<uint16_t>(std::lrint((std::ldexp(a, -e) - 1.0) * 1024.0));
        bits = static_cast<uint16_t>(((e + 15) << 10) | mant);
      }
      bits |= s;
      std::memcpy(dst, &bits, 2);
      return;
    }
    default: {  // e4m3fn
      uint8_t s = std::signbit(r) ? 0x80 : 0;
      double a = std::fabs(r);
      uint8_t bits;
      if (a < 0x1p-6) {
        bits = static_cast<uint8_t>(std::lrint(a / 0x1p-9));
      } else {
        int E;
        std::frexp(a, &E);
        int e = E - 1;
        uint8_t mant = static_cast<uint8_t>(std::lrint((std::ldexp(a, -e) - 1.0) * 8.0));
        bits = static_cast<uint8_t>(((e + 7) << 3) | mant);
      }
      *dst = bits | s;
      return;
    }
  }
}

// fmt_mask bit 5: the rule takes Table 1's printed unit roundoff of the
// 8-bit format (2.5e-1) instead of e4m3's 2^-4; storage and bounds keep 2^-4
constexpr uint32_t kRuleQ43 = 1u << 5;

int choose_format(double tau, uint32_t mask) {
  int best = F64;
  double bu = unit_roundoff(F64);
  for (int f = F32; f <= E4M3; ++f) {
    if (!(mask & (1u << f))) continue;
    double u = (f == E4M3 && (mask & kRuleQ43)) ? 0.25 : unit_roundoff(f);
    if (u <= tau && u > bu) {
      best = f;
      bu = u;
    }
  }
  return best;
}

double block_tau(double tol, int level, double nb, double nall) {
  double xi = nb / nall;
  if (xi == 0.0) return std::numeric_limits<double>::infinity();
  return tol / (std::sqrt(std::ldexp(1.0, level)) * xi);
}

int64_t ld_for(int64_t rows, int fmt) {
  int64_t per = 16 / fmt_bytes(fmt);
  return (rows + per - 1) / per * per;
}

template <class F>
void parallel_for(int64_t count, int threads, F&& fn) {
  if (count <= 0) return;
  int nt = threads > 0 ? threads : static_cast<int>(std::thread::hardware_concurrency());
  if (nt <= 0) nt = 1;
  nt = static_cast<int>(std::min<int64_t>(nt, count));
  std::atomic<int64_t> next{0};
  std::exception_ptr err;
  std::atomic<bool> failed{false};
  auto work = [&]() {
    for (;;) {
      int64_t t = next.fetch_add(1);
      if (t >= count || failed.load()) return;
      try {
        fn(t);
      } catch (...) {
        if (!failed.exchange(true)) err = std::current_exception();
        return;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int i = 1; i < nt; ++i) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  if (err) std::rethrow_exception(err);
}

struct FactorRef {
  LRBlock meta;      // everything but exponents, offsets and leading dims
  const double* U;   // m x k column-major (ld = m), the H~ factor
  const double* V;   // n x k column-major (ld = n)
};

// Lay out the factor arena grouped by format (fp64 first, 256-byte aligned
// factors, leading dimensions padded to 16 bytes) and store every factor in
// its format with a power-of-two scale.
void layout_and_store(const std::vector<FactorRef>& refs, int threads, HostMatrix& h) {
  std::vector<size_t> by_fmt(refs.size());
  std::iota(by_fmt.begin(), by_fmt.end(), 0);
  std::stable_sort(by_fmt.begin(), by_fmt.end(),
                   [&](size_t a, size_t b) { return refs[a].meta.fmt < refs[b].meta.fmt; });
  h.lr.resize(refs.size());
  int64_t pos = 0;
  for (size_t t : by_fmt) {
    LRBlock& B = h.lr[t];
    B = refs[t].meta;
    B.ldu = ld_for(B.m, B.fmt);
    B.ldv = ld_for(B.n, B.fmt);
    const int sz = fmt_bytes(B.fmt);
    B.u_off = pos;
    pos += (B.ldu * B.k * sz + 255) / 256 * 256;
    B.v_off = pos;
    pos += (B.ldv * B.k * sz + 255) / 256 * 256;
  }
  h.arena.assign(static_cast<size_t>(pos), 0);
  parallel_for(static_cast<int64_t>(refs.size()), threads, [&](int64_t t) {
    LRBlock& B = h.lr[t];
    const int sz = fmt_bytes(B.fmt);
    auto put = [&](const double* A, int64_t rows, int64_t off, int64_t ld, int32_t& expo) {
      double mx = 0.0;
      for (int64_t q = 0; q < rows * B.k; ++q) mx = std::max(mx, std::fabs(A[q]));
      expo = scale_exponent(mx, B.fmt);
      for (int64_t c = 0; c < B.k; ++c)
        for (int64_t r = 0; r < rows; ++r) {
          double v = round_to(std::ldexp(A[r + c * rows], -expo), B.fmt);
          store_value(&h.arena[off + (r + c * ld) * sz], v, B.fmt);
        }
    };
    put(refs[t].U, B.m, B.u_off, B.ldu, B.exp_u);
    put(refs[t].V, B.n, B.v_off, B.ldv, B.exp_v);
  });
}

}  // namespace

static void build_impl(const double* points, int64_t n, int dim, const BuildParams& p, HostMatrix& h,
                       CompressionCache* cache) {
  auto t0 = std::chrono::steady_clock::now();
  if (n < 1 || dim < 1 || dim > 3) throw std::invalid_argument("need n >= 1 and 1 <= dim <= 3");
  if (n > (int64_t(1) << 31) - 64) throw std::invalid_argument("n too large for 32-bit positions");
  if (p.leaf < 1) throw std::invalid_argument("leaf_size must be >= 1");
  if (!(p.eta > 0)) throw std::invalid_argument("eta must be > 0");
  if (!(p.tol > 0 && p.tol < 1)) throw std::invalid_argument("tol must be in (0, 1)");
  if (p.kernel < 0 || p.kernel > 4) throw std::invalid_argument("unknown kernel");
  if (!(p.kparam > 0)) throw std::invalid_argument("kernel_param must be > 0");
  if (p.fmt_mask & ~63u) throw std::invalid_argument("unknown bits in fmt_mask");
  for (int64_t i = 0; i < n * dim; ++i)
    if (!std::isfinite(points[i])) throw std::invalid_argument("points must be finite");
  h = HostMatrix();
  h.n = n;
  h.dim = dim;
  h.leaf = p.leaf;
  h.kernel = p.kernel;
  h.eta = p.eta;
  h.tol = p.tol;
  h.kparam = p.kparam;
  h.fmt_mask = p.fmt_mask | 1u;
  h.seed = p.seed;
  h.points.assign(points, points + n * dim);
  if (p.tree == 1)
    build_tree_2d(points, n, dim, p.leaf, h);
  else if (p.tree == 0)
    build_tree(points, n, dim, p.leaf, h);
  else
    throw std::invalid_argument("unknown tree kind");
  if (h.L + 1 > 47) throw std::invalid_argument("tree too deep");
  // ell in tree levels, stored as a binary level
  int ell = (p.ell < 0 ? (h.L / h.step) / 2 : p.ell);
  if (ell > h.L / h.step) throw std::domain_error("switch level exceeds the tree depth L");
  ell *= h.step;
  h.ell = ell;

  std::vector<Pair> lrp, dnp;
  hybrid_partition(h, p.eta, ell, lrp, dnp);

  std::vector<double> tp(static_cast<size_t>(n * dim));
  for (int64_t q = 0; q < n; ++q)
    for (int d = 0; d < dim; ++d) tp[q * dim + d] = points[int64_t(h.perm[q]) * dim + d];
  Geometry g{tp.data(), dim, p.kernel, p.kparam};
  auto rng = [&](int level, int i, int64_t& off, int64_t& size) {
    int64_t node = (int64_t(1) << level) - 1 + i;
    off = h.node_off[node];
    size = h.node_size[node];
  };

  // Algorithm 1: compress the admissible blocks (and, when ell == L, the
  // leaf neighbours, to decide Section 4.3's special case)
  std::vector<Pair> jobs = lrp;
  std::vector<size_t> nbr_idx;
  for (size_t d = 0; d < dnp.size(); ++d)
    if (dnp[d].kind == KIND_NBR) {
      nbr_idx.push_back(d);
      jobs.push_back(dnp[d]);
    }
  std::vector<std::shared_ptr<const Compressed>> comp(jobs.size());
  std::vector<std::shared_ptr<Compressed>> fresh(jobs.size());
  std::vector<int64_t> order;
  std::vector<double> cost(jobs.size());
  for (size_t b = 0; b < jobs.size(); ++b) {
    if (cache) {
      auto it = cache->find(std::make_tuple(jobs[b].level, jobs[b].i, jobs[b].j));
      if (it != cache->end()) {
        comp[b] = it->second;
        continue;
      }
    }
    int64_t o1, m, o2, nn;
    rng(jobs[b].level, jobs[b].i, o1, m);
    rng(jobs[b].level, jobs[b].j, o2, nn);
    cost[b] = double(m) * double(nn);
    fresh[b] = std::make_shared<Compressed>();
    order.push_back(static_cast<int64_t>(b));
  }
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
  std::vector<int64_t> host_jobs = order;
  if (p.device >= 0 && !order.empty()) {
    // LRcompression on the GPU; blocks it leaves (rank capacity, failed
    // factorization) are compressed here
    std::vector<DeviceJob> dj(order.size());
    for (size_t t = 0; t < order.size(); ++t) {
      const Pair& q = jobs[order[t]];
      rng(q.level, q.i, dj[t].r0, dj[t].m);
      rng(q.level, q.j, dj[t].c0, dj[t].n);
    }
    std::vector<la::Mat> du, dv;
    std::vector<std::vector<double>> ds;
    std::vector<char> dok;
    DeviceStats st;
    compress_on_device(p.device, tp.data(), n, dim, p.kernel, p.kparam, p.tol, dj, du, dv, ds, dok, &st);
    host_jobs.clear();
    for (size_t t = 0; t < order.size(); ++t) {
      if (!dok[t]) {
        host_jobs.push_back(order[t]);
        continue;
      }
      Compressed& c = *fresh[order[t]];
      c.U = std::move(du[t]);
      c.V = std::move(dv[t]);
      c.s = std::move(ds[t]);
    }
    h.build_device = p.device;
    h.build_fallback += static_cast<int64_t>(host_jobs.size());
    h.build_device_seconds += st.seconds;
  }
  parallel_for(static_cast<int64_t>(host_jobs.size()), p.threads, [&](int64_t t) {
    const Pair& q = jobs[host_jobs[t]];
    int64_t o1, m, o2, nn;
    rng(q.level, q.i, o1, m);
    rng(q.level, q.j, o2, nn);
    compress_block(g, o1, m, o2, nn, p.tol, *fresh[host_jobs[t]]);
  });
  for (int64_t b : order) {
    comp[b] = fresh[b];
    if (cache) (*cache)[std::make_tuple(jobs[b].level, jobs[b].i, jobs[b].j)] = fresh[b];
  }

  // dense blocks (diagonal; with ell == L also the leaf neighbours)
  std::vector<std::vector<double>> dvals(dnp.size());
  parallel_for(static_cast<int64_t>(dnp.size()), p.threads, [&](int64_t d) {
    int64_t o1, m, o2, nn;
    rng(dnp[d].level, dnp[d].i, o1, m);
    rng(dnp[d].level, dnp[d].j, o2, nn);
    dvals[d].resize(static_cast<size_t>(m * nn));
    for (int64_t c = 0; c < nn; ++c)
      for (int64_t r = 0; r < m; ++r) dvals[d][r + c * m] = g.entry(o1 + r, o2 + c);
  });

  // Algorithm 5: ||H~||^2 = sum trace(Sigma^2) + sum ||H_II||^2 (+ dense neighbours)
  std::vector<double> bnorm(jobs.size());
  double norm2 = 0.0;
  for (size_t b = 0; b < lrp.size(); ++b) {
    double s2 = 0.0;
    for (double s : comp[b]->s) s2 += s * s;
    bnorm[b] = std::sqrt(s2);
    norm2 += s2;
  }
  for (size_t b = lrp.size(); b < jobs.size(); ++b) {
    double s2 = 0.0;
    for (double s : comp[b]->s) s2 += s * s;
    bnorm[b] = std::sqrt(s2);
  }
  for (size_t d = 0; d < dnp.size(); ++d) {
    double s2 = 0.0;
    for (double v : dvals[d]) s2 += v * v;
    norm2 += s2;
  }
  h.norm_ht = std::sqrt(norm2);

  // Algorithm 3: format of every admissible block; Section 4.3 for ell == L
  struct Chosen {
    size_t job;
    int fmt;
  };
  std::vector<Chosen> keep;
  for (size_t b = 0; b < lrp.size(); ++b)
    keep.push_back({b, choose_format(block_tau(p.tol, lrp[b].level, bnorm[b], h.norm_ht), h.fmt_mask)});
  std::vector<char> dense_keep(dnp.size(), 1);
  for (size_t q = 0; q < nbr_idx.size(); ++q) {
    size_t b = lrp.size() + q;
    int64_t o1, m, o2, nn;
    rng(jobs[b].level, jobs[b].i, o1, m);
    rng(jobs[b].level, jobs[b].j, o2, nn);
    int f = choose_format(block_tau(p.tol, jobs[b].level, bnorm[b], h.norm_ht), h.fmt_mask);
    const int64_t pk = comp[b]->U.n;
    if (double(pk) * double(m + nn) * fmt_bits(f) / 64.0 < double(m) * double(nn)) {
      keep.push_back({b, f});
      dense_keep[nbr_idx[q]] = 0;
    }
  }

  std::vector<FactorRef> refs(keep.size());
  for (size_t t = 0; t < keep.size(); ++t) {
    const Chosen& c = keep[t];
    const Pair& q = jobs[c.job];
    LRBlock B;
    std::memset(&B, 0, sizeof(B));
    B.level = q.level;
    B.kind = c.job < lrp.size() ? q.kind : KIND_NBR;
    B.i = q.i;
    B.j = q.j;
    rng(q.level, q.i, B.row_off, B.m);
    rng(q.level, q.j, B.col_off, B.n);
    B.k = static_cast<int32_t>(comp[c.job]->U.n);
    B.fmt = c.fmt;
    B.norm = bnorm[c.job];
    refs[t] = {B, comp[c.job]->U.a.data(), comp[c.job]->V.a.data()};
  }
  layout_and_store(refs, p.threads, h);

  int64_t dpos = 0;
  for (size_t d = 0; d < dnp.size(); ++d) {
    if (!dense_keep[d]) continue;
    DenseBlock D;
    std::memset(&D, 0, sizeof(D));
    D.level = dnp[d].level;
    D.i = dnp[d].i;
    D.j = dnp[d].j;
    rng(D.level, D.i, D.row_off, D.m);
    rng(D.level, D.j, D.col_off, D.n);
    D.d_off = dpos;
    dpos += D.m * D.n;
    h.dense.push_back(D);
    h.dense_data.insert(h.dense_data.end(), dvals[d].begin(), dvals[d].end());
  }
  h.build_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

void build(const double* points, int64_t n, int dim, const BuildParams& p, HostMatrix& h) {
  build_impl(points, n, dim, p, h, nullptr);
}

void reencode(const HostMatrix& src, uint32_t fmt_mask, int threads, HostMatrix& h) {
  if (fmt_mask & ~63u) throw std::invalid_argument("unknown bits in fmt_mask");
  if (src.ell == src.L && src.L > 0)
    throw std::domain_error("re-encoding needs ell < L (with ell == L the dense/low-rank choice depends on the format)");
  for (const LRBlock& b : src.lr)
    if (b.fmt != F64) throw std::invalid_argument("re-encoding needs a matrix stored in uniform fp64");
  h = src;
  h.fmt_mask = fmt_mask | 1u;
  h.lr.clear();
  h.arena.clear();
  // unpack the exact fp64 factors, then apply Algorithm 3 with the new set U
  std::vector<std::vector<double>> fac(2 * src.lr.size());
  std::vector<FactorRef> refs(src.lr.size());
  for (size_t t = 0; t < src.lr.size(); ++t) {
    const LRBlock& b = src.lr[t];
    fac[2 * t].resize(static_cast<size_t>(b.m * b.k));
    fac[2 * t + 1].resize(static_cast<size_t>(b.n * b.k));
    for (int64_t c = 0; c < b.k; ++c) {
      std::memcpy(&fac[2 * t][c * b.m], &src.arena[b.u_off + c * b.ldu * 8], 8 * b.m);
      std::memcpy(&fac[2 * t + 1][c * b.n], &src.arena[b.v_off + c * b.ldv * 8], 8 * b.n);
    }
    for (double& v : fac[2 * t]) v = std::ldexp(v, b.exp_u);       // exact: undo the scales
    for (double& v : fac[2 * t + 1]) v = std::ldexp(v, b.exp_v);
    LRBlock B = b;
    B.fmt = choose_format(block_tau(src.tol, b.level, b.norm, src.norm_ht), h.fmt_mask);
    refs[t] = {B, fac[2 * t].data(), fac[2 * t + 1].data()};
  }
  layout_and_store(refs, threads, h);
}

// Algorithm 2.  The H_s and H_h(ell) storages share the far-field blocks of
// levels 1..ell and the dense diagonal (Section 3.3), so their difference is
// S_1(ell) - S_2(ell); storage is Section 5.2's count in fp64 words with each
// block's format bits (summarize().storage_amp).  Each S_2 evaluation is a
// construction of that H_h matrix (Algorithm 1).
int optimal_switch_level(const double* points, int64_t n, int dim, const BuildParams& p, std::vector<double>& gains,
                         int& depth) {
  if (n < 1 || dim < 1 || p.leaf < 1) throw std::invalid_argument("bad sizes");
  int L = tree_depth(n, p.leaf);  // in tree levels
  if (p.tree == 1) {
    L = 0;
    while (dim * L < 46 && ((n + (int64_t(1) << (dim * L)) - 1) >> (dim * L)) > p.leaf) ++L;
  }
  depth = L;
  gains.assign(static_cast<size_t>(L) + 1, std::nan(""));
  CompressionCache cache;  // the levels share most blocks
  auto storage_at = [&](int ell) {
    BuildParams q = p;
    q.ell = ell;
    HostMatrix h;
    build_impl(points, n, dim, q, h, &cache);
    return summarize(h).storage_amp;
  };
  const double ss = storage_at(L);
  int ell = L;
  double s = 0.0;  // S_1(L) - S_2(L)
  gains[L] = 0.0;
  while (ell > 0) {
    const double s_new = ss - storage_at(ell - 1);
    gains[ell - 1] = s_new;
    if (s_new <= s) break;
    s = s_new;
    --ell;
  }
  return ell;
}

Summary summarize(const HostMatrix& h) {
  Summary s;
  s.csp.assign(static_cast<size_t>(h.L) + 1, 0);
  std::vector<std::vector<int32_t>> cnt(static_cast<size_t>(h.L) + 1);
  for (int l = 0; l <= h.L; ++l) cnt[l].assign(size_t(1) << l, 0);
  for (const LRBlock& b : h.lr) {
    s.blocks_per_fmt[b.fmt] += 1;
    const int64_t fb = (b.m + b.n) * int64_t(b.k) * fmt_bytes(b.fmt);
    s.bytes_per_fmt[b.fmt] += fb;
    s.u_bytes += b.m * int64_t(b.k) * fmt_bytes(b.fmt);
    s.v_bytes += b.n * int64_t(b.k) * fmt_bytes(b.fmt);
    s.max_rank = std::max<int64_t>(s.max_rank, b.k);
    s.storage_amp += double(b.k) * double(b.m + b.n) * fmt_bits(b.fmt) / 64.0;
    s.storage_fp64 += double(b.k) * double(b.m + b.n);
    s.bytes_per_matvec += double(fb);
    s.flops_per_matvec += 2.0 * double(b.k) * double(b.m + b.n);
    if (b.level <= h.L) cnt[b.level][b.i] += 1;
    if (b.fmt != F64) {
      double u = unit_roundoff(b.fmt);
      double e = (2.0 + std::sqrt(double(b.k)) * u) * u * b.norm;
      s.bound_round += e * e;
    }
  }
  for (const DenseBlock& d : h.dense) {
    s.dense_bytes += 8 * d.m * d.n;
    s.storage_amp += double(d.m) * double(d.n);
    s.storage_fp64 += double(d.m) * double(d.n);
    s.bytes_per_matvec += 8.0 * double(d.m) * double(d.n);
    s.flops_per_matvec += 2.0 * double(d.m) * double(d.n);
  }
  s.bytes_per_matvec += 16.0 * double(h.n);  // x read once, y written once
  double sum = 0.0;
  for (int l = 0; l <= h.L; ++l) {
    for (int32_t c : cnt[l]) s.csp[l] = std::max(s.csp[l], c);
    sum += s.csp[l];
  }
  s.bound42 = (2.0 * std::sqrt(sum) + 1.0) * h.tol;
  s.bound44 = 2.0 * s.bound42;
  s.bound_round = h.norm_ht > 0 ? std::sqrt(s.bound_round) / h.norm_ht : 0.0;
  return s;
}

}  // namespace hh
