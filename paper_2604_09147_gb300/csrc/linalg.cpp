// Dense linear algebra for the host builder (see linalg.h).
#include "linalg.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace hh {
namespace la {

namespace {

// two-wide vectors (SSE2 / NEON) with four independent partial sums
typedef double v2d __attribute__((vector_size(16)));

inline double dot(const double* a, const double* b, int64_t n) {
  v2d s0 = {0, 0}, s1 = {0, 0}, s2 = {0, 0}, s3 = {0, 0};
  int64_t i = 0;
  for (; i + 8 <= n; i += 8) {
    v2d a0, a1, a2, a3, b0, b1, b2, b3;
    __builtin_memcpy(&a0, a + i, 16);
    __builtin_memcpy(&a1, a + i + 2, 16);
    __builtin_memcpy(&a2, a + i + 4, 16);
    __builtin_memcpy(&a3, a + i + 6, 16);
    __builtin_memcpy(&b0, b + i, 16);
    __builtin_memcpy(&b1, b + i + 2, 16);
    __builtin_memcpy(&b2, b + i + 4, 16);
    __builtin_memcpy(&b3, b + i + 6, 16);
    s0 += a0 * b0;
    s1 += a1 * b1;
    s2 += a2 * b2;
    s3 += a3 * b3;
  }
  v2d t = (s0 + s1) + (s2 + s3);
  double s = t[0] + t[1];
  for (; i < n; ++i) s += a[i] * b[i];
  return s;
}

inline void axpy(double alpha, const double* x, double* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] += alpha * x[i];
}

// Householder reflector for x[0..len): on return x[0] = beta (the new
// leading entry), x[1..] = v[1..] (v[0] = 1); returns tau.
double householder(double* x, int64_t len) {
  if (len <= 0) return 0.0;
  double tail = len > 1 ? dot(x + 1, x + 1, len - 1) : 0.0;
  if (tail == 0.0) return 0.0;  // already reduced
  double nrm = std::sqrt(x[0] * x[0] + tail);
  double beta = x[0] >= 0 ? -nrm : nrm;
  double tau = (beta - x[0]) / beta;
  double scale = 1.0 / (x[0] - beta);
  for (int64_t i = 1; i < len; ++i) x[i] *= scale;
  x[0] = beta;
  return tau;
}

// apply H = I - tau v v^T (v[0] = 1 implicit, v[1..] = vt[1..]) to y[0..len)
inline void apply_reflector(const double* vt, double tau, double* y, int64_t len) {
  if (tau == 0.0) return;
  double w = y[0] + dot(vt + 1, y + 1, len - 1);
  w *= tau;
  y[0] -= w;
  axpy(-w, vt + 1, y + 1, len - 1);
}

}  // namespace

void gemm_nn(const Mat& A, const Mat& B, int64_t r, Mat& C) {
  const int64_t m = A.m, k = A.n;
  for (int64_t c = 0; c < r; ++c) {
    double* dst = C.col(c);
    for (int64_t q = 0; q < k; ++q) {
      const double b = B(q, c);
      if (b != 0.0) axpy(b, A.col(q), dst, m);
    }
  }
}

void qr_thin(const Mat& A, Mat& Q, Mat& R) {
  const int64_t m = A.m, k = A.n;
  Mat W = A;
  std::vector<double> tau(static_cast<size_t>(k), 0.0);
  for (int64_t j = 0; j < k && j < m; ++j) {
    tau[j] = householder(W.col(j) + j, m - j);
    for (int64_t c = j + 1; c < k; ++c) apply_reflector(W.col(j) + j, tau[j], W.col(c) + j, m - j);
  }
  R = Mat(k, k);
  for (int64_t c = 0; c < k; ++c)
    for (int64_t r = 0; r <= c && r < m; ++r) R(r, c) = W(r, c);
  Q = Mat(m, k);
  for (int64_t c = 0; c < k && c < m; ++c) Q(c, c) = 1.0;
  for (int64_t j = std::min(k, m) - 1; j >= 0; --j)
    for (int64_t c = j; c < k; ++c) apply_reflector(W.col(j) + j, tau[j], Q.col(c) + j, m - j);
}

void svd_jacobi(const Mat& A, Mat& U, std::vector<double>& s, Mat& V) {
  const int64_t m = A.m, n = A.n;
  U = A;
  V = Mat(n, n);
  for (int64_t i = 0; i < n; ++i) V(i, i) = 1.0;
  const double tol = 1e-15;
  std::vector<double> nrm(static_cast<size_t>(n));
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int64_t j = 0; j < n; ++j) nrm[j] = dot(U.col(j), U.col(j), m);
    for (int64_t p = 0; p + 1 < n; ++p) {
      for (int64_t q = p + 1; q < n; ++q) {
        double alpha = nrm[p], beta = nrm[q];
        if (alpha == 0.0 || beta == 0.0) continue;
        double gamma = dot(U.col(p), U.col(q), m);
        if (std::fabs(gamma) <= tol * std::sqrt(alpha) * std::sqrt(beta)) continue;
        rotated = true;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::hypot(1.0, zeta));
        double c = 1.0 / std::hypot(1.0, t);
        double sn = c * t;
        double* up = U.col(p);
        double* uq = U.col(q);
        for (int64_t i = 0; i < m; ++i) {
          double a = up[i], b = uq[i];
          up[i] = c * a - sn * b;
          uq[i] = sn * a + c * b;
        }
        double* vp = V.col(p);
        double* vq = V.col(q);
        for (int64_t i = 0; i < n; ++i) {
          double a = vp[i], b = vq[i];
          vp[i] = c * a - sn * b;
          vq[i] = sn * a + c * b;
        }
        nrm[p] = dot(up, up, m);
        nrm[q] = dot(uq, uq, m);
      }
    }
    if (!rotated) break;
  }
  std::vector<double> sv(static_cast<size_t>(n));
  for (int64_t j = 0; j < n; ++j) sv[j] = std::sqrt(dot(U.col(j), U.col(j), m));
  std::vector<int64_t> order(static_cast<size_t>(n));
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return sv[a] > sv[b]; });
  Mat U2(m, n), V2(n, n);
  s.assign(static_cast<size_t>(n), 0.0);
  for (int64_t c = 0; c < n; ++c) {
    int64_t o = order[c];
    s[c] = sv[o];
    double inv = sv[o] > 0 ? 1.0 / sv[o] : 0.0;
    for (int64_t i = 0; i < m; ++i) U2(i, c) = U(i, o) * inv;
    for (int64_t i = 0; i < n; ++i) V2(i, c) = V(i, o);
  }
  U = std::move(U2);
  V = std::move(V2);
}

int trunc_rank(const std::vector<double>& s, double eps) {
  const int n = static_cast<int>(s.size());
  std::vector<double> tail(static_cast<size_t>(n) + 1, 0.0);
  for (int i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + s[i] * s[i];
  if (tail[0] == 0.0) return 0;
  const double lim = eps * std::sqrt(tail[0]);
  for (int r = 0; r <= n; ++r)
    if (std::sqrt(tail[r]) <= lim) return r;
  return n;
}

void cpqr_trunc(Mat A, double tol, Mat& Q, Mat& R) {
  const int64_t m = A.m, n = A.n, kmax = std::min(m, n);
  std::vector<int64_t> piv(static_cast<size_t>(n));
  std::iota(piv.begin(), piv.end(), 0);
  std::vector<double> pn(static_cast<size_t>(n)), tau;
  double total = 0.0;
  for (int64_t c = 0; c < n; ++c) {
    pn[c] = dot(A.col(c), A.col(c), m);
    total += pn[c];
  }
  const double lim = tol * std::sqrt(total);
  int64_t r = 0;
  for (; r < kmax; ++r) {
    double trail = 0.0;
    for (int64_t c = r; c < n; ++c) trail += pn[c];
    if (std::sqrt(trail) <= lim) break;
    int64_t best = r;
    for (int64_t c = r + 1; c < n; ++c)
      if (pn[c] > pn[best]) best = c;
    if (best != r) {
      std::swap_ranges(A.col(r), A.col(r) + m, A.col(best));
      std::swap(pn[r], pn[best]);
      std::swap(piv[r], piv[best]);
    }
    tau.push_back(householder(A.col(r) + r, m - r));
    for (int64_t c = r + 1; c < n; ++c) {
      apply_reflector(A.col(r) + r, tau[r], A.col(c) + r, m - r);
      pn[c] = (m - r - 1 > 0) ? dot(A.col(c) + r + 1, A.col(c) + r + 1, m - r - 1) : 0.0;
    }
  }
  R = Mat(r, n);
  for (int64_t c = 0; c < n; ++c)
    for (int64_t i = 0; i < r && i <= c; ++i) R(i, piv[c]) = A(i, c);
  Q = Mat(m, r);
  for (int64_t c = 0; c < r; ++c) Q(c, c) = 1.0;
  for (int64_t j = r - 1; j >= 0; --j)
    for (int64_t c = j; c < r; ++c) apply_reflector(A.col(j) + j, tau[j], Q.col(c) + j, m - j);
}

void aca(const std::function<void(int64_t, double*)>& row,
         const std::function<void(int64_t, double*)>& col, int64_t m, int64_t n, double tol,
         int patience, Mat& U, Mat& V) {
  const int64_t kmax = std::min(m, n);
  int64_t cap = std::min<int64_t>(kmax, 64);
  std::vector<double> Ub(static_cast<size_t>(m * cap)), Vb(static_cast<size_t>(n * cap));
  std::vector<char> used(static_cast<size_t>(m), 0);
  std::vector<double> rbuf(static_cast<size_t>(n)), cbuf(static_cast<size_t>(m));
  int64_t k = 0, i = 0, nused = 0;
  double norm2 = 0.0;
  int calm = 0;
  while (k < kmax) {
    row(i, rbuf.data());
    for (int64_t l = 0; l < k; ++l) axpy(-Ub[i + l * m], Vb.data() + l * n, rbuf.data(), n);
    if (!used[i]) {
      used[i] = 1;
      ++nused;
    }
    int64_t j = 0;
    double best = -1.0;
    for (int64_t c = 0; c < n; ++c) {
      double a = std::fabs(rbuf[c]);
      if (a > best) {
        best = a;
        j = c;
      }
    }
    const double pivot = rbuf[j];
    if (pivot == 0.0) {
      int64_t f = -1;
      for (int64_t r = 0; r < m; ++r)
        if (!used[r]) {
          f = r;
          break;
        }
      if (f < 0) break;
      i = f;
      continue;
    }
    const double inv = 1.0 / pivot;
    for (int64_t c = 0; c < n; ++c) rbuf[c] *= inv;
    col(j, cbuf.data());
    for (int64_t l = 0; l < k; ++l) axpy(-Vb[j + l * n], Ub.data() + l * m, cbuf.data(), m);
    double cross = 0.0;
    for (int64_t l = 0; l < k; ++l)
      cross += dot(Ub.data() + l * m, cbuf.data(), m) * dot(Vb.data() + l * n, rbuf.data(), n);
    const double uu = dot(cbuf.data(), cbuf.data(), m), vv = dot(rbuf.data(), rbuf.data(), n);
    norm2 = norm2 + 2.0 * cross + uu * vv;
    if (k == cap) {
      int64_t ncap = std::min(kmax, 2 * cap);
      Ub.resize(static_cast<size_t>(m * ncap));
      Vb.resize(static_cast<size_t>(n * ncap));
      cap = ncap;
    }
    std::copy(cbuf.begin(), cbuf.end(), Ub.begin() + k * m);
    std::copy(rbuf.begin(), rbuf.end(), Vb.begin() + k * n);
    ++k;
    if (std::sqrt(uu) * std::sqrt(vv) <= tol * std::sqrt(std::max(norm2, 0.0))) {
      if (++calm >= patience) break;
    } else {
      calm = 0;
    }
    if (nused == m) break;
    double bu = -1.0;
    int64_t ni = 0;
    for (int64_t r = 0; r < m; ++r) {
      double a = used[r] ? -1.0 : std::fabs(cbuf[r]);
      if (a > bu) {
        bu = a;
        ni = r;
      }
    }
    i = ni;
  }
  U = Mat(m, k);
  V = Mat(n, k);
  std::copy(Ub.begin(), Ub.begin() + m * k, U.a.begin());
  std::copy(Vb.begin(), Vb.begin() + n * k, V.a.begin());
}

}  // namespace la
}  // namespace hh
