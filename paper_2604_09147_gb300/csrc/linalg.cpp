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

// ------------------------------------------------------------ matrix product
// GotoBLAS-style blocking: B is packed in k-chunks of kKC rows into strips of
// kNR columns, A in kMC x kKC panels into strips of kMR rows (alpha folded
// in), and a 4 x 4 register tile accumulates kKC products per pass.
constexpr int64_t kMR = 4, kNR = 4, kKC = 256, kMC = 128;

void pack_a(const double* A, int64_t rs, int64_t cs, int64_t mc, int64_t kc, double alpha, double* Ap) {
  for (int64_t i0 = 0; i0 < mc; i0 += kMR) {
    const int64_t mr = std::min(kMR, mc - i0);
    for (int64_t q = 0; q < kc; ++q) {
      for (int64_t i = 0; i < mr; ++i) Ap[q * kMR + i] = alpha * A[(i0 + i) * rs + q * cs];
      for (int64_t i = mr; i < kMR; ++i) Ap[q * kMR + i] = 0.0;
    }
    Ap += kc * kMR;
  }
}

void pack_b(const double* B, int64_t rs, int64_t cs, int64_t kc, int64_t nc, double* Bp) {
  for (int64_t j0 = 0; j0 < nc; j0 += kNR) {
    const int64_t nr = std::min(kNR, nc - j0);
    for (int64_t q = 0; q < kc; ++q) {
      for (int64_t j = 0; j < nr; ++j) Bp[q * kNR + j] = B[q * rs + (j0 + j) * cs];
      for (int64_t j = nr; j < kNR; ++j) Bp[q * kNR + j] = 0.0;
    }
    Bp += kc * kNR;
  }
}

// C[0:mr, 0:nr] += Ap-strip * Bp-strip over kc products
void micro(int64_t kc, const double* Ap, const double* Bp, double* C, int64_t ldc, int64_t mr, int64_t nr) {
  v2d c00 = {0, 0}, c01 = {0, 0}, c10 = {0, 0}, c11 = {0, 0}, c20 = {0, 0}, c21 = {0, 0}, c30 = {0, 0},
      c31 = {0, 0};
  for (int64_t q = 0; q < kc; ++q) {
    v2d a0, a1;
    __builtin_memcpy(&a0, Ap + q * kMR, 16);
    __builtin_memcpy(&a1, Ap + q * kMR + 2, 16);
    const double* b = Bp + q * kNR;
    const v2d b0 = {b[0], b[0]}, b1 = {b[1], b[1]}, b2 = {b[2], b[2]}, b3 = {b[3], b[3]};
    c00 += a0 * b0;
    c01 += a1 * b0;
    c10 += a0 * b1;
    c11 += a1 * b1;
    c20 += a0 * b2;
    c21 += a1 * b2;
    c30 += a0 * b3;
    c31 += a1 * b3;
  }
  double t[16];
  __builtin_memcpy(t + 0, &c00, 16);
  __builtin_memcpy(t + 2, &c01, 16);
  __builtin_memcpy(t + 4, &c10, 16);
  __builtin_memcpy(t + 6, &c11, 16);
  __builtin_memcpy(t + 8, &c20, 16);
  __builtin_memcpy(t + 10, &c21, 16);
  __builtin_memcpy(t + 12, &c30, 16);
  __builtin_memcpy(t + 14, &c31, 16);
  for (int64_t j = 0; j < nr; ++j)
    for (int64_t i = 0; i < mr; ++i) C[i + j * ldc] += t[i + 4 * j];
}

// ------------------------------------------------------------ blocked QR
constexpr int64_t kNB = 32;

// Compact WY form of the jb reflectors starting at column j0 of a factored
// matrix: H_{j0} ... H_{j0+jb-1} = I - Y T Y^T on rows j0..m-1, with Y
// (mm x jb, unit lower trapezoidal, explicit) and T (jb x jb, upper).
void build_wy(const Mat& F, const std::vector<double>& tau, int64_t j0, int64_t jb, std::vector<double>& Y,
              std::vector<double>& T) {
  const int64_t m = F.m, mm = m - j0;
  Y.assign(static_cast<size_t>(mm * jb), 0.0);
  for (int64_t c = 0; c < jb; ++c) {
    double* y = Y.data() + c * mm;
    y[c] = 1.0;
    const double* f = F.col(j0 + c) + j0;
    for (int64_t r = c + 1; r < mm; ++r) y[r] = f[r];
  }
  T.assign(static_cast<size_t>(jb * jb), 0.0);
  std::vector<double> w(static_cast<size_t>(jb));
  for (int64_t i = 0; i < jb; ++i) {
    const double ti = tau[j0 + i];
    T[i + i * jb] = ti;
    if (i == 0 || ti == 0.0) continue;
    const double* yi = Y.data() + i * mm;
    for (int64_t p = 0; p < i; ++p) w[p] = dot(Y.data() + p * mm + i, yi + i, mm - i);
    for (int64_t p = 0; p < i; ++p) {
      double s = 0.0;
      for (int64_t q = p; q < i; ++q) s += T[p + q * jb] * w[q];
      T[p + i * jb] = -ti * s;
    }
  }
}

}  // namespace

void gemm(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t a_rs, int64_t a_cs,
          const double* B, int64_t b_rs, int64_t b_cs, double* C, int64_t ldc) {
  if (m <= 0 || n <= 0 || k <= 0) return;
  const int64_t nstrips = (n + kNR - 1) / kNR;
  std::vector<double> Bp(static_cast<size_t>(std::min(k, kKC) * nstrips * kNR));
  std::vector<double> Ap(static_cast<size_t>(std::min(k, kKC) * ((std::min(m, kMC) + kMR - 1) / kMR) * kMR));
  for (int64_t pc = 0; pc < k; pc += kKC) {
    const int64_t kc = std::min(kKC, k - pc);
    pack_b(B + pc * b_rs, b_rs, b_cs, kc, n, Bp.data());
    for (int64_t ic = 0; ic < m; ic += kMC) {
      const int64_t mc = std::min(kMC, m - ic);
      pack_a(A + ic * a_rs + pc * a_cs, a_rs, a_cs, mc, kc, alpha, Ap.data());
      for (int64_t js = 0; js < nstrips; ++js) {
        const int64_t nr = std::min(kNR, n - js * kNR);
        for (int64_t i0 = 0; i0 < mc; i0 += kMR)
          micro(kc, Ap.data() + (i0 / kMR) * kc * kMR, Bp.data() + js * kc * kNR, C + ic + i0 + js * kNR * ldc, ldc,
                std::min(kMR, mc - i0), nr);
      }
    }
  }
}

void qr_factor(Mat& A, std::vector<double>& tau) {
  const int64_t m = A.m, k = A.n, kk = std::min(m, k);
  tau.assign(static_cast<size_t>(kk), 0.0);
  std::vector<double> Y, T, W;
  for (int64_t j0 = 0; j0 < kk; j0 += kNB) {
    const int64_t jb = std::min(kNB, kk - j0);
    // the panel, one reflector at a time
    for (int64_t j = j0; j < j0 + jb; ++j) {
      tau[j] = householder(A.col(j) + j, m - j);
      for (int64_t c = j + 1; c < j0 + jb; ++c) apply_reflector(A.col(j) + j, tau[j], A.col(c) + j, m - j);
    }
    const int64_t nc = k - (j0 + jb);
    if (nc <= 0) continue;
    // trailing columns: C <- (I - Y T Y^T)^T C = C - Y (T^T (Y^T C))
    const int64_t mm = m - j0;
    build_wy(A, tau, j0, jb, Y, T);
    double* C = A.col(j0 + jb) + j0;
    W.assign(static_cast<size_t>(jb * nc), 0.0);
    gemm(jb, nc, mm, 1.0, Y.data(), mm, 1, C, 1, m, W.data(), jb);
    for (int64_t c = 0; c < nc; ++c) {
      double* w = W.data() + c * jb;
      for (int64_t i = jb - 1; i >= 0; --i) {  // w <- T^T w (rows below i still old)
        double s = 0.0;
        for (int64_t p = 0; p <= i; ++p) s += T[p + i * jb] * w[p];
        w[i] = s;
      }
    }
    gemm(mm, nc, jb, -1.0, Y.data(), 1, mm, W.data(), 1, jb, C, m);
  }
}

Mat qr_r(const Mat& F) {
  const int64_t k = F.n;
  Mat R(k, k);
  for (int64_t c = 0; c < k; ++c)
    for (int64_t r = 0; r <= c && r < F.m; ++r) R(r, c) = F(r, c);
  return R;
}

void qr_apply_q(const Mat& F, const std::vector<double>& tau, const Mat& X, Mat& out) {
  const int64_t m = F.m, kk = static_cast<int64_t>(tau.size()), r = X.n;
  out = Mat(m, r);
  for (int64_t c = 0; c < r; ++c)
    for (int64_t i = 0; i < X.m && i < m; ++i) out(i, c) = X(i, c);
  if (kk == 0 || r == 0) return;
  std::vector<double> Y, T, W;
  // Q = (block 0)(block 1)...: apply the last block first
  for (int64_t j0 = (kk - 1) / kNB * kNB; j0 >= 0; j0 -= kNB) {
    const int64_t jb = std::min(kNB, kk - j0), mm = m - j0;
    build_wy(F, tau, j0, jb, Y, T);
    double* C = out.a.data() + j0;
    W.assign(static_cast<size_t>(jb * r), 0.0);
    gemm(jb, r, mm, 1.0, Y.data(), mm, 1, C, 1, m, W.data(), jb);
    for (int64_t c = 0; c < r; ++c) {
      double* w = W.data() + c * jb;
      for (int64_t i = 0; i < jb; ++i) {  // w <- T w (rows above i already new are not read)
        double s = 0.0;
        for (int64_t p = i; p < jb; ++p) s += T[i + p * jb] * w[p];
        w[i] = s;
      }
    }
    gemm(mm, r, jb, -1.0, Y.data(), 1, mm, W.data(), 1, jb, C, m);
  }
}

void svd_left(const Mat& A, Mat& W, std::vector<double>& s) {
  const int64_t m = A.m, n = A.n;
  W = A;
  const double tol = 1e-15;
  std::vector<double> nrm(static_cast<size_t>(n));
  // each sweep visits every pair once, block pair by block pair, so that the
  // two column blocks of a block pair stay in cache (about 512 KB)
  const int64_t bs = std::max<int64_t>(8, std::min<int64_t>(128, 32768 / std::max<int64_t>(m, 1)));
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int64_t j = 0; j < n; ++j) nrm[j] = dot(W.col(j), W.col(j), m);
    for (int64_t b0 = 0; b0 < n; b0 += bs)
    for (int64_t c0 = b0; c0 < n; c0 += bs)
    for (int64_t p = b0; p < std::min(n, b0 + bs); ++p) {
      for (int64_t q = std::max(p + 1, c0); q < std::min(n, c0 + bs); ++q) {
        const double alpha = nrm[p], beta = nrm[q];
        if (alpha == 0.0 || beta == 0.0) continue;
        const double gamma = dot(W.col(p), W.col(q), m);
        if (std::fabs(gamma) <= tol * std::sqrt(alpha) * std::sqrt(beta)) continue;
        rotated = true;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::hypot(1.0, zeta));
        const double c = 1.0 / std::hypot(1.0, t);
        const double sn = c * t;
        double* up = W.col(p);
        double* uq = W.col(q);
        for (int64_t i = 0; i < m; ++i) {
          const double a = up[i], b = uq[i];
          up[i] = c * a - sn * b;
          uq[i] = sn * a + c * b;
        }
        // the rotation moves t*gamma of squared norm from column p to q;
        // recompute a norm that this update would mostly cancel
        const double np = alpha - t * gamma, nq = beta + t * gamma;
        nrm[p] = np > 0.25 * alpha ? np : dot(up, up, m);
        nrm[q] = nq > 0.25 * beta ? nq : dot(uq, uq, m);
      }
    }
    if (!rotated) break;
  }
  std::vector<double> sv(static_cast<size_t>(n));
  for (int64_t j = 0; j < n; ++j) sv[j] = std::sqrt(dot(W.col(j), W.col(j), m));
  std::vector<int64_t> order(static_cast<size_t>(n));
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return sv[a] > sv[b]; });
  Mat W2(m, n);
  s.assign(static_cast<size_t>(n), 0.0);
  for (int64_t c = 0; c < n; ++c) {
    const int64_t o = order[c];
    s[c] = sv[o];
    const double inv = sv[o] > 0 ? 1.0 / sv[o] : 0.0;
    for (int64_t i = 0; i < m; ++i) W2(i, c) = W(i, o) * inv;
  }
  W = std::move(W2);
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
  std::vector<double> gu(static_cast<size_t>(kmax)), gv(static_cast<size_t>(kmax));
  int64_t k = 0, i = 0, nused = 0;
  double norm2 = 0.0;
  int calm = 0;
  // The stopping test of step k - 1 needs u_l . u_{k-1} and v_l . v_{k-1}
  // (l < k - 1) for ||S_{k-1}||_F^2.  They are taken in step k's residual
  // updates, which stream every u_l and v_l anyway; if the test then stops,
  // step k is dropped, so the result is the one of testing right away.
  bool pending = false;
  double pu = 0.0, pv = 0.0;  // ||u_{k-1}||^2, ||v_{k-1}||^2
  // y -= coef[l] B_l for l < k and, with `last`, d[l] = B_l . last for l < k - 1
  auto update = [&](const double* B, int64_t len, const double* coef, int64_t ld_coef, const double* last,
                    double* y, double* d) {
    for (int64_t l = 0; l < k; ++l) {
      const double* b = B + l * len;
      const double a = -coef[l * ld_coef];
      const v2d av = {a, a};
      const bool want = last && l + 1 < k;
      v2d s0 = {0, 0}, s1 = {0, 0};
      int64_t e = 0;
      for (; e + 4 <= len; e += 4) {
        v2d b0, b1, y0, y1;
        __builtin_memcpy(&b0, b + e, 16);
        __builtin_memcpy(&b1, b + e + 2, 16);
        __builtin_memcpy(&y0, y + e, 16);
        __builtin_memcpy(&y1, y + e + 2, 16);
        if (want) {
          v2d o0, o1;
          __builtin_memcpy(&o0, last + e, 16);
          __builtin_memcpy(&o1, last + e + 2, 16);
          s0 += b0 * o0;
          s1 += b1 * o1;
        }
        y0 += av * b0;
        y1 += av * b1;
        __builtin_memcpy(y + e, &y0, 16);
        __builtin_memcpy(y + e + 2, &y1, 16);
      }
      const v2d t = s0 + s1;
      double sd = t[0] + t[1];
      for (; e < len; ++e) {
        if (want) sd += b[e] * last[e];
        y[e] += a * b[e];
      }
      if (want) d[l] = sd;
    }
  };
  // finish the stopping test of step k - 1; true = stop
  auto settle = [&]() {
    pending = false;
    double cross = 0.0;
    for (int64_t l = 0; l + 1 < k; ++l) cross += gu[l] * gv[l];
    norm2 = norm2 + 2.0 * cross + pu * pv;
    if (std::sqrt(pu) * std::sqrt(pv) <= tol * std::sqrt(std::max(norm2, 0.0))) return ++calm >= patience;
    calm = 0;
    return false;
  };
  while (k < kmax) {
    row(i, rbuf.data());
    update(Vb.data(), n, Ub.data() + i, m, pending ? Vb.data() + (k - 1) * n : nullptr, rbuf.data(), gv.data());
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
      if (pending) {
        for (int64_t l = 0; l + 1 < k; ++l) gu[l] = dot(Ub.data() + l * m, Ub.data() + (k - 1) * m, m);
        if (settle()) break;
      }
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
    update(Ub.data(), m, Vb.data() + j, n, pending ? Ub.data() + (k - 1) * m : nullptr, cbuf.data(), gu.data());
    if (pending && settle()) break;
    if (k == cap) {
      cap = std::min(kmax, 2 * cap);
      Ub.resize(static_cast<size_t>(m * cap));
      Vb.resize(static_cast<size_t>(n * cap));
    }
    std::copy(cbuf.begin(), cbuf.end(), Ub.begin() + k * m);
    std::copy(rbuf.begin(), rbuf.end(), Vb.begin() + k * n);
    pu = dot(cbuf.data(), cbuf.data(), m);
    pv = dot(rbuf.data(), rbuf.data(), n);
    pending = true;
    ++k;
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
