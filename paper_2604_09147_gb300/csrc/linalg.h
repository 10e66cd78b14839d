// Small dense linear algebra for the host builder: column-major matrices,
// Householder QR, column-pivoted QR with a Frobenius stopping rule,
// one-sided Jacobi SVD and adaptive cross approximation (ACA).
#pragma once

#include <cstdint>
#include <functional>
#include <vector>

namespace hh {
namespace la {

struct Mat {
  int64_t m = 0, n = 0;
  std::vector<double> a;  // column-major, ld = m
  Mat() = default;
  Mat(int64_t m_, int64_t n_) : m(m_), n(n_), a(static_cast<size_t>(m_ * n_), 0.0) {}
  double& operator()(int64_t i, int64_t j) { return a[static_cast<size_t>(i + j * m)]; }
  double operator()(int64_t i, int64_t j) const { return a[static_cast<size_t>(i + j * m)]; }
  double* col(int64_t j) { return a.data() + j * m; }
  const double* col(int64_t j) const { return a.data() + j * m; }
};

// C[:, 0:r] = A * B[:, 0:r]  (A m x k, B k x >= r, C m x >= r, preallocated)
void gemm_nn(const Mat& A, const Mat& B, int64_t r, Mat& C);

// Thin Householder QR of A (m x k, m >= k): A = Q R, Q (m x k) orthonormal,
// R (k x k) upper triangular.
void qr_thin(const Mat& A, Mat& Q, Mat& R);

// One-sided (Hestenes) Jacobi SVD of A (m x n, m >= n): A = U diag(s) V^T,
// singular values in descending order, U (m x n), V (n x n).
void svd_jacobi(const Mat& A, Mat& U, std::vector<double>& s, Mat& V);

// Smallest r with sqrt(sum_{i>=r} s_i^2) <= eps * sqrt(sum_i s_i^2)
// (s sorted descending); 0 for an all-zero s.
int trunc_rank(const std::vector<double>& s, double eps);

// Column-pivoted Householder QR of A (m x n) stopped at the first rank r
// whose trailing block satisfies ||A P - Q_r R_r||_F <= tol ||A||_F.
// Returns Q (m x r) and R (r x n) with A ~= Q R in the original column order.
void cpqr_trunc(Mat A, double tol, Mat& Q, Mat& R);

// ACA with partial pivoting on an implicitly given m x n matrix.
// row(i, out[n]) and col(j, out[m]) write exact entries.  Start row 0; the
// next row is the unused row with the largest |u_k|; stops when
// |u_k| |v_k| <= tol ||S_k||_F on `patience` consecutive steps.
// Returns U (m x k) residual columns and V (n x k) pivot-scaled rows.
void aca(const std::function<void(int64_t, double*)>& row,
         const std::function<void(int64_t, double*)>& col, int64_t m, int64_t n, double tol,
         int patience, Mat& U, Mat& V);

}  // namespace la
}  // namespace hh
