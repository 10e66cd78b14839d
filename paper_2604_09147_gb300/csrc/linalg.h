// Small dense linear algebra for the host builder: column-major matrices,
// a register-blocked matrix product, blocked Householder QR, column-pivoted
// QR with a Frobenius stopping rule, one-sided Jacobi SVD and adaptive cross
// approximation (ACA).  Every routine fixes its order of operations and is
// compiled without floating-point contraction, so results are the same on
// every host.
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

// C (m x n, leading dimension ldc) += alpha * A * B with A(i, q) =
// A[i * a_rs + q * a_cs] (m x k) and B(q, j) = B[q * b_rs + j * b_cs] (k x n):
// the strides select plain or transposed operands.
void gemm(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t a_rs, int64_t a_cs,
          const double* B, int64_t b_rs, int64_t b_cs, double* C, int64_t ldc);

// Householder QR of A (m x k, m >= k) in place: R in the upper triangle, the
// reflectors' tails below it (H_j = I - tau_j v_j v_j^T, v_j[j] = 1), so that
// A_in = H_0 H_1 ... H_{k-1} [R; 0].
void qr_factor(Mat& A, std::vector<double>& tau);

// The k x k upper triangular R of a factored matrix.
Mat qr_r(const Mat& F);

// out (m x r) = Q [X; 0] for X (k x r) with Q = H_0 ... H_{k-1} of a
// factored m x k matrix: the thin Q times X without forming Q.
void qr_apply_q(const Mat& F, const std::vector<double>& tau, const Mat& X, Mat& out);

// One-sided (Hestenes) Jacobi SVD of A (m x n, m >= n), left side only:
// A = W diag(s) Z^T with s descending and W (m x n) orthonormal (columns of
// zero singular values are zero); Z is not formed (Z S = A^T W).
void svd_left(const Mat& A, Mat& W, std::vector<double>& s);

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
