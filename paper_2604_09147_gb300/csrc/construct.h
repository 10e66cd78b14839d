// Construction on the device: LRcompression (Eq. 2.1) of many admissible
// blocks at once, for the host builder (builder.cpp).  Plain C++ interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "linalg.h"

namespace hh {

// one block to compress: rows [r0, r0 + m) and columns [c0, c0 + n) of the
// kernel matrix in tree order
struct DeviceJob {
  int64_t r0, m, c0, n;
};

struct DeviceStats {
  double seconds = 0;        // wall time of the device compression
  int64_t fallback = 0;      // blocks left to the host (rank cap, failed factorization)
  int64_t waves = 0;         // batches that fit the device memory budget
};

// Compresses every job to eps on `device` (ACA to eps / 100, CholeskyQR2 of
// both cross factors, one-sided Jacobi SVD of the k x k core, truncation of
// the Frobenius tail at 0.99 eps): U (m x r, orthonormal), V (n x r, carries
// the singular values), s (r).  ok[j] = 0 marks a job the caller must
// compress itself.  tp: the points in tree order (n_pts x dim, host).
// Throws std::runtime_error on a CUDA error.
void compress_on_device(int device, const double* tp, int64_t n_pts, int dim, int kernel, double kparam,
                        double eps, const std::vector<DeviceJob>& jobs, std::vector<la::Mat>& U,
                        std::vector<la::Mat>& V, std::vector<std::vector<double>>& s, std::vector<char>& ok,
                        DeviceStats* stats);

}  // namespace hh
