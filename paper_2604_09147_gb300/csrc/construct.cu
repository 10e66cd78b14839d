// LRcompression (Eq. 2.1) of the admissible blocks on the device.
//
// The same algorithm as the host builder's large-block path, batched over
// blocks, in fp64:
//   1. aca_kernel: adaptive cross approximation with partial pivoting
//      (Section 2.2's compression, reading R4), one CTA per block, entries of
//      the kernel matrix (Eq. 5.1) generated from the tree-ordered points;
//      stops when |u_k| |v_k| <= (eps / 100) ||S_k||_F on three consecutive
//      steps, ||S_k||_F^2 kept up to date with the cross terms u_l.u_k and
//      v_l.v_k.  A block whose rank would pass its column capacity is left
//      to the host.
//   2. CholeskyQR2 of both cross factors (Gram matrix, Cholesky of its
//      column-scaled form, Q = U R^-1, twice): U = Q_u R_u, V = Q_v R_v.
//   3. T = R_u R_v^T and its one-sided (Hestenes) Jacobi SVD T J = W Sigma.
//   4. Truncation to the smallest r whose Frobenius tail is <= 0.99 eps of
//      the whole; U_b = Q_u W_r (orthonormal), V_b = Q_v J_r Sigma_r.
// Every loop is bounded (rank capacity, sweep limit); nothing waits on a
// flag.  Blocks are processed in waves that fit a device-memory budget.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <string>

#include <cuda_runtime.h>

#include "construct.h"

namespace hh {

namespace {

constexpr int kAcaThreads = 512;
constexpr double kAcaShare = 0.01;  // ACA to eps / 100, truncation at 0.99 eps
constexpr int kAcaPatience = 3;
constexpr int kMaxRankCap = 2048;   // columns of a block's cross factors on the device
constexpr int kJacobiSweeps = 40;

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw std::runtime_error(std::string("device compression: ") + what + ": " +
                                                 cudaGetErrorString(e));
}

// Eq. 5.1: f(r), f(0) = 0 for the singular kernels
__device__ __forceinline__ double kernel_value(int kernel, double p, double r) {
  switch (kernel) {
    case 0: return exp(-r / p);
    case 1: return r == 0.0 ? 0.0 : 1.0 / r;
    case 2: return exp(-(r * r) / p);
    case 3: return r == 0.0 ? 0.0 : log(r);
    default: return r == 0.0 ? 0.0 : 1.0 / (r * r);
  }
}

struct Geo {
  const double* pts;  // tree order, n x dim
  int dim, kernel;
  double p;
};

__device__ __forceinline__ double entry(const Geo& g, int64_t a, int64_t b) {
  const double* x = g.pts + a * g.dim;
  const double* y = g.pts + b * g.dim;
  double s = 0.0;
  for (int d = 0; d < g.dim; ++d) {
    const double t = x[d] - y[d];
    s = s + t * t;
  }
  return kernel_value(g.kernel, g.p, sqrt(s));
}

// device descriptor of one block in the ACA stage
struct AcaJob {
  int64_t r0, m, c0, n;
  double* U;   // m x cap, column-major
  double* V;   // n x cap
  int* used;   // m flags
  int cap;     // column capacity
  int k;       // out: rank
  int status;  // out: 0 ok, 1 capacity reached before the stopping test
  int pad;
};

// CTA-wide sum (every thread gets it); red: kAcaThreads / 32 doubles
__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// CTA-wide argmax of a (first index among equal values; a < 0 never wins over
// a >= 0); every thread gets (value, index)
__device__ void cta_argmax(double a, int64_t idx, double* redv, int64_t* redi, double& best, int64_t& at) {
  for (int o = 16; o > 0; o >>= 1) {
    const double b = __shfl_xor_sync(0xffffffffu, a, o);
    const int64_t j = __shfl_xor_sync(0xffffffffu, idx, o);
    if (b > a || (b == a && j < idx)) {
      a = b;
      idx = j;
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    redv[w] = a;
    redi[w] = idx;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? redv[threadIdx.x] : -2.0;
    int64_t j = threadIdx.x < (blockDim.x >> 5) ? redi[threadIdx.x] : INT64_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      const double b = __shfl_xor_sync(0xffffffffu, v, o);
      const int64_t q = __shfl_xor_sync(0xffffffffu, j, o);
      if (b > v || (b == v && q < j)) {
        v = b;
        j = q;
      }
    }
    if (threadIdx.x == 0) {
      redv[0] = v;
      redi[0] = j;
    }
  }
  __syncthreads();
  best = redv[0];
  at = redi[0];
  __syncthreads();
}

// ------------------------------------------------------------------ 1. ACA
// One CTA per block.  Shared memory: coef (the pivot row of U or column of V
// for the residual update), gu / gv (u_l . u_{k-1} and v_l . v_{k-1} for the
// stopping test of step k - 1, taken at the top of step k: the test depends
// only on columns < k, so a stop drops step k exactly as testing at once).
__global__ void __launch_bounds__(kAcaThreads) aca_kernel(AcaJob* jobs, Geo g, double tol, int patience) {
  AcaJob& J = jobs[blockIdx.x];
  const int64_t m = J.m, n = J.n, r0 = J.r0, c0 = J.c0;
  double* U = J.U;
  double* V = J.V;
  int* used = J.used;
  const int64_t kmax = m < n ? m : n;
  const int cap = J.cap;
  extern __shared__ double sm[];
  double* coef = sm;
  double* gu = sm + cap;
  double* gv = sm + 2 * cap;
  __shared__ double redv[32];
  __shared__ int64_t redi[32];
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  for (int64_t r = tid; r < m; r += nt) used[r] = 0;
  __syncthreads();
  int64_t k = 0, i = 0, nused = 0;
  double norm2 = 0.0, pu = 0.0, pv = 0.0;
  int calm = 0, status = 0;
  bool pending = false;
  // d[l] = B[:, l] . B[:, k-1] for l < k - 1 (warps over l)
  auto dots = [&](const double* B, int64_t len, double* d) {
    const double* last = B + (k - 1) * len;
    for (int64_t l = warp; l + 1 < k; l += nw) {
      const double* b = B + l * len;
      double s = 0.0;
      for (int64_t e = lane; e < len; e += 32) s += b[e] * last[e];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) d[l] = s;
    }
    __syncthreads();
  };
  while (k < kmax) {
    if (pending) {  // stopping test of step k - 1
      dots(V, n, gv);
      dots(U, m, gu);
      double part = 0.0;
      for (int64_t l = tid; l + 1 < k; l += nt) part += gu[l] * gv[l];
      const double cross = cta_sum(part, redv);
      pending = false;
      norm2 = norm2 + 2.0 * cross + pu * pv;
      if (sqrt(pu) * sqrt(pv) <= tol * sqrt(fmax(norm2, 0.0))) {
        if (++calm >= patience) break;
      } else {
        calm = 0;
      }
    }
    if (k == cap) {  // the rank would pass the capacity: leave the block to the host
      status = 1;
      break;
    }
    // row i of the residual -> V[:, k]
    for (int64_t l = tid; l < k; l += nt) coef[l] = U[i + l * m];
    __syncthreads();
    double* vk = V + k * n;
    for (int64_t c = tid; c < n; c += nt) {
      double val = entry(g, r0 + i, c0 + c);
      for (int64_t l = 0; l < k; ++l) val -= coef[l] * V[c + l * n];
      vk[c] = val;
    }
    const int was = used[i];
    __syncthreads();
    if (tid == 0) used[i] = 1;
    if (!was) ++nused;
    double a = -1.0, best;
    int64_t at = 0, j;
    for (int64_t c = tid; c < n; c += nt) {
      const double v = fabs(vk[c]);
      if (v > a) {
        a = v;
        at = c;
      }
    }
    cta_argmax(a, at, redv, redi, best, j);
    const double pivot = vk[j];
    if (pivot == 0.0) {  // zero residual row: continue with the first unused row
      a = -1.0;
      at = 0;
      for (int64_t r = tid; r < m; r += nt)
        if (!used[r] && a < 1.0) {
          a = 1.0;
          at = r;
        }
      cta_argmax(a, at, redv, redi, best, j);
      if (best < 0.0) break;
      i = j;
      continue;
    }
    const double inv = 1.0 / pivot;
    for (int64_t c = tid; c < n; c += nt) vk[c] *= inv;
    // column j of the residual -> U[:, k]
    for (int64_t l = tid; l < k; l += nt) coef[l] = V[j + l * n];
    __syncthreads();
    double* uk = U + k * m;
    for (int64_t r = tid; r < m; r += nt) {
      double val = entry(g, r0 + r, c0 + j);
      for (int64_t l = 0; l < k; ++l) val -= coef[l] * U[r + l * m];
      uk[r] = val;
    }
    __syncthreads();
    double su = 0.0, sv = 0.0;
    for (int64_t r = tid; r < m; r += nt) su += uk[r] * uk[r];
    for (int64_t c = tid; c < n; c += nt) sv += vk[c] * vk[c];
    pu = cta_sum(su, redv);
    pv = cta_sum(sv, redv);
    pending = true;
    ++k;
    if (nused == m) break;
    // next row: the unused row with the largest |u_k|
    a = -1.0;
    at = 0;
    for (int64_t r = tid; r < m; r += nt) {
      const double v = used[r] ? -1.0 : fabs(uk[r]);
      if (v > a) {
        a = v;
        at = r;
      }
    }
    cta_argmax(a, at, redv, redi, best, j);
    i = j;
  }
  if (tid == 0) {
    J.k = static_cast<int>(k);
    J.status = status;
  }
}

// ------------------------------------------------------- batched fp64 GEMM
// C (M x N, ldc) = alpha op(A) op(B) (+ C with acc) for many jobs of their
// own sizes: A(i, q) = A[i a_rs + q a_cs], B(q, j) = B[q b_rs + j b_cs].  A
// CTA computes a 64 x 64 tile (256 threads, 4 x 4 each) over K in steps of
// 16 staged in shared memory.  Tiles of all jobs form one grid: tile t
// belongs to the job whose tile prefix covers t (binary search).
struct GemmJob {
  const double* A;
  const double* B;
  double* C;
  int64_t a_rs, a_cs, b_rs, b_cs, ldc;
  int M, N, K, acc;
  double alpha;
};
constexpr int kGT = 64, kGK = 16;

__global__ void __launch_bounds__(256) gemm_kernel(const GemmJob* jobs, const int64_t* tile_start, int njobs) {
  __shared__ double As[kGK][kGT + 1];
  __shared__ double Bs[kGK][kGT + 1];
  const int64_t t = blockIdx.x;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (tile_start[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  const GemmJob jb = jobs[lo];
  const int64_t local = t - tile_start[lo];
  const int tm = (jb.M + kGT - 1) / kGT;
  const int i0 = static_cast<int>(local % tm) * kGT, j0 = static_cast<int>(local / tm) * kGT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int q0 = 0; q0 < jb.K; q0 += kGK) {
    for (int e = threadIdx.x; e < kGK * kGT; e += 256) {
      const int q = e / kGT, r = e % kGT;
      const int gi = i0 + r, gq = q0 + q, gj = j0 + r;
      As[q][r] = (gi < jb.M && gq < jb.K) ? jb.A[gi * jb.a_rs + gq * jb.a_cs] : 0.0;
      Bs[q][r] = (gj < jb.N && gq < jb.K) ? jb.B[gq * jb.b_rs + gj * jb.b_cs] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kGK; ++q) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[q][ty * 4 + u];
        b[u] = Bs[q][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int gi = i0 + ty * 4 + u, gj = j0 + tx * 4 + v;
      if (gi < jb.M && gj < jb.N) {
        double* c = jb.C + gi + static_cast<int64_t>(gj) * jb.ldc;
        *c = jb.acc ? *c + jb.alpha * acc[u][v] : jb.alpha * acc[u][v];
      }
    }
}

// ------------------------------------------------- 2. Cholesky and inverse
// One CTA per job: G (k x k, ld k, symmetric positive definite in exact
// arithmetic) -> R upper triangular with D G D = Rs^T Rs, D = diag(G)^-1/2
// (column scaling), R = Rs D^-1 (so G = R^T R) and Ri = D Rs^-1 (= R^-1).
// A non-positive pivot sets *status = 2 (the block goes to the host).
struct CholJob {
  const double* G;
  double* R;
  double* Ri;
  int k, pad;
  int* status;
};

__global__ void __launch_bounds__(256) chol_kernel(const CholJob* jobs) {
  const CholJob jb = jobs[blockIdx.x];
  const int k = jb.k;
  if (k == 0 || *jb.status != 0) return;
  double* L = jb.Ri;  // lower Cholesky factor of D G D, built in Ri's storage first
  extern __shared__ double d[];  // [k] scale
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double g = jb.G[i + static_cast<int64_t>(i) * k];
    d[i] = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
    if (!(g > 0.0)) bad = 1;
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) *jb.status = 2;
    return;
  }
  // left-looking: column j of L from the scaled G and columns < j
  for (int j = 0; j < k; ++j) {
    __shared__ double piv;
    if (threadIdx.x == 0) {
      double s = jb.G[j + static_cast<int64_t>(j) * k] * d[j] * d[j];
      for (int l = 0; l < j; ++l) s -= L[j + static_cast<int64_t>(l) * k] * L[j + static_cast<int64_t>(l) * k];
      piv = s > 0.0 ? sqrt(s) : -1.0;
    }
    __syncthreads();
    if (piv <= 0.0) {
      if (threadIdx.x == 0) *jb.status = 2;
      return;
    }
    for (int i = j + threadIdx.x; i < k; i += blockDim.x) {
      if (i == j) {
        L[j + static_cast<int64_t>(j) * k] = piv;
        continue;
      }
      double s = jb.G[i + static_cast<int64_t>(j) * k] * d[i] * d[j];
      for (int l = 0; l < j; ++l) s -= L[i + static_cast<int64_t>(l) * k] * L[j + static_cast<int64_t>(l) * k];
      L[i + static_cast<int64_t>(j) * k] = s / piv;
    }
    __syncthreads();
  }
  // R = Rs D^-1 = L^T D^-1 (upper), zero below the diagonal
  for (int64_t e = threadIdx.x; e < static_cast<int64_t>(k) * k; e += blockDim.x) {
    const int i = static_cast<int>(e % k), c = static_cast<int>(e / k);
    jb.R[e] = i <= c ? L[c + static_cast<int64_t>(i) * k] / d[c] : 0.0;
  }
  __syncthreads();
  // X = Rs^-1 (upper triangular) by back substitution, one column c per
  // thread: X[c][c] = 1 / Rs[c][c], X[i][c] = -(sum_{l=i+1..c} Rs[i][l]
  // X[l][c]) / Rs[i][i] with Rs[i][l] = L[l][i] read below the diagonal; X's
  // strictly upper part is written above the diagonal (where L holds
  // nothing), so a thread writes only its own column.
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double xcc = 1.0 / L[c + static_cast<int64_t>(c) * k];
    for (int i = c - 1; i >= 0; --i) {
      double s = L[c + static_cast<int64_t>(i) * k] * xcc;
      for (int l = i + 1; l < c; ++l) s += L[l + static_cast<int64_t>(i) * k] * L[l + static_cast<int64_t>(c) * k];
      L[i + static_cast<int64_t>(c) * k] = -s / L[i + static_cast<int64_t>(i) * k];
    }
  }
  __syncthreads();
  // Ri = D X in place: each element reads and writes only its own position
  for (int64_t e = threadIdx.x; e < static_cast<int64_t>(k) * k; e += blockDim.x) {
    const int i = static_cast<int>(e % k), c = static_cast<int>(e / k);
    const double v = L[e];
    L[e] = i < c ? d[i] * v : (i == c ? d[i] / v : 0.0);
  }
}

// ------------------------------------- 3. SVD of the core, QR-preconditioned
// The left singular vectors of T (k x k) as the host builder takes them:
// T P = Q1 R1 (Householder QR with column pivoting), R1^T = Q2 R2, so that
// T = Q1 R2^T Q2^T P^T and the left singular vectors of T are Q1 times those
// of X = R2^T, whose columns are nearly orthogonal; a one-sided (Hestenes)
// Jacobi iteration on X's columns then converges in a few sweeps.

// Householder QR of A (k x k, ld k) in place, one CTA per job: R in the upper
// triangle, reflector tails below it (v_j[j] = 1), tau[j]; with pivot the
// column of largest remaining norm goes first (norms kept in nrm, downdated
// and recomputed when cancellation eats them).
struct QrJob {
  double* A;
  double* tau;
  double* nrm;  // k scratch
  int k, pivot;
  int* status;
};

__global__ void __launch_bounds__(512) qr_kernel(const QrJob* jobs) {
  const QrJob jb = jobs[blockIdx.x];
  const int k = jb.k;
  if (k == 0 || *jb.status != 0) return;
  double* A = jb.A;
  __shared__ double redv[32];
  __shared__ int64_t redi[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  auto col = [&](int c) { return A + static_cast<int64_t>(c) * k; };
  if (jb.pivot) {
    for (int c = warp; c < k; c += nw) {
      const double* a = col(c);
      double s = 0.0;
      for (int e = lane; e < k; e += 32) s += a[e] * a[e];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) jb.nrm[c] = s;
    }
    __syncthreads();
  }
  for (int j = 0; j < k; ++j) {
    if (jb.pivot) {
      double a = -1.0, best;
      int64_t at = j, p;
      for (int c = j + threadIdx.x; c < k; c += blockDim.x)
        if (jb.nrm[c] > a) {
          a = jb.nrm[c];
          at = c;
        }
      cta_argmax(a, at, redv, redi, best, p);
      if (p != j) {
        for (int e = threadIdx.x; e < k; e += blockDim.x) {
          const double t = col(j)[e];
          col(j)[e] = col(static_cast<int>(p))[e];
          col(static_cast<int>(p))[e] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          const double t = jb.nrm[j];
          jb.nrm[j] = jb.nrm[p];
          jb.nrm[p] = t;
        }
      }
    }
    double* v = col(j);
    double s = 0.0;
    for (int e = j + 1 + threadIdx.x; e < k; e += blockDim.x) s += v[e] * v[e];
    const double sigma = cta_sum(s, redv);
    const double alpha = v[j];
    double tau = 0.0, beta = alpha;
    if (sigma > 0.0) {
      beta = (alpha >= 0.0 ? -1.0 : 1.0) * sqrt(alpha * alpha + sigma);
      tau = (beta - alpha) / beta;
      const double sc = 1.0 / (alpha - beta);
      for (int e = j + 1 + threadIdx.x; e < k; e += blockDim.x) v[e] *= sc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      v[j] = beta;
      jb.tau[j] = tau;
    }
    // apply H_j to the columns c > j (a warp per column)
    if (tau != 0.0)
      for (int c = j + 1 + warp; c < k; c += nw) {
        double* a = col(c);
        double w = lane == 0 ? a[j] : 0.0;
        for (int e = j + 1 + lane; e < k; e += 32) w += v[e] * a[e];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w *= tau;
        if (lane == 0) a[j] -= w;
        for (int e = j + 1 + lane; e < k; e += 32) a[e] -= w * v[e];
      }
    __syncthreads();
    if (jb.pivot)
      for (int c = j + 1 + warp; c < k; c += nw) {
        const double* a = col(c);
        const double r = a[j];
        double nv = jb.nrm[c] - r * r;
        if (!(nv > 1e-2 * jb.nrm[c])) {  // cancellation: recompute the trailing norm
          double t = 0.0;
          for (int e = j + 1 + lane; e < k; e += 32) t += a[e] * a[e];
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          nv = t;
        }
        __syncwarp();
        if (lane == 0) jb.nrm[c] = nv;
      }
    __syncthreads();
  }
}

// out (k x k) = R^T of the upper triangle of in (zero above the diagonal)
__global__ void rt_kernel(const double* const* in, double* const* out, const int* ks, const int* const* status) {
  const int k = ks[blockIdx.x];
  if (k == 0 || *status[blockIdx.x] != 0) return;
  const double* a = in[blockIdx.x];
  double* b = out[blockIdx.x];
  for (int64_t e = threadIdx.x; e < static_cast<int64_t>(k) * k; e += blockDim.x) {
    const int i = static_cast<int>(e % k), c = static_cast<int>(e / k);
    b[e] = i >= c ? a[c + static_cast<int64_t>(i) * k] : 0.0;
  }
}

// One-sided Jacobi on the columns of X (k x k) until every pair is
// orthogonal to 1e-15 relative (at most kJacobiSweeps sweeps, else *status =
// 3); pairs in k' - 1 round-robin rounds of k' / 2 disjoint pairs per sweep
// (k' = k rounded up to even, index k a dummy), a warp per pair.
struct JacJob {
  double* X;
  int k, pad;
  int* status;
  int* sweeps;  // out: sweeps taken
};

__global__ void __launch_bounds__(512) jacobi_kernel(const JacJob* jobs) {
  const JacJob jb = jobs[blockIdx.x];
  const int k = jb.k;
  if (k == 0 || *jb.status != 0) return;
  double* X = jb.X;
  extern __shared__ double nrm[];  // squared column norms, updated by each rotation
  const int kk = (k + 1) & ~1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __shared__ int rotated;
  int sweep = 0;
  for (; sweep < kJacobiSweeps; ++sweep) {
    for (int c = warp; c < k; c += nw) {  // exact norms at the start of every sweep
      const double* x = X + static_cast<int64_t>(c) * k;
      double t = 0.0;
      for (int e = lane; e < k; e += 32) t += x[e] * x[e];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) nrm[c] = t;
    }
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r + 1 < kk; ++r) {
      for (int a = warp; a < kk / 2; a += nw) {
        const int pa = a == 0 ? 0 : 1 + (a - 1 + r) % (kk - 1);
        const int pb = 1 + (kk - 2 - a + r) % (kk - 1);
        const int p = pa < pb ? pa : pb, q = pa < pb ? pb : pa;
        if (q >= k) continue;
        double* xp = X + static_cast<int64_t>(p) * k;
        double* xq = X + static_cast<int64_t>(q) * k;
        const double al = nrm[p], be = nrm[q];
        if (al == 0.0 || be == 0.0) continue;
        double ga = 0.0;
        for (int e = lane; e < k; e += 32) ga += xp[e] * xq[e];
        for (int o = 16; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
        if (!(fabs(ga) > 1e-15 * sqrt(al) * sqrt(be))) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        double np = 0.0, nq = 0.0;
        for (int e = lane; e < k; e += 32) {
          const double x = xp[e], y = xq[e];
          const double u = c * x - s * y, v = s * x + c * y;
          xp[e] = u;
          xq[e] = v;
          np += u * u;
          nq += v * v;
        }
        // the rotation moves t gamma of squared norm from p to q; where that
        // update would mostly cancel, take the norm just accumulated
        const double up = al - t * ga, uq = be + t * ga;
        if (!(up > 0.25 * al) || !(uq > 0.25 * be)) {
          for (int o = 16; o > 0; o >>= 1) {
            np += __shfl_xor_sync(0xffffffffu, np, o);
            nq += __shfl_xor_sync(0xffffffffu, nq, o);
          }
        }
        if (lane == 0) {
          nrm[p] = up > 0.25 * al ? up : np;
          nrm[q] = uq > 0.25 * be ? uq : nq;
          rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  if (threadIdx.x == 0) {
    *jb.sweeps = sweep;
    if (sweep == kJacobiSweeps) *jb.status = 3;
  }
}

// ------------------------------------------------------------ 4. truncation
// One CTA per job: sigma_i = |X[:, i]| (X rotated), sorted descending (ties
// by column); r = smallest rank whose Frobenius tail is <= teps times the
// whole; W[:, t] = X[:, i_t] / sigma_t for t < r; sig[t] = sigma_t; *r_out = r.
struct FinJob {
  const double* X;
  double* W;
  double* sig;   // 2k doubles (the unsorted norms at sig + k)
  int* order;    // k
  int k, pad;
  int* r_out;
  int* status;
};

__global__ void __launch_bounds__(256) finalize_kernel(const FinJob* jobs, double teps) {
  const FinJob jb = jobs[blockIdx.x];
  const int k = jb.k;
  if (k == 0 || *jb.status != 0) {
    if (threadIdx.x == 0) *jb.r_out = 0;
    return;
  }
  double* nrm = jb.sig + k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = warp; c < k; c += nw) {
    const double* t = jb.X + static_cast<int64_t>(c) * k;
    double s = 0.0;
    for (int e = lane; e < k; e += 32) s += t[e] * t[e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[c] = sqrt(s);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    int pos = 0;
    const double v = nrm[i];
    for (int j = 0; j < k; ++j) pos += (nrm[j] > v || (nrm[j] == v && j < i)) ? 1 : 0;
    jb.order[pos] = i;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k; t += blockDim.x) jb.sig[t] = nrm[jb.order[t]];
  __syncthreads();
  __shared__ int rr;
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int t = k - 1; t >= 0; --t) total += jb.sig[t] * jb.sig[t];
    int r = k;
    if (total == 0.0) {
      r = 0;
    } else {
      const double lim = teps * sqrt(total);
      double tail = 0.0;  // sum of sig[t..k)^2, from the end
      for (int t = k - 1; t >= 0; --t) {
        const double nt = tail + jb.sig[t] * jb.sig[t];
        if (sqrt(nt) <= lim) {
          tail = nt;
          r = t;
        } else {
          break;
        }
      }
    }
    rr = r;
    *jb.r_out = r;
  }
  __syncthreads();
  const int r = rr;
  for (int64_t e = threadIdx.x; e < static_cast<int64_t>(k) * r; e += blockDim.x) {
    const int row = static_cast<int>(e % k), t = static_cast<int>(e / k);
    jb.W[row + static_cast<int64_t>(t) * k] = jb.X[row + static_cast<int64_t>(jb.order[t]) * k] / jb.sig[t];
  }
}

// W (k x r, ld k) <- Q1 W with Q1 = H_0 ... H_{k-1} held as reflector tails
// below the diagonal of F (k x k) and tau: the reflectors applied last to
// first, a warp per column of W
struct ApplyQJob {
  const double* F;
  const double* tau;
  double* W;
  int k, r;
  int* status;
};

__global__ void __launch_bounds__(512) applyq_kernel(const ApplyQJob* jobs) {
  const ApplyQJob jb = jobs[blockIdx.x];
  const int k = jb.k, r = jb.r;
  if (k == 0 || r == 0 || *jb.status != 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = warp; c < r; c += nw) {
    double* w = jb.W + static_cast<int64_t>(c) * k;
    for (int j = k - 1; j >= 0; --j) {
      const double tau = jb.tau[j];
      if (tau == 0.0) continue;
      const double* v = jb.F + static_cast<int64_t>(j) * k;
      double d = lane == 0 ? w[j] : 0.0;
      for (int e = j + 1 + lane; e < k; e += 32) d += v[e] * w[e];
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      d *= tau;
      if (lane == 0) w[j] -= d;
      for (int e = j + 1 + lane; e < k; e += 32) w[e] -= d * v[e];
      __syncwarp();
    }
  }
}

}  // namespace

namespace {

// device buffer freed at scope exit
struct DevBuf {
  void* p = nullptr;
  explicit DevBuf(size_t bytes) {
    if (bytes) ck(cudaMalloc(&p, bytes), "cudaMalloc");
  }
  ~DevBuf() { cudaFree(p); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  template <class T>
  T* as(size_t byte_off = 0) const { return reinterpret_cast<T*>(static_cast<char*>(p) + byte_off); }
};

template <class T>
void upload_vec(const std::vector<T>& v, DevBuf& b) {
  if (!v.empty()) ck(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
}

// one batched GEMM launch over `js`
void run_gemms(const std::vector<GemmJob>& js) {
  if (js.empty()) return;
  std::vector<int64_t> start(js.size());
  int64_t tiles = 0;
  for (size_t q = 0; q < js.size(); ++q) {
    start[q] = tiles;
    tiles += int64_t((js[q].M + kGT - 1) / kGT) * ((js[q].N + kGT - 1) / kGT);
  }
  if (tiles == 0) return;
  DevBuf dj(js.size() * sizeof(GemmJob)), ds(start.size() * sizeof(int64_t));
  upload_vec(js, dj);
  upload_vec(start, ds);
  gemm_kernel<<<static_cast<unsigned>(tiles), 256>>>(dj.as<GemmJob>(), ds.as<int64_t>(), static_cast<int>(js.size()));
  ck(cudaGetLastError(), "gemm launch");
  ck(cudaDeviceSynchronize(), "gemm");
}

GemmJob gj(const double* A, int64_t a_rs, int64_t a_cs, const double* B, int64_t b_rs, int64_t b_cs, double* C,
           int64_t ldc, int M, int N, int K) {
  GemmJob g;
  g.A = A;
  g.B = B;
  g.C = C;
  g.a_rs = a_rs;
  g.a_cs = a_cs;
  g.b_rs = b_rs;
  g.b_cs = b_cs;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.acc = 0;
  g.alpha = 1.0;
  return g;
}

// wall time per stage, printed to stderr when HH_CONSTRUCT_TIMING is set
struct StageClock {
  bool on = std::getenv("HH_CONSTRUCT_TIMING") != nullptr;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  double acc[8] = {};
  void mark(int stage) {
    if (!on) return;
    cudaDeviceSynchronize();
    const auto now = std::chrono::steady_clock::now();
    acc[stage] += std::chrono::duration<double>(now - t).count();
    t = now;
  }
  void report() const {
    if (!on) return;
    std::fprintf(stderr, "device compression stages (s): aca %.3f qr %.3f core %.3f jacobi %.3f final %.3f copy %.3f\n",
                 acc[0], acc[1], acc[2], acc[3], acc[4], acc[5]);
  }
};

// per job of a wave: where its buffers live (byte offsets)
struct Slot {
  size_t u, v, used;                 // ACA: U (m x cap), V (n x cap), flags
  size_t q1u, q1v;                   // recompression: Q1 of U / V, later the final factors
  size_t gu, ru1, riu1, ru2, riu2;   // k x k each
  size_t gv, rv1, riv1, rv2, riv2;
  size_t t, j, w, jr, sig, order, st, tau1, tau2;
};

}  // namespace

void compress_on_device(int device, const double* tp, int64_t n_pts, int dim, int kernel, double kparam,
                        double eps, const std::vector<DeviceJob>& jobs, std::vector<la::Mat>& U,
                        std::vector<la::Mat>& V, std::vector<std::vector<double>>& s, std::vector<char>& ok,
                        DeviceStats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  const size_t nj = jobs.size();
  U.assign(nj, la::Mat());
  V.assign(nj, la::Mat());
  s.assign(nj, {});
  ok.assign(nj, 0);
  if (nj == 0) return;
  ck(cudaSetDevice(device), "cudaSetDevice");
  DevBuf dpts(sizeof(double) * static_cast<size_t>(n_pts * dim));
  ck(cudaMemcpy(dpts.p, tp, sizeof(double) * n_pts * dim, cudaMemcpyHostToDevice), "points");
  const Geo geo{dpts.as<double>(), dim, kernel, kparam};
  ck(cudaFuncSetAttribute(aca_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * kMaxRankCap * 8),
     "smem attribute");
  size_t free_b = 0, total_b = 0;
  ck(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
  const size_t budget = std::min<size_t>(free_b / 2, size_t(64) << 30);
  auto a256 = [](size_t x) { return (x + 255) / 256 * 256; };
  // jobs by cost, largest first
  std::vector<size_t> order(nj);
  std::iota(order.begin(), order.end(), size_t(0));
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return jobs[a].m * jobs[a].n > jobs[b].m * jobs[b].n;
  });
  auto cap_of = [](const DeviceJob& j) { return static_cast<int>(std::min<int64_t>({j.m, j.n, kMaxRankCap})); };
  int64_t fallback = 0, waves = 0;
  StageClock clk;
  size_t next = 0;
  while (next < nj) {
    // ---- a wave: as many jobs as fit the budget with their ACA workspace
    std::vector<size_t> wave;
    std::vector<Slot> slot;
    size_t bytes = 0;
    while (next < nj) {
      const DeviceJob& J = jobs[order[next]];
      const size_t c = cap_of(J);
      const size_t need = a256(8 * J.m * c) + a256(8 * J.n * c) + a256(4 * J.m);
      if (!wave.empty() && bytes + 3 * need > budget) break;  // room for the recompression too
      Slot sl{};
      sl.u = bytes;
      sl.v = sl.u + a256(8 * J.m * c);
      sl.used = sl.v + a256(8 * J.n * c);
      bytes = sl.used + a256(4 * J.m);
      wave.push_back(order[next++]);
      slot.push_back(sl);
    }
    ++waves;
    const size_t nw = wave.size();
    DevBuf ws(bytes);
    std::vector<AcaJob> aj(nw);
    for (size_t q = 0; q < nw; ++q) {
      const DeviceJob& J = jobs[wave[q]];
      aj[q] = AcaJob{J.r0, J.m, J.c0, J.n, ws.as<double>(slot[q].u), ws.as<double>(slot[q].v),
                     ws.as<int>(slot[q].used), cap_of(J), 0, 0, 0};
    }
    DevBuf daj(nw * sizeof(AcaJob));
    upload_vec(aj, daj);
    int capmax = 1;
    for (auto& a : aj) capmax = std::max(capmax, a.cap);
    aca_kernel<<<static_cast<unsigned>(nw), kAcaThreads, 3 * capmax * 8>>>(daj.as<AcaJob>(), geo, kAcaShare * eps,
                                                                          kAcaPatience);
    ck(cudaGetLastError(), "aca launch");
    ck(cudaDeviceSynchronize(), "aca");
    ck(cudaMemcpy(aj.data(), daj.p, nw * sizeof(AcaJob), cudaMemcpyDeviceToHost), "aca results");
    clk.mark(0);
    // ---- recompression of the jobs ACA finished (buffers sized by rank)
    std::vector<size_t> live;  // wave positions
    std::vector<Slot> rs;
    size_t rbytes = 0;
    for (size_t q = 0; q < nw; ++q) {
      if (aj[q].status != 0) {
        ++fallback;
        continue;
      }
      const DeviceJob& J = jobs[wave[q]];
      const size_t k = static_cast<size_t>(aj[q].k);
      if (k == 0) {  // zero block
        U[wave[q]] = la::Mat(J.m, 0);
        V[wave[q]] = la::Mat(J.n, 0);
        ok[wave[q]] = 1;
        continue;
      }
      Slot sl = slot[q];
      auto take = [&](size_t b) {
        const size_t o = rbytes;
        rbytes += a256(b);
        return o;
      };
      sl.q1u = take(8 * J.m * k);
      sl.q1v = take(8 * J.n * k);
      size_t* kk[] = {&sl.gu, &sl.ru1, &sl.riu1, &sl.ru2, &sl.riu2, &sl.gv, &sl.rv1, &sl.riv1, &sl.rv2, &sl.riv2,
                      &sl.t, &sl.j, &sl.w, &sl.jr};
      for (size_t* p : kk) *p = take(8 * k * k);
      sl.sig = take(16 * k);
      sl.tau1 = take(8 * k);
      sl.tau2 = take(8 * k);
      sl.order = take(4 * k);
      sl.st = take(8);
      live.push_back(q);
      rs.push_back(sl);
    }
    if (!live.empty()) {
      DevBuf rb(rbytes);
      ck(cudaMemset(rb.p, 0, rbytes), "clear");
      const size_t nl = live.size();
      auto D = [&](size_t off) { return rb.as<double>(off); };
      auto Uq = [&](size_t i) { return ws.as<double>(rs[i].u); };
      auto Vq = [&](size_t i) { return ws.as<double>(rs[i].v); };
      std::vector<GemmJob> g;
      auto dims = [&](size_t i, int& m, int& n, int& k) {
        const DeviceJob& J = jobs[wave[live[i]]];
        m = static_cast<int>(J.m);
        n = static_cast<int>(J.n);
        k = aj[live[i]].k;
      };
      auto chol = [&](bool second) {
        std::vector<CholJob> cj;
        for (size_t i = 0; i < nl; ++i) {
          int m, n, k;
          dims(i, m, n, k);
          const Slot& sl = rs[i];
          int* st = rb.as<int>(sl.st);
          cj.push_back(CholJob{D(sl.gu), D(second ? sl.ru2 : sl.ru1), D(second ? sl.riu2 : sl.riu1), k, 0, st});
          cj.push_back(CholJob{D(sl.gv), D(second ? sl.rv2 : sl.rv1), D(second ? sl.riv2 : sl.riv1), k, 0, st});
        }
        DevBuf dc(cj.size() * sizeof(CholJob));
        upload_vec(cj, dc);
        chol_kernel<<<static_cast<unsigned>(cj.size()), 256, kMaxRankCap * 8>>>(dc.as<CholJob>());
        ck(cudaGetLastError(), "cholesky launch");
        ck(cudaDeviceSynchronize(), "cholesky");
      };
      // Gram matrices of the cross factors
      for (size_t i = 0; i < nl; ++i) {
        int m, n, k;
        dims(i, m, n, k);
        g.push_back(gj(Uq(i), m, 1, Uq(i), 1, m, D(rs[i].gu), k, k, k, m));
        g.push_back(gj(Vq(i), n, 1, Vq(i), 1, n, D(rs[i].gv), k, k, k, n));
      }
      run_gemms(g);
      chol(false);
      g.clear();  // Q1 = X R1^-1
      for (size_t i = 0; i < nl; ++i) {
        int m, n, k;
        dims(i, m, n, k);
        g.push_back(gj(Uq(i), 1, m, D(rs[i].riu1), 1, k, D(rs[i].q1u), m, m, k, k));
        g.push_back(gj(Vq(i), 1, n, D(rs[i].riv1), 1, k, D(rs[i].q1v), n, n, k, k));
      }
      run_gemms(g);
      g.clear();  // Gram of Q1
      for (size_t i = 0; i < nl; ++i) {
        int m, n, k;
        dims(i, m, n, k);
        g.push_back(gj(D(rs[i].q1u), m, 1, D(rs[i].q1u), 1, m, D(rs[i].gu), k, k, k, m));
        g.push_back(gj(D(rs[i].q1v), n, 1, D(rs[i].q1v), 1, n, D(rs[i].gv), k, k, k, n));
      }
      run_gemms(g);
      chol(true);
      g.clear();  // Q = Q1 R2^-1 (into the ACA buffers), R = R2 R1 (into the Gram buffers)
      for (size_t i = 0; i < nl; ++i) {
        int m, n, k;
        dims(i, m, n, k);
        g.push_back(gj(D(rs[i].q1u), 1, m, D(rs[i].riu2), 1, k, Uq(i), m, m, k, k));
        g.push_back(gj(D(rs[i].q1v), 1, n, D(rs[i].riv2), 1, k, Vq(i), n, n, k, k));
        g.push_back(gj(D(rs[i].ru2), 1, k, D(rs[i].ru1), 1, k, D(rs[i].gu), k, k, k, k));
        g.push_back(gj(D(rs[i].rv2), 1, k, D(rs[i].rv1), 1, k, D(rs[i].gv), k, k, k, k));
      }
      run_gemms(g);
      clk.mark(1);
      g.clear();  // T = R_u R_v^T
      for (size_t i = 0; i < nl; ++i) {
        int m, n, k;
        dims(i, m, n, k);
        g.push_back(gj(D(rs[i].gu), 1, k, D(rs[i].gv), k, 1, D(rs[i].t), k, k, k, k));
      }
      run_gemms(g);
      clk.mark(2);
      // SVD of T, QR-preconditioned: F = copy of T, F P = Q1 R1; X = R1^T = Q2 R2;
      // Jacobi on X2 = R2^T (in jr); W = Q1 (left singular vectors of X2)_r
      for (size_t i = 0; i < nl; ++i) {
        int m, n, k;
        dims(i, m, n, k);
        ck(cudaMemcpy(D(rs[i].j), D(rs[i].t), 8 * size_t(k) * k, cudaMemcpyDeviceToDevice), "copy T");
      }
      auto launch_qr = [&](bool first) {
        std::vector<QrJob> qj;
        for (size_t i = 0; i < nl; ++i) {
          int m, n, k;
          dims(i, m, n, k);
          qj.push_back(QrJob{D(first ? rs[i].j : rs[i].w), D(first ? rs[i].tau1 : rs[i].tau2), D(rs[i].sig) + k, k,
                             first ? 1 : 0, rb.as<int>(rs[i].st)});
        }
        DevBuf dq(qj.size() * sizeof(QrJob));
        upload_vec(qj, dq);
        qr_kernel<<<static_cast<unsigned>(nl), 512>>>(dq.as<QrJob>());
        ck(cudaGetLastError(), "qr launch");
        ck(cudaDeviceSynchronize(), "qr");
      };
      auto launch_rt = [&](bool first) {  // first: w = R1^T from j; else jr = R2^T from w
        std::vector<const double*> in(nl);
        std::vector<double*> out(nl);
        std::vector<int> ks(nl);
        std::vector<const int*> sts(nl);
        for (size_t i = 0; i < nl; ++i) {
          int m, n, k;
          dims(i, m, n, k);
          in[i] = D(first ? rs[i].j : rs[i].w);
          out[i] = D(first ? rs[i].w : rs[i].jr);
          ks[i] = k;
          sts[i] = rb.as<int>(rs[i].st);
        }
        DevBuf di(nl * sizeof(void*)), dout(nl * sizeof(void*)), dk(nl * sizeof(int)), ds(nl * sizeof(void*));
        upload_vec(in, di);
        upload_vec(out, dout);
        upload_vec(ks, dk);
        upload_vec(sts, ds);
        rt_kernel<<<static_cast<unsigned>(nl), 256>>>(di.as<const double*>(), dout.as<double*>(), dk.as<int>(),
                                                      ds.as<const int*>());
        ck(cudaGetLastError(), "transpose launch");
        ck(cudaDeviceSynchronize(), "transpose");
      };
      launch_qr(true);
      launch_rt(true);
      launch_qr(false);
      launch_rt(false);
      std::vector<JacJob> jj;
      std::vector<FinJob> fj;
      DevBuf rout(nl * sizeof(int)), dsw(nl * sizeof(int));
      for (size_t i = 0; i < nl; ++i) {
        int m, n, k;
        dims(i, m, n, k);
        int* st = rb.as<int>(rs[i].st);
        jj.push_back(JacJob{D(rs[i].jr), k, 0, st, dsw.as<int>(i * sizeof(int))});
        fj.push_back(FinJob{D(rs[i].jr), D(rs[i].w), D(rs[i].sig), rb.as<int>(rs[i].order), k, 0,
                            rout.as<int>(i * sizeof(int)), st});
      }
      DevBuf djj(jj.size() * sizeof(JacJob)), dfj(fj.size() * sizeof(FinJob));
      upload_vec(jj, djj);
      upload_vec(fj, dfj);
      jacobi_kernel<<<static_cast<unsigned>(nl), 512, kMaxRankCap * 8>>>(djj.as<JacJob>());
      ck(cudaGetLastError(), "jacobi launch");
      ck(cudaDeviceSynchronize(), "jacobi");
      clk.mark(3);
      if (clk.on) {
        std::vector<int> sw(nl);
        ck(cudaMemcpy(sw.data(), dsw.p, nl * sizeof(int), cudaMemcpyDeviceToHost), "sweeps");
        int kmx = 0, smx = 0;
        double sm = 0.0;
        for (size_t i = 0; i < nl; ++i) {
          int m, n, k;
          dims(i, m, n, k);
          kmx = std::max(kmx, k);
          smx = std::max(smx, sw[i]);
          sm += sw[i];
        }
        std::fprintf(stderr, "jacobi: %zu cores, largest k %d, sweeps max %d mean %.1f\n", nl, kmx, smx, sm / nl);
      }
      finalize_kernel<<<static_cast<unsigned>(nl), 256>>>(dfj.as<FinJob>(), (1.0 - kAcaShare) * eps);
      ck(cudaGetLastError(), "truncation launch");
      ck(cudaDeviceSynchronize(), "truncation");
      std::vector<int> rr(nl), stv(nl);
      ck(cudaMemcpy(rr.data(), rout.p, nl * sizeof(int), cudaMemcpyDeviceToHost), "ranks");
      for (size_t i = 0; i < nl; ++i)
        ck(cudaMemcpy(&stv[i], rb.as<int>(rs[i].st), sizeof(int), cudaMemcpyDeviceToHost), "status");
      {  // W <- Q1 W
        std::vector<ApplyQJob> aq;
        for (size_t i = 0; i < nl; ++i) {
          int m, n, k;
          dims(i, m, n, k);
          aq.push_back(ApplyQJob{D(rs[i].j), D(rs[i].tau1), D(rs[i].w), k, stv[i] == 0 ? rr[i] : 0,
                                 rb.as<int>(rs[i].st)});
        }
        DevBuf da(aq.size() * sizeof(ApplyQJob));
        upload_vec(aq, da);
        applyq_kernel<<<static_cast<unsigned>(nl), 512>>>(da.as<ApplyQJob>());
        ck(cudaGetLastError(), "apply Q launch");
        ck(cudaDeviceSynchronize(), "apply Q");
      }
      g.clear();  // Y = T^T W (= Z_r Sigma_r) into jr
      for (size_t i = 0; i < nl; ++i) {
        int m, n, k;
        dims(i, m, n, k);
        if (stv[i] != 0 || rr[i] == 0) continue;
        g.push_back(gj(D(rs[i].t), k, 1, D(rs[i].w), 1, k, D(rs[i].jr), k, k, rr[i], k));
      }
      run_gemms(g);
      g.clear();  // U_b = Q_u W_r, V_b = Q_v Y (into the Q1 buffers)
      for (size_t i = 0; i < nl; ++i) {
        int m, n, k;
        dims(i, m, n, k);
        if (stv[i] != 0 || rr[i] == 0) continue;
        g.push_back(gj(Uq(i), 1, m, D(rs[i].w), 1, k, D(rs[i].q1u), m, m, rr[i], k));
        g.push_back(gj(Vq(i), 1, n, D(rs[i].jr), 1, k, D(rs[i].q1v), n, n, rr[i], k));
      }
      run_gemms(g);
      clk.mark(4);
      for (size_t i = 0; i < nl; ++i) {
        const size_t job = wave[live[i]];
        const DeviceJob& J = jobs[job];
        if (stv[i] != 0) {
          ++fallback;
          continue;
        }
        const int r = rr[i];
        U[job] = la::Mat(J.m, r);
        V[job] = la::Mat(J.n, r);
        s[job].resize(static_cast<size_t>(r));
        if (r > 0) {
          ck(cudaMemcpy(U[job].a.data(), D(rs[i].q1u), 8 * J.m * r, cudaMemcpyDeviceToHost), "U");
          ck(cudaMemcpy(V[job].a.data(), D(rs[i].q1v), 8 * J.n * r, cudaMemcpyDeviceToHost), "V");
          ck(cudaMemcpy(s[job].data(), D(rs[i].sig), 8 * r, cudaMemcpyDeviceToHost), "sigma");
        }
        ok[job] = 1;
      }
      clk.mark(5);
    }
  }
  clk.report();
  if (stats) {
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->fallback = fallback;
    stats->waves = waves;
  }
}

}  // namespace hh
