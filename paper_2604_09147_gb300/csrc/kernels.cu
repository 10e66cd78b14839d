// Permutation kernels of the H_h product and the kernel-variant selection.
//
//   prep   : input vector (caller's order, column-major) -> tree order, as
//            its fp32 leading half hi = fl32(x) and trailing half
//            lo = fl32(x - hi), each in four copies shifted by 0..3 positions
//            so that every 16-byte vector of a factor column meets an aligned
//            vector of the input; clears the fp64 output accumulator (unless
//            it is passed as null) and the work counters of the two passes.
//   finish : output accumulator (tree order) -> the caller's order, through
//            the inverse permutation (caller position -> tree position).
//   presplit: fp64 factors and dense blocks -> pairs of fp32 values, once
//            when a matrix is uploaded.
// The two streaming passes between them live in stream.cu.
#include "hh_device.h"

namespace hh {
namespace dev {

namespace {

__global__ void prep_kernel(const double* __restrict__ in, int64_t ld, int nr,
                            const int32_t* __restrict__ perm, int64_t n, int64_t npad,
                            float* __restrict__ xs, float* __restrict__ xs_lo, double* __restrict__ acc,
                            int* __restrict__ counters) {
  if (counters && blockIdx.x == 0 && threadIdx.x < 2) counters[threadIdx.x] = 0;
  // one gather per tree position q, written into the four copies at q - s
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < npad + 3;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t u = q < n ? static_cast<int64_t>(perm[q]) : -1;
    for (int r = 0; r < nr; ++r) {
      const double v = u >= 0 ? in[u + r * ld] : 0.0;
      float hi, lo;
      split_f64(v, hi, lo);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int64_t p = q - s;
        if (p >= 0 && p < npad) {
          xs[(static_cast<int64_t>(s) * nr + r) * npad + p] = hi;
          xs_lo[(static_cast<int64_t>(s) * nr + r) * npad + p] = lo;
        }
      }
      if (acc && q < npad) acc[static_cast<int64_t>(r) * npad + q] = 0.0;
    }
  }
}

// fp64 values -> (hi, lo) = (fl32(v), fl32(v - hi)) in place, over spans
// {byte offset, count} of base: the device form of fp64 factors and dense
// blocks that the streaming and dense kernels read (run once per upload)
__global__ void presplit_kernel(uint8_t* __restrict__ base, const int64_t* __restrict__ spans, int nspans) {
  for (int s = blockIdx.x; s < nspans; s += gridDim.x) {
    double* p = reinterpret_cast<double*>(base + spans[2 * s]);
    float2* q = reinterpret_cast<float2*>(p);
    const int64_t n = spans[2 * s + 1];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      float hi, lo;
      split_f64(p[i], hi, lo);
      q[i] = make_float2(hi, lo);
    }
  }
}

// out[u + r ld] = acc[r npad + iperm[u]], column by column: consecutive
// threads take consecutive caller positions u of the same column, so the
// writes of a warp are coalesced and the gathered reads of the threads in
// flight stay in a few accumulator columns (L2); each thread handles four
// pairs with independent loads
__global__ void finish_kernel(const double* __restrict__ acc, int nr, const int32_t* __restrict__ iperm,
                              int64_t n, int64_t npad, double* __restrict__ out, int64_t ld) {
  // launched as a programmatic dependent of the last pass: wait for it
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t total = static_cast<int64_t>(nr) * n;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t q0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q0 < total; q0 += 4 * stride) {
    double v[4];
    int64_t o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t q = q0 + j * stride;
      o[j] = -1;
      if (q < total) {
        const int64_t r = q / n, u = q - r * n;
        v[j] = acc[r * npad + iperm[u]];
        o[j] = u + r * ld;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (o[j] >= 0) out[o[j]] = v[j];
  }
}

}  // namespace

cudaError_t launch_prep(const double* in, int64_t ld, int nr, const int32_t* perm, int64_t n,
                        int64_t npad, float* xs, float* xs_lo, double* acc, cudaStream_t st, int* counters) {
  int64_t blocks = (npad + 3 + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  prep_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(in, ld, nr, perm, n, npad, xs, xs_lo, acc, counters);
  return cudaGetLastError();
}

cudaError_t launch_presplit_f64(uint8_t* base, const int64_t* spans, int nspans, cudaStream_t st) {
  if (nspans <= 0) return cudaSuccess;
  presplit_kernel<<<nspans < 4096 ? nspans : 4096, 256, 0, st>>>(base, spans, nspans);
  return cudaGetLastError();
}

cudaError_t launch_finish(const double* acc, int nr, const int32_t* iperm, int64_t n, int64_t npad,
                          double* out, int64_t ld, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(blocks));
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, finish_kernel, acc, nr, iperm, n, npad, out, ld);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

unsigned pass_set_for(unsigned fmts_present) {
  if ((fmts_present & ~kSetF64) == 0) return kSetF64;
  if ((fmts_present & ~kSetF32) == 0) return kSetF32;
  return kSetAll;
}

}  // namespace dev
}  // namespace hh

// ---------------------------------------------------------------------------
// Batches of independent matrices: the tree-order positions of matrix j
// occupy [pofs[j], pofs[j] + npad_j) of one concatenated position space, its
// caller-order vector [xofs[j], xofs[j] + n_j) of the concatenated input and
// output.  The streaming passes then run over the concatenated tables.
namespace hh {
namespace dev {
namespace {


__global__ void bprep_kernel(const double* __restrict__ x, const int64_t* __restrict__ xofs,
                             const int32_t* __restrict__ perm, const int64_t* __restrict__ pofs,
                             const int64_t* __restrict__ ns, int count, int64_t np, float* __restrict__ xs,
                             float* __restrict__ xs_lo, double* __restrict__ acc, int* __restrict__ counters) {
  if (counters && blockIdx.x == 0 && threadIdx.x < 2) counters[threadIdx.x] = 0;
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < np;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x)
    batch_prep_position(p, x, xofs, perm, pofs, ns, count, np, xs, xs_lo, acc);
}

__global__ void bfinish_kernel(const double* __restrict__ acc, const int64_t* __restrict__ xofs,
                               const int32_t* __restrict__ perm, const int64_t* __restrict__ pofs,
                               const int64_t* __restrict__ ns, int count, int64_t np, double* __restrict__ y) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < np;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x)
    batch_finish_position(p, acc, xofs, perm, pofs, ns, count, y);
}

}  // namespace

cudaError_t launch_batch_prep(const double* x, const int64_t* xofs, const int32_t* perm, const int64_t* pofs,
                              const int64_t* ns, int count, int64_t np, float* xs, float* xs_lo, double* acc,
                              int* counters, cudaStream_t st) {
  int64_t blocks = (np + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  bprep_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(x, xofs, perm, pofs, ns, count, np, xs, xs_lo, acc,
                                                          counters);
  return cudaGetLastError();
}

cudaError_t launch_batch_finish(const double* acc, const int64_t* xofs, const int32_t* perm, const int64_t* pofs,
                                const int64_t* ns, int count, int64_t np, double* y, cudaStream_t st) {
  int64_t blocks = (np + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  bfinish_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(acc, xofs, perm, pofs, ns, count, np, y);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace hh

// ---------------------------------------------------------------------------
// Vector kernels of the conjugate-gradient solver (capi.cu: hh_solve_cg).
// Dot products are reduced per block into `partials` (block b writes
// partials[b]); the caller adds the partials in block order, so the result
// does not depend on scheduling.
namespace hh {
namespace dev {
namespace {

constexpr int kVecThreads = 256;

__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                           double* __restrict__ partials) {
  __shared__ double red[kVecThreads];
  double s = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    s += a[i] * b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kVecThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// q += shift p
__global__ void shift_kernel(double* __restrict__ q, const double* __restrict__ p, double shift, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    q[i] += shift * p[i];
}

// x += alpha p, r -= alpha q
// The solver's scalars live on the device (CgState); each kernel reads them
// there, so an iteration needs no host round trip.  `active` is decided at
// the start of an iteration: a converged, broken-down or finished solve
// leaves x, r and p untouched from then on.
__global__ void cg_step_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                               const double* __restrict__ q, const CgState* __restrict__ s, int64_t n) {
  if (s->active == 0.0) return;
  const double alpha = s->alpha;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
  }
}
__global__ void cg_dir_kernel(double* __restrict__ p, const double* __restrict__ r, const CgState* __restrict__ s,
                              int64_t n) {
  if (s->active == 0.0) return;
  const double beta = s->beta;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    p[i] = r[i] + beta * p[i];
}
// sum of the dot kernel's partials in block order (one thread: deterministic)
__device__ double sum_partials(const double* part) {
  double v = 0.0;
  for (int b = 0; b < kDotBlocks; ++b) v += part[b];
  return v;
}
// start of an iteration: pq = p . q; alpha = rr / pq, or a breakdown
__global__ void cg_alpha_kernel(const double* __restrict__ part, CgState* __restrict__ s) {
  if (threadIdx.x != 0) return;
  s->active = (s->done == 0.0 && s->iters < s->max_iter) ? 1.0 : 0.0;
  if (s->active == 0.0) return;
  const double pq = sum_partials(part);
  if (!(pq > 0.0)) {
    s->breakdown = 1.0;
    s->done = 1.0;
    s->active = 0.0;
    return;
  }
  s->alpha = s->rr / pq;
}
// end of an iteration: rr_new = r . r, beta = rr_new / rr, convergence test
__global__ void cg_beta_kernel(const double* __restrict__ part, CgState* __restrict__ s) {
  if (threadIdx.x != 0 || s->active == 0.0) return;
  const double rr_new = sum_partials(part);
  s->beta = rr_new / s->rr;
  s->rr = rr_new;
  s->iters += 1.0;
  if (!(sqrt(rr_new) > s->threshold)) s->done = 1.0;
}

int vec_blocks(int64_t n) {
  int64_t b = (n + kVecThreads - 1) / kVecThreads;
  if (b > kDotBlocks) b = kDotBlocks;
  return b < 1 ? 1 : static_cast<int>(b);
}

}  // namespace

cudaError_t launch_dot(const double* a, const double* b, int64_t n, double* partials, cudaStream_t st) {
  dot_kernel<<<kDotBlocks, kVecThreads, 0, st>>>(a, b, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_shift(double* q, const double* p, double shift, int64_t n, cudaStream_t st) {
  shift_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>(q, p, shift, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_step(double* x, double* r, const double* p, const double* q, const CgState* s, int64_t n,
                           cudaStream_t st) {
  cg_step_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>(x, r, p, q, s, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_dir(double* p, const double* r, const CgState* s, int64_t n, cudaStream_t st) {
  cg_dir_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>(p, r, s, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_alpha(const double* partials, CgState* s, cudaStream_t st) {
  cg_alpha_kernel<<<1, 32, 0, st>>>(partials, s);
  return cudaGetLastError();
}

cudaError_t launch_cg_beta(const double* partials, CgState* s, cudaStream_t st) {
  cg_beta_kernel<<<1, 32, 0, st>>>(partials, s);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace hh
