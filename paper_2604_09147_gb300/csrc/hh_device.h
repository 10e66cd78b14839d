// Device-side descriptors shared by the kernels and the C-ABI host code.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace hh {
namespace dev {

// One low-rank block seen from one direction of the product.
// Forward (y = A x):     f1 = V (rows n1 = |J|, input segment c1 = off(J)),
//                        f2 = U (rows n2 = |I|, output segment c2 = off(I)).
// Transpose (x = A^T y): f1 = U, f2 = V, c1 = off(I), c2 = off(J).
// Phase 1 computes t_j = sum_i f1[i, j] in[c1 + i] (scaled units),
// phase 2 adds 2^e * sum_j f2[i, j] t_j into out[c2 + i].
struct BlkDesc {
  const uint8_t* f1;
  const uint8_t* f2;
  int64_t ld1, ld2;  // leading dimensions in elements (multiples of 16 bytes)
  int32_t n1, n2;    // rows of f1 / f2
  int32_t c1, c2;    // tree positions of the input / output segments
  int32_t k, fmt;
  int32_t e;         // exp_u + exp_v: value = 2^e * stored products
  int32_t pad;
  int64_t toff;      // offset of t_b in the t arena of its precision (per RHS)
};
static_assert(sizeof(BlkDesc) == 72, "descriptor size");

// One dense fp64 block, column-major with leading dimension ld.
// Forward: out[r0 + i] += sum_j D[i, j] in[c0 + j];  transpose: roles of
// (r0, m) and (c0, n) swap and D is read as D^T.
struct DenseDesc {
  const double* d;
  int64_t ld;
  int32_t m, n, r0, c0;
};
static_assert(sizeof(DenseDesc) == 32, "descriptor size");

// A unit of work for one warp.
//   kind 0: phase-1 columns [lo, hi) of low-rank block idx
//   kind 1: phase-2 rows [lo, hi) of low-rank block idx
//   kind 2: dense block idx, forward, rows [lo, hi)
//   kind 3: dense block idx, transposed, columns [lo, hi) of D
struct Item {
  int32_t kind, idx, lo, hi;
};

// Arguments of one pass (phase 1 or phase 2) over a list of items.
struct PassArgs {
  const BlkDesc* blk;
  const DenseDesc* dns;
  const Item* items;
  int32_t n_items;
  int32_t nr;           // right-hand sides in this chunk (1, 2 or 4)
  int64_t npad;         // padded vector length (multiple of 4, >= n + 32)
  const float* xs;      // [4][nr][npad] fp32 copies of the input, shifted by s
  const double* xs64;   // [2][nr][npad] fp64 copies, shifted by s
  float* t32;           // t of non-fp64 blocks  [toff + j * nr + r]
  double* t64;          // t of fp64 blocks
  double* acc;          // [nr][npad] fp64 output accumulator (tree order)
  int* status;          // device status word (bit 0: bad descriptor)
};

// host-callable launchers (kernels.cu)
cudaError_t launch_prep(const double* in, int64_t ld, int nr, const int32_t* perm, int64_t n,
                        int64_t npad, float* xs, double* xs64, double* acc, cudaStream_t st);
// kernel variants by the set of factor formats they contain (bit f = fmt f)
constexpr unsigned kSetF64 = 1u;         // fp64 factors (and dense blocks)
constexpr unsigned kSetF32 = 1u | 2u;    // fp64 + fp32
constexpr unsigned kSetAll = 31u;        // every format
unsigned pass_set_for(unsigned fmts_present);
cudaError_t launch_pass(int phase, unsigned fset, const PassArgs& a, int grid, cudaStream_t st);
cudaError_t launch_finish(const double* acc, int nr, const int32_t* perm, int64_t n, int64_t npad,
                          double* out, int64_t ld, cudaStream_t st);
// blocks per SM the pass kernels reach at 256 threads (occupancy query)
int pass_blocks_per_sm(int phase, unsigned fset, int nr);

constexpr int kThreads = 128;
constexpr int kMinBlocks = 4;  // pass kernels: at most 128 registers per thread
constexpr int kMaxNR = 4;

}  // namespace dev
}  // namespace hh
