// Host-side representation of a built H_h matrix and the builder entry
// points shared by the C-ABI translation units.  Plain C++17, no CUDA.
#pragma once

#include <cstddef>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

namespace hh {

// file could not be opened, read or written
struct IoError : std::runtime_error {
  explicit IoError(const std::string& s) : std::runtime_error(s) {}
};

enum Fmt : int { F64 = 0, F32 = 1, F16 = 2, BF16 = 3, E4M3 = 4, NFMT = 5 };
enum Kind : int { KIND_STD = 0, KIND_FINER = 1, KIND_WEAK = 2, KIND_NBR = 3 };

int fmt_bytes(int fmt);
int fmt_bits(int fmt);
double unit_roundoff(int fmt);

// One admissible block: U (m x k) and V (n x k), column-major, stored in
// `fmt` inside the arena at byte offsets u_off / v_off with leading
// dimensions ldu / ldv (elements).  Decoded value = stored * 2^exp.
struct LRBlock {
  int32_t level, kind, i, j;
  int64_t row_off, m, col_off, n;
  int32_t k, fmt, exp_u, exp_v;
  int64_t u_off, v_off, ldu, ldv;
  double norm;  // ||H~_b||_F
};
static_assert(sizeof(LRBlock) == 104, "LRBlock layout is part of the file format");

// One dense block (fp64, column-major, ld = m) at element offset d_off.
struct DenseBlock {
  int32_t level, i, j, pad;
  int64_t row_off, m, col_off, n, d_off;
};
static_assert(sizeof(DenseBlock) == 56, "DenseBlock layout is part of the file format");

struct HostMatrix {
  int64_t n = 0;
  // L, ell and block levels are binary levels; step = binary levels per tree
  // level (1: binary KD tree, dim: the 2^d-tree held as a binary tree)
  int32_t dim = 0, L = 0, ell = 0, leaf = 0, kernel = 0, step = 1;
  double eta = 0, tol = 0, kparam = 1, norm_ht = 0;
  uint32_t fmt_mask = 1;
  uint64_t seed = 0;
  double build_seconds = 0;
  int32_t build_device = -1;       // GPU that compressed the blocks (-1: the host)
  int64_t build_fallback = 0;      // blocks the host compressed in a device build
  double build_device_seconds = 0; // wall time of the device compression
  std::vector<double> points;        // n x dim, user order
  std::vector<int32_t> perm;         // perm[p] = user index at tree position p
  std::vector<int64_t> node_off, node_size;
  std::vector<double> node_lo, node_hi;  // n_nodes x dim
  std::vector<LRBlock> lr;
  std::vector<DenseBlock> dense;
  std::vector<uint8_t> arena;        // factor storage
  std::vector<double> dense_data;    // dense blocks
};

struct BuildParams {
  int kernel;
  double kparam;
  int leaf;
  double eta;
  int ell;  // -1 -> floor(L/2)
  double tol;
  uint32_t fmt_mask;
  uint64_t seed;
  int threads;  // <= 0: hardware concurrency
  int tree;     // 0: binary KD bisection; 1: balanced 2^d-tree (ell in its levels)
  int device = -1;  // >= 0: LRcompression of the admissible blocks on this GPU (construct.cu)
};

// Algorithm 1 + 5 + 3: throws std::runtime_error / std::invalid_argument.
void build(const double* points, int64_t n, int dim, const BuildParams& p, HostMatrix& out);

// Algorithm 3 applied again to a uniform-fp64 matrix with another set of
// formats (same compression, tree and partition; requires ell < L).
void reencode(const HostMatrix& src, uint32_t fmt_mask, int threads, HostMatrix& out);

// Serialized file (layout documented in include/hh.h's companion, hhio.cpp).
void save_file(const HostMatrix& h, const std::string& path);
void load_file(const std::string& path, HostMatrix& h);
// Validate offsets, sizes and alignment of a matrix (throws on violation).
void validate(const HostMatrix& h);

// Algorithm 2: the switching level with the largest storage gain
// S_1(ell) - S_2(ell) = S_s - S_h(ell) over the H_s matrix (ell = L), walking
// up from the leaves while the gain grows.  Returns ell*; gains[l] holds the
// gain of every level evaluated (NaN elsewhere), sized L + 1; depth = L.
int optimal_switch_level(const double* points, int64_t n, int dim, const BuildParams& p, std::vector<double>& gains,
                         int& depth);

// Several GPUs (shard.cpp): contiguous ranges of tree positions, one per
// rank, balanced by the factor and dense bytes of their block rows
// (bounds[0] = 0 <= ... <= bounds[nranks] = n); and the matrix of the block
// rows [p0, p1): blocks cut to those rows, points in tree order, identity
// permutation (its vectors are in tree order).
void shard_plan(const HostMatrix& h, int nranks, std::vector<int64_t>& bounds);
void make_shard(const HostMatrix& src, int64_t p0, int64_t p1, HostMatrix& out);

// Derived quantities for hh_info.
struct Summary {
  int64_t blocks_per_fmt[NFMT] = {0, 0, 0, 0, 0};
  int64_t bytes_per_fmt[NFMT] = {0, 0, 0, 0, 0};
  int64_t dense_bytes = 0, max_rank = 0, u_bytes = 0, v_bytes = 0;
  double storage_amp = 0, storage_fp64 = 0, bytes_per_matvec = 0, flops_per_matvec = 0;
  std::vector<int32_t> csp;
  double bound42 = 0, bound44 = 0, bound_round = 0;
};
Summary summarize(const HostMatrix& h);

}  // namespace hh
