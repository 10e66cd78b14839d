// Device-side descriptors shared by the kernels and the C-ABI host code.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace hh {
namespace dev {

// A unit of work of a streaming pass: columns (phase 1) or rows (phase 2)
// [lo, hi) of the factor described by StreamDesc idx.
struct Item {
  int32_t kind, idx, lo, hi;
};

// One factor (or dense block) as seen by a streaming pass.  fp64 data is
// held as float2 pairs (hi, lo) in the same 8 bytes (launch_presplit_f64).
//   phase 1: columns j of f (rows x cols, column-major, ld elements) dotted
//            with in[in_off + i]; mode 0: t[toff + j*nr + r] = sum (scaled
//            units), mode 1: acc[out_off + j] += sum (dense block, A^T).
//   phase 2: acc[out_off + i] += 2^e sum_j f[i, j] t_j; mode 0: t from the
//            t arena at toff, mode 1: t_j = in[in_off + j] (dense block, A).
struct StreamDesc {
  const uint8_t* f;
  int64_t ld;
  int32_t rows, cols;
  int32_t fmt, e;
  int32_t in_off, out_off;
  int64_t toff;
  int32_t mode, pad;
};
static_assert(sizeof(StreamDesc) == 56, "descriptor size");

struct StreamArgs {
  const StreamDesc* desc;
  const Item* items;  // {unused, desc index, lo, hi}
  int32_t n_items;
  int32_t nr;
  int64_t npad;
  const float* xs;     // [4][nr][npad] fp32 (leading half) of the input, shifted by s
  const float* xs_lo;  // [4][nr][npad] the input minus its leading half, shifted by s
  float* t32;
  float2* t64;         // t of fp64 blocks as (leading, trailing) fp32 halves
  double* acc;
  int* status;   // bit 0 bad descriptor, bit 2 a bounded wait expired, bit 4 batch kernel not cooperative
  int* counter;  // work counter of this pass (zeroed by the prep launch)
};

// host-callable launchers (kernels.cu, stream.cu); launch_prep clears acc
// (nr columns) unless it is null
cudaError_t launch_prep(const double* in, int64_t ld, int nr, const int32_t* perm, int64_t n,
                        int64_t npad, float* xs, float* xs_lo, double* acc, cudaStream_t st,
                        int* counters = nullptr);
// pdl (phase 2 only, and only directly after a phase-1 launch of the same
// sequence): programmatic dependent launch, see stream.cu
// nst: pipeline depth (stages per CTA) of one-column launches, 3, 4 or 6
// (other values: 4); launches of 2 or 4 columns use 4
cudaError_t launch_stream(int phase, unsigned fset, const StreamArgs& a, int grid, cudaStream_t st,
                          bool pdl = false, int nst = 4);
int stream_blocks_per_sm(int phase, unsigned fset, int nr, int nst = 4);
int stream_rows_per_item(int fmt);   // phase-2 rows per item (1 KB of factor data per column)
int stream_cols_per_item();          // phase-1 columns per item
// kernel variants by the set of factor formats they contain (bit f = fmt f)
constexpr unsigned kSetF64 = 1u;         // fp64 factors (and dense blocks)
constexpr unsigned kSetF32 = 1u | 2u;    // fp64 + fp32
constexpr unsigned kSetAll = 31u;        // every format
unsigned pass_set_for(unsigned fmts_present);

// fp64 values at the spans {byte offset, count} (device array of 2 nspans
// int64) of base rewritten in place as float2 (fl32(v), fl32(v - fl32(v))):
// the form in which every kernel reads fp64 factors and dense blocks
cudaError_t launch_presplit_f64(uint8_t* base, const int64_t* spans, int nspans, cudaStream_t st);
// out[u + r ld] = acc[r npad + iperm[u]] (iperm: caller position -> tree position)
cudaError_t launch_finish(const double* acc, int nr, const int32_t* iperm, int64_t n, int64_t npad,
                          double* out, int64_t ld, cudaStream_t st);

constexpr int kMaxNR = 4;  // right-hand sides per launch sequence

// batches (kernels.cu): one right-hand side per matrix; matrix j's tree-order
// positions are [pofs[j], pofs[j] + npad_j) of the concatenated position space
// (np in total), its caller-order vector starts at xofs[j] of the
// concatenated input / output; perm holds each matrix's permutation at pofs[j]
cudaError_t launch_batch_prep(const double* x, const int64_t* xofs, const int32_t* perm, const int64_t* pofs,
                              const int64_t* ns, int count, int64_t np, float* xs, float* xs_lo, double* acc,
                              int* counters, cudaStream_t st);
cudaError_t launch_batch_finish(const double* acc, const int64_t* xofs, const int32_t* perm, const int64_t* pofs,
                                const int64_t* ns, int count, int64_t np, double* y, cudaStream_t st);

// A whole batch product in one persistent cooperative kernel (stream.cu):
// prep, phase 1, phase 2 and finish separated by grid-wide barriers.
struct BatchArgs {
  StreamArgs pass[2];  // phase 1, phase 2 (counters zeroed by the prep stage)
  const double* x;
  double* y;
  const int64_t* xofs;
  const int32_t* perm;
  const int64_t* pofs;
  const int64_t* ns;
  int32_t count, pad;
  int64_t np;
};
// CTAs of the persistent batch kernel that are co-resident on the device
// (sms x its occupancy); the launch must not use more
int batch_persistent_grid(unsigned fset, int sms);
cudaError_t launch_batch_persistent(unsigned fset, const BatchArgs& a, int grid, cudaStream_t st);

#ifdef __CUDACC__
// matrix j of a batch holding concatenated position q: pofs[j] <= q < pofs[j + 1]
__device__ __forceinline__ int batch_find(const int64_t* __restrict__ pofs, int count, int64_t q) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pofs[mid] <= q)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}
// d as an unevaluated fp32 pair hi + lo (hi = fl32(d) rounded to nearest
// even, lo = fl32(d - hi)) from d's bits with integer operations: the
// device's fp64 conversions and subtraction run on its low-rate fp64 units.
// Zero, subnormal, non-finite or out-of-range values (|d| below 2^-74 or
// above the fp32 range) take the fp64 conversions in a function that is not
// inlined (rare).
static __device__ __noinline__ void split_f64_rare(double d, float& hi, float& lo) {
  hi = __double2float_rn(d);
  lo = __double2float_rn(d - static_cast<double>(hi));
}
__device__ __forceinline__ void split_f64(double d, float& hi, float& lo) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  const int E = static_cast<int>((b >> 52) & 0x7ffu);
  const int e = E - 1023 + 127;  // fp32 biased exponent of hi (before rounding up)
  if (E == 0 || e < 53 || e > 253) {
    if ((b << 1) == 0) {
      hi = lo = 0.f;
      return;
    }
    split_f64_rare(d, hi, lo);
    return;
  }
  const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);  // 53-bit significand
  unsigned long long top = m >> 29;                                      // 24 bits
  const unsigned long long rem = m & ((1ull << 29) - 1);
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (top & 1ull))) top += 1;
  const int r = static_cast<int>(static_cast<long long>(m) - static_cast<long long>(top << 29));  // |r| <= 2^28
  const uint32_t sign = static_cast<uint32_t>(b >> 32) & 0x80000000u;
  const uint32_t hb = top == (1ull << 24) ? (static_cast<uint32_t>(e + 1) << 23)
                                          : ((static_cast<uint32_t>(e) << 23) | static_cast<uint32_t>(top & 0x7fffffu));
  hi = __uint_as_float(hb | sign);
  // lo = r 2^(E - 1075): the integer rounded once to fp32, then an exact
  // scaling by a normal power of two (e - 52 >= 1)
  const float lf = static_cast<float>(r) * __uint_as_float(static_cast<uint32_t>(e - 52) << 23);
  lo = sign ? -lf : lf;
}
// position p of a batch's input images: the four shifted copies of the fp32
// leading / trailing halves, and the cleared accumulator
__device__ __forceinline__ void batch_prep_position(int64_t p, const double* __restrict__ x,
                                                    const int64_t* __restrict__ xofs, const int32_t* __restrict__ perm,
                                                    const int64_t* __restrict__ pofs, const int64_t* __restrict__ ns,
                                                    int count, int64_t np, float* __restrict__ xs,
                                                    float* __restrict__ xs_lo, double* __restrict__ acc) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int64_t q = p + s;
    double v = 0.0;
    if (q < np) {
      const int j = batch_find(pofs, count, q);
      const int64_t l = q - pofs[j];
      if (l < ns[j]) v = x[xofs[j] + perm[pofs[j] + l]];
    }
    float hi, lo;
    split_f64(v, hi, lo);
    xs[static_cast<int64_t>(s) * np + p] = hi;
    xs_lo[static_cast<int64_t>(s) * np + p] = lo;
  }
  acc[p] = 0.0;
}
// v 2^e as an fp64 value built from v's bits with integer operations (exact),
// so that adding an fp32 result into an fp64 accumulator costs no instruction
// on the low-rate fp64 units.  Subnormal, non-finite or out-of-range results
// (rare) take fp64 arithmetic in a function that is not inlined, so that the
// compiler cannot predicate its fp64 instructions into the common path.
static __device__ __noinline__ double f32_to_f64_rare(float v, int e) { return ldexp(static_cast<double>(v), e); }
__device__ __forceinline__ double f32_to_f64(float v, int e) {
  const uint32_t b = __float_as_uint(v);
  if ((b & 0x7fffffffu) == 0u) return 0.0;
  const int ex = static_cast<int>((b >> 23) & 0xffu);
  const int de = ex - 127 + 1023 + e;
  if (ex == 0 || ex == 255 || de < 1 || de > 2046) return f32_to_f64_rare(v, e);
  const unsigned long long bits = (static_cast<unsigned long long>(b & 0x80000000u) << 32) |
                                  (static_cast<unsigned long long>(de) << 52) |
                                  (static_cast<unsigned long long>(b & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(bits));
}
// (S + C) 2^e as an fp64 value from the bits of the fp32 values S and C with
// 64-bit integer operations only: both significands aligned in units of
// 2^-32 of the larger one's exponent, added, normalised to 53 bits
// (truncating below 2^-52 of the sum) and packed.  Returns false, leaving
// out untouched, for zero, subnormal or non-finite inputs and out-of-range
// results; the caller handles those (rare) with pair_to_f64_rare outside its
// hot loop, so that no fp64 instruction is predicated into it.
__device__ __forceinline__ bool pair_to_f64_fast(float S, float C, int e, double& out) {
  if (fabsf(C) > fabsf(S)) {
    const float t = S;
    S = C;
    C = t;
  }
  const uint32_t bs = __float_as_uint(S), bc = __float_as_uint(C);
  if ((bs & 0x7fffffffu) == 0u) {  // both zero
    out = 0.0;
    return true;
  }
  const int es = static_cast<int>((bs >> 23) & 0xffu), ec = static_cast<int>((bc >> 23) & 0xffu);
  long long ms = static_cast<long long>((bs & 0x7fffffu) | 0x800000u);
  long long mc = static_cast<long long>((bc & 0x7fffffu) | 0x800000u);
  if (bs >> 31) ms = -ms;
  if (bc >> 31) mc = -mc;
  if (ec == 0) mc = 0;  // C zero (or subnormal: below 2^-126, dropped only if S is normal)
  const int d = es - ec;
  const long long sum = ms * (1LL << 32) + (d <= 32 ? mc * (1LL << (32 - d)) : (d < 56 ? (mc >> (d - 32)) : 0LL));
  const unsigned long long sign = sum < 0 ? 1ull : 0ull;
  const unsigned long long mag = static_cast<unsigned long long>(sum < 0 ? -sum : sum);
  const int sh = 11 - __clzll(static_cast<long long>(mag));
  const unsigned long long mant = sh >= 0 ? (mag >> sh) : (mag << -sh);
  const int de = es - 130 + sh + 1023 + e;
  out = __longlong_as_double(
      static_cast<long long>((sign << 63) | (static_cast<unsigned long long>(de) << 52) | (mant & 0xfffffffffffffull)));
  return es != 0 && es != 255 && ec != 255 && mag != 0 && de >= 1 && de <= 2046;
}
static __device__ __noinline__ double pair_to_f64_rare(float S, float C, int e) {
  return ldexp(static_cast<double>(S) + static_cast<double>(C), e);
}
// position p of a batch's output: y in each matrix's caller order
__device__ __forceinline__ void batch_finish_position(int64_t p, const double* __restrict__ acc,
                                                      const int64_t* __restrict__ xofs,
                                                      const int32_t* __restrict__ perm,
                                                      const int64_t* __restrict__ pofs,
                                                      const int64_t* __restrict__ ns, int count,
                                                      double* __restrict__ y) {
  const int j = batch_find(pofs, count, p);
  const int64_t l = p - pofs[j];
  if (l < ns[j]) y[xofs[j] + perm[pofs[j] + l]] = acc[p];
}
#endif

// ---- vector kernels of the conjugate-gradient solver (kernels.cu) ----
constexpr int kDotBlocks = 256;  // a dot product writes kDotBlocks partial sums
cudaError_t launch_dot(const double* a, const double* b, int64_t n, double* partials, cudaStream_t st);
cudaError_t launch_shift(double* q, const double* p, double shift, int64_t n, cudaStream_t st);  // q += shift p
// scalars of one conjugate-gradient solve, kept on the device
struct CgState {
  double rr, alpha, beta, threshold;  // threshold: rtol ||b||
  double done, breakdown, iters, max_iter, active;
};
cudaError_t launch_cg_step(double* x, double* r, const double* p, const double* q, const CgState* s, int64_t n,
                           cudaStream_t st);  // x += alpha p, r -= alpha q (active iterations)
cudaError_t launch_cg_dir(double* p, const double* r, const CgState* s, int64_t n, cudaStream_t st);  // p = r + beta p
cudaError_t launch_cg_alpha(const double* partials, CgState* s, cudaStream_t st);  // alpha = rr / (p . q)
cudaError_t launch_cg_beta(const double* partials, CgState* s, cudaStream_t st);   // rr, beta, convergence

// ---- tensor-core path for many right-hand sides (tc.cu) ----
// A piece: ranks [r0, r0 + k) of one low-rank block stored in fp32, fp16, bf16
// or e4m3.  f1 / f2 point at the piece's first rank column of the phase-1
// factor (V forward, U transpose) and the phase-2 factor; rows1 / rows2 are
// the sizes of the input / output clusters, which start at tree positions
// in_off / out_off (both multiples of 16).
struct TcPiece {
  const uint8_t* f1;
  const uint8_t* f2;
  int64_t ld1, ld2;
  int64_t toff;        // byte offset of the piece's T image: [k-step][slice][128 rows x 32 B]
  int32_t rows1, rows2;
  int32_t in_off, out_off;
  int32_t k, kp;       // ranks, ranks rounded up to 16
  int32_t fmt, e;      // storage format, exp_u + exp_v
  int32_t col;         // operand row / accumulator column of the piece in its phase-1 group
  int32_t pad;
};
// phase-1 item: positions [p0, p1) of the input cluster [in_off, in_off + rows)
// for the pieces [first, first + count) of one format (nk = sum of their kp,
// at most kTcGroupRanks).  img: byte offset of the group's packed operand
// panel, [16-position block][slice][nk rows x 32 B] (all items of a group
// share it).  A group whose cluster is longer than the split length is split
// into nsplit items; each writes its partial sums to part + poff (fp32
// [128][nk]), and for each quarter of the right-hand sides the last item to
// finish (counter cnt[4 gid + quarter]) adds them in split order and writes
// the T images.
struct TcGroup {
  int32_t first, count, nk, fmt;
  int32_t in_off, rows, p0, p1;
  int32_t nsplit, split, gid, pad;
  int64_t poff;
  int64_t img;
};
// phase-2 item: output rows [row0, row0 + rows) (row0 a multiple of kTcRows)
// and entries [first, first + count); tensor-core path: nst stages of up to
// kTcKSteps K steps, accumulators drained every `chunk` stages
struct TcTile {
  int32_t row0, rows, first, count;
  int32_t nst, chunk;
};
// rows [src, src + nrows) of a piece's output cluster land on tile rows
// [dst, dst + nrows).  Tensor-core path: img, byte offset of the entry's
// packed operand panel [k-step][slice][128 tile rows x 32 B]; toff, nks, fmt:
// the piece's T image offset, K steps and format (so that a stage needs no
// second lookup)
struct TcEntry {
  int32_t piece, src, dst, nrows;
  int64_t img;
  int64_t toff;
  int32_t nks, fmt;
};
struct TcArgs {
  const TcPiece* pieces;
  const TcGroup* groups;
  const TcTile* tiles;
  const TcEntry* entries;
  int32_t n_groups, n_tiles;
  int32_t nr, rp;        // right-hand sides of this launch (<= 128), nr rounded up to 16
  const uint8_t* ximg;   // input image [nblk][3 slices][128 rows x 32 B] (tc prep)
  int64_t nblk;
  const uint8_t* img;    // packed factor panels (groups, then entries)
  uint8_t* timg;         // T images of the pieces
  float* part;           // partial sums of split groups
  int* cnt;              // arrival counters of split groups (cleared by the prep launch)
  int32_t n_cnt, pad;
  int* work;             // work counters of phase 1 and phase 2 (cleared by the prep launch)
  double* acc;           // output accumulator [nr][npad], tree order
  int64_t npad;
  int* status;           // bit 3: a bounded wait expired
};
constexpr int kTcMaxRhs = 128;          // right-hand sides per tensor-core launch sequence
constexpr int kTcRows = 128;            // phase-2 tile rows
constexpr int kTcGroupRanks = 128;      // ranks of one phase-1 group
constexpr int kTcSplitPositions = 8192; // positions of one phase-1 item (default)
constexpr int kTcKSteps = 2;            // K steps (16 positions or ranks) per pipeline stage
// stages whose K steps add into one tensor-memory bank before it is drained
// (fp32 pieces; the 16- and 8-bit pieces)
constexpr int kTcChunkF32 = 2;
constexpr int kTcChunk16 = 16;
// bf16 slices per element: factor panels (fp32 3, fp16 2, bf16 / e4m3 1),
// input and T images (fp32 pieces 3, the others 2)
inline __host__ __device__ int tc_factor_slices(int fmt) { return fmt == 1 ? 3 : (fmt == 2 ? 2 : 1); }
inline __host__ __device__ int tc_input_slices(int fmt) { return fmt == 1 ? 3 : 2; }
// input images of the many-column sequence (both the tensor-core image and
// the fp32 halves [npos][128] of mr.cu, npos <= 16 nblk) and the clearing of
// acc, cnt and t32; xt: scratch [nr][npad] fp64 for the tree-ordered input
cudaError_t launch_tc_prep(const double* x, int64_t ld, int nr, const int32_t* perm, int64_t n, int64_t nblk,
                           uint8_t* ximg, double* acc, int64_t npad, int* cnt, int n_cnt, float* xh, float* xl,
                           int64_t npos, float* t32, int64_t t_floats, double* xt, cudaStream_t st);
// packs the factor panels of a set's groups (phase 1) and entries (phase 2) into img
cudaError_t launch_tc_pack(const TcPiece* pieces, const TcGroup* groups, int n_groups, const TcEntry* entries,
                           int n_entries, uint8_t* img, cudaStream_t st);
// phase 1 or 2 over every group / tile; grid: persistent CTAs (<= SMs)
cudaError_t launch_tc(int phase, const TcArgs& a, int grid, cudaStream_t st);

// ---- dense blocks for many right-hand sides on the tensor cores (dense_tc.cu) ----
// One dense block's share of a 128-row output tile, over at most
// kTdMaxK contracted positions.  Forward: A[m][k] = H[src + m - dst][k0 + k];
// transposed: A[m][k] = H[k0 + k][src + m - dst]; H is column-major with
// leading dimension ld, held as fp32 pairs (hi, lo) of its value times 2^-e.
struct TdEntry {
  const float2* d;
  int64_t ld;
  int64_t img;          // byte offset of the packed digit panel [k-step][6 digits][128 rows x 32 B]
  int64_t xoff;         // byte offset of the input's digit panel [pass][k-step][6 digits][64 rows x 32 B]
  int32_t src, dst, nrows;
  int32_t in_off;       // tree position of contracted position k0
  int32_t k0, kc;       // contracted positions k0 .. k0 + kc - 1 (kc <= kTdMaxK)
  int32_t e, trans;
  int32_t first;        // 1: no earlier entry of the tile covers these rows (store, not add)
  int32_t pad;
};
struct TdArgs {
  const TcTile* tiles;      // row0, rows, first, count (entries [first, first + count))
  const TdEntry* entries;
  int32_t n_tiles, nr;      // tiles; right-hand sides of this launch (<= 128)
  const uint8_t* img;       // packed digit panels of H
  const int32_t* rexp;      // [entry][128]: power of two of tile row m's digits
  const float* xh;          // input, tree order, fp32 leading halves [npos][128] (td_prep)
  const float* xl;          // trailing halves
  uint8_t* xdig;            // the input's digit panels (written by td_prep, read by td_kernel)
  int32_t* bexp;            // [entry][128]: b_r - 7 of right-hand side r's digits
  double* acc;              // output accumulator [nr][npad], tree order, all zero before
                            // the launch (the first entry over a row stores into it)
  int64_t npad;
  int* status;              // bit 3: a bounded wait expired
};
constexpr int kTdMaxK = 128;       // contracted positions of one entry
constexpr int kTdDigits = 6;       // digits per value (8 bits each)
constexpr int64_t kTdStepBytes = int64_t(kTdDigits) * 4096;  // one k-step of an H digit panel
constexpr int64_t kTdXStepBytes = int64_t(kTdDigits) * 2048; // one k-step of an input digit panel (64 columns)
// digit panels of the entries [0, n) (one CTA per entry) and their row exponents
cudaError_t launch_td_pack(const TdEntry* entries, int n, uint8_t* img, int32_t* rexp, cudaStream_t st);
// the input's digit panels and column exponents of every entry (n_entries CTAs)
cudaError_t launch_td_prep(const TdArgs& a, int n_entries, cudaStream_t st);
// Y += H X over every tile; grid: persistent CTAs (<= SMs)
cudaError_t launch_td(const TdArgs& a, int grid, cudaStream_t st);

// ---- CUDA-core products for many right-hand sides (mr.cu) ----
// Work lists in the tensor-core structures: phase-1 groups of at most
// kMrRanks ranks (pieces with kp = ranks rounded up to 4, T at toff floats,
// [rank][128]); phase-2 tiles of kMrRows rows.
struct MrArgs {
  const TcPiece* pieces;
  const TcGroup* groups;
  const TcTile* tiles;
  const TcEntry* entries;
  int32_t n_groups, n_tiles;
  int32_t nr, rp;       // right-hand sides (<= 128); nr rounded up to 32, 64 or 128
  const float* xh;      // input, tree order, fp32 leading halves [npos][128]
  const float* xl;      // trailing halves
  float* t32;           // T of the pieces
  double* acc;          // output accumulator [nr][npad], tree order
  int64_t npad;
  int* status;
};
constexpr int kMrRanks = 64;
constexpr int kMrRows = 128;
// kind 1: phase 1, 2: phase 2
cudaError_t launch_mr(int kind, const MrArgs& a, cudaStream_t st);

}  // namespace dev
}  // namespace hh
