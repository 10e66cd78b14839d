// Dense diagonal blocks of the H_h product for many right-hand sides on the
// tensor cores, at the working precision of the fp64 path.  Algorithm 4's
// dense term Y_I += H_IJ X_J (Section 4.4; its transpose for the backward
// product) is a small dense contraction per leaf cluster: 128 output rows,
// up to 128 contracted positions, R right-hand sides.
//
// Digits.  A value v with |v| < 2^a is written as
//     v = 2^(a-7) (d_0 + 2^-8 d_1 + ... + 2^-40 d_5) + r,   |r| <= 2^(a-48),
// every digit an integer with |d_s| <= 128, found by rounding to nearest
// and carrying the exact remainder as an fp32 pair.  Integers of at most 8
// significant bits, and d_s 2^-8s, are exactly bf16 numbers.  H's digits use
// one exponent per output row (its largest magnitude in the block), X's one
// exponent per right-hand side (its largest magnitude over the contracted
// positions), so that
//     (H X)[m][r] ~= 2^(a_m + b_r) sum_g sum_{s+t=g} sum_k (2^-8s d_s[m][k]) (2^-8t c_t[k][r]).
// Every product of two digits is exact in fp32.  The sum of diagonal g
// (s + t = g) is an integer multiple of 2^-8g below 4 * 128 * 2^14 = 2^23 of
// those units for g <= 3, so the tensor core's fp32 accumulation of each of
// D_0, D_1, D_2, D_3 is exact whatever order and rounding it uses;
// diagonals 4 and 5 share a fifth accumulator, whose fp32 roundings stay
// below about 2^-46 of the largest possible D_0.  Diagonals 6 and above are dropped (below 2^-45 of
// sum |H||X|), so with the digit remainders the product is exact to about
// 2^-45 of sum_k |H[m][k]| |X[k][r]| -- the fp64 path's accuracy, with no
// instruction on the device's low-rate fp64 units except the final
// addition into the fp64 output.
//
// Kernels.  td_prep (one CTA per entry, every launch) takes each right-hand
// side's exponent over the entry's contracted positions and writes X's
// digits in the operand layout; the H digits are packed once per matrix and
// direction (td_pack).  td_kernel is persistent and warp-specialized, one
// CTA per SM (320 threads):
//   warp 0      lane 0 copies both digit panels into a 3-deep ring of stages
//               of two k-steps (16 positions each), with bulk copies;
//   warp 1      lane 0 issues 21 MMAs per k-step (M = 128 rows, N = up to
//               64 right-hand sides, K = 16) into five tensor-memory
//               accumulators of N columns;
//   warps 2-9   drain the accumulators (tensor-memory lane quarter w mod 4,
//               half of each pass's columns per warp):
//               D_0 + ... + D_45 as an fp32 pair by two-sums, turned into
//               one fp64 value of (S + C) 2^(a_m + b_r) with integer
//               operations (this device's fp64 units are far too slow for
//               one instruction per output), stored into the accumulator.
// The dense blocks run first in a product, on the cleared accumulator: the
// first entry over a row stores its result, a later one (a cluster longer
// than kTdMaxK, or a second dense block on the same rows) loads and adds.
// A unit of work is (entry, pass of at most 64 right-hand sides).  Every
// mbarrier wait has a clock limit; an expired wait sets an abort flag that
// the other roles see and bit 3 of the status word, and the CTA ends after
// its copies and MMAs have completed and its tensor memory has been
// released.
#include <cuda_bf16.h>

#include "hh_device.h"

namespace hh {
namespace dev {

namespace {

constexpr long long kWaitCycles = 4000000000LL;
constexpr int kThreads = 320;
constexpr int kDrainWarps = 8;  // two per tensor-memory lane quarter, half the columns each
constexpr int kDepth = 3;
constexpr int kKS = 2;                           // k-steps per stage
constexpr int kPass = 64;                        // right-hand sides per pass
constexpr int kABytes = kKS * kTdDigits * 4096;  // H digits: [k-step][digit][128 rows x 32 B]
constexpr int kBStep = kTdXStepBytes;            // X digits of one k-step: [digit][64 rows x 32 B]
constexpr int kBBytes = kKS * kBStep;
constexpr int kStage = kABytes + kBBytes;
constexpr int kAcc = 5;                          // accumulators D_0, D_1, D_2, D_3, D_45
constexpr uint32_t kTmemCols = 512;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major operand without swizzling: 8-row x 16-byte core matrices, the two
// of one k-step 128 bytes apart, successive 8-row groups 256 bytes apart
__device__ __forceinline__ uint64_t op_desc(uint32_t a) {
  uint64_t d = static_cast<uint64_t>((a >> 4) & 0x3fff);
  d |= static_cast<uint64_t>(128 >> 4) << 16;
  d |= static_cast<uint64_t>(256 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}
// byte offset of (row, 8-element half c of the k-step) in a K-major operand tile
__device__ __forceinline__ int core_off(int row, int c) { return (row >> 3) * 256 + c * 128 + (row & 7) * 16; }

// D fp32, A and B bf16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) | (8u << 24);
}
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// exponent a with |v| < 2^a for the largest magnitude m (m >= 0); -200 for 0
__device__ __forceinline__ int exp_above(float m) {
  if (!(m > 0.f)) return -200;
  int a;
  frexpf(m, &a);  // m = f 2^a, f in [1/2, 1)
  return a;
}

// The six digits of (vh + vl) 2^sc (|.| <= 128 + 2^-16) as bf16 values
// d_s 2^-8s.  The scaling is two exact multiplies by powers of two (f1 f2 =
// 2^sc).  The remainder is carried as an fp32 pair (h, l) with |l| at most
// half an ulp of the leading value: h - d is exact, so a fast two-sum
// renormalises the pair before each digit, and the scalings by 256 are
// exact.
__device__ __forceinline__ void digits6(float vh, float vl, float f1, float f2, float* dig) {
  float h = (vh * f1) * f2, l = (vl * f1) * f2;
#pragma unroll
  for (int s = 0; s < kTdDigits; ++s) {
    const float t = h + l;
    l = l - (t - h);
    h = t;
    const float d = rintf(h);
    dig[s] = d * __int_as_float((127 - 8 * s) << 23);
    h = (h - d) * 256.f;
    l *= 256.f;
  }
}

// eight values -> their six digit vectors (16 bytes each) at dst + s * stride
__device__ __forceinline__ void store_digits8(const float* vh, const float* vl, int sc, uint8_t* dst, int stride) {
  sc = max(-250, min(250, sc));
  const int e1 = sc / 2;
  const float f1 = __int_as_float((127 + e1) << 23), f2 = __int_as_float((127 + sc - e1) << 23);
  __align__(16) __nv_bfloat16 out[kTdDigits][8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    float dig[kTdDigits];
    digits6(vh[t], vl[t], f1, f2, dig);
#pragma unroll
    for (int s = 0; s < kTdDigits; ++s) out[s][t] = __float2bfloat16_rn(dig[s]);
  }
#pragma unroll
  for (int s = 0; s < kTdDigits; ++s)
    *reinterpret_cast<uint4*>(dst + s * stride) = *reinterpret_cast<const uint4*>(out[s]);
}

// k-th item of this CTA: rounds of gridDim.x items, dealt forwards in even
// rounds and backwards in odd ones; -1 when the list is exhausted
__device__ __forceinline__ int item_of(int k, int n_items) {
  const int g = gridDim.x, c = (k & 1) ? g - 1 - static_cast<int>(blockIdx.x) : static_cast<int>(blockIdx.x);
  const long long i = static_cast<long long>(k) * g + c;
  return i < n_items ? static_cast<int>(i) : -1;
}

struct Ctl {
  uint64_t full[kDepth], empty[kDepth];
  uint64_t dfull, dempty;  // accumulators ready for the drain / released by it
  uint32_t tmem;
  int abort;
};

// bounded wait that also gives up when another role set the abort flag
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  uint32_t ok;
  auto probe = [&]() {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
  };
  if (probe()) return true;
  const long long t0 = clock64();
  for (int n = 1;; ++n) {
    if (probe()) return true;
    if ((n & 63) == 0 && *abort) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort = 1;
      return false;
    }
  }
}

// the same walk for every role: units (tile item k, entry e, pass p)
struct Walk {
  int k, it, e, p, passes;
  TcTile tl;
  __device__ bool next_tile(const TdArgs& a) {
    e = 0;
    p = 0;
    for (;;) {
      it = item_of(++k, a.n_tiles);
      if (it < 0) return false;
      tl = a.tiles[it];
      if (tl.count > 0) return true;
    }
  }
  __device__ bool start(const TdArgs& a) {
    k = -1;
    passes = (a.nr + kPass - 1) / kPass;
    return next_tile(a);
  }
  __device__ bool next(const TdArgs& a) {
    if (++p < passes) return true;
    p = 0;
    if (++e < tl.count) return true;
    return next_tile(a);
  }
  __device__ int ncols(const TdArgs& a) const { return min(kPass, a.nr - kPass * p); }
};

__global__ void __launch_bounds__(kThreads, 1) td_kernel(TdArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  Ctl* c = reinterpret_cast<Ctl*>(base + kDepth * kStage);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kDepth; ++s) {
      mbar_init(&c->full[s], 1);
      mbar_init(&c->empty[s], 1);
    }
    mbar_init(&c->dfull, 1);
    mbar_init(&c->dempty, kDrainWarps);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    c->abort = 0;
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&c->tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  volatile int* abort = &c->abort;
  int produced = 0, mmas = 0;

  if (w == 0) {  // producer: H digit panels and this pass's X digit panel
    if (lane == 0) {
      Walk wk;
      int gs = 0;
      bool ok = wk.start(a);
      while (ok) {
        const TdEntry en = a.entries[wk.tl.first + wk.e];
        const int nks = (en.kc + 15) >> 4;
        const uint8_t* xp = a.xdig + en.xoff + static_cast<int64_t>(wk.p) * nks * kBStep;
        for (int i = 0; i < nks && ok; i += kKS, ++gs) {
          const int s = gs % kDepth, nb = min(kKS, nks - i);
          if (gs >= kDepth && !ws_wait(&c->empty[s], ((gs / kDepth) - 1) & 1, abort)) {
            ok = false;
            break;
          }
          uint8_t* st = base + s * kStage;
          const uint32_t abytes = static_cast<uint32_t>(nb * kTdStepBytes), bbytes = static_cast<uint32_t>(nb * kBStep);
          mbar_expect_tx(&c->full[s], abytes + bbytes);
          bulk_copy(st, a.img + en.img + static_cast<int64_t>(i) * kTdStepBytes, abytes, &c->full[s]);
          bulk_copy(st + kABytes, xp + static_cast<int64_t>(i) * kBStep, bbytes, &c->full[s]);
          produced = gs + 1;
        }
        if (ok) ok = wk.next(a);
      }
    }
  } else if (w == 1) {  // MMA issuer
    if (lane == 0) {
      Walk wk;
      int gs = 0, u = 0;
      bool ok = wk.start(a);
      const uint32_t sbase = saddr(base);
      while (ok) {
        const TdEntry en = a.entries[wk.tl.first + wk.e];
        const int nks = (en.kc + 15) >> 4, n = (wk.ncols(a) + 15) & ~15;
        const uint32_t idesc = idesc_bf16(n);
        if (u > 0 && !ws_wait(&c->dempty, (u - 1) & 1, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int i = 0; i < nks && ok; i += kKS, ++gs) {
          const int s = gs % kDepth, nb = min(kKS, nks - i);
          if (!ws_wait(&c->full[s], (gs / kDepth) & 1, abort)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = sbase + s * kStage, sb = sa + kABytes;
          for (int t = 0; t < nb; ++t) {
            const bool first = (i + t) == 0;
#pragma unroll
            for (int g = 0; g < 6; ++g) {
              const int acc_i = g < 4 ? g : 4;
#pragma unroll
              for (int sd = 0; sd <= g; ++sd) {
                const uint64_t da = op_desc(sa + t * kTdStepBytes + sd * 4096);
                const uint64_t db = op_desc(sb + t * kBStep + (g - sd) * 2048);
                // the first product into an accumulator in this unit starts it
                const bool fresh = first && sd == 0 && g <= 4;
                mma(c->tmem + static_cast<uint32_t>(acc_i * kPass), da, db, idesc, fresh ? 0u : 1u);
              }
            }
          }
          mma_commit(&c->empty[s]);
          mmas = gs + 1;
        }
        if (!ok) break;
        mma_commit(&c->dfull);
        ++u;
        ok = wk.next(a);
      }
    }
  } else {  // drain: tile row m of this lane, columns of half hh of each pass
    const int q = w & 3, hh = (w - 2) >> 2, m = 32 * q + lane;
    Walk wk;
    int u = 0;
    bool ok = wk.start(a);
    while (ok) {
      const int ei = wk.tl.first + wk.e;
      const TdEntry en = a.entries[ei];
      const int ncol = wk.ncols(a);
      const int am = a.rexp[static_cast<int64_t>(ei) * 128 + m];
      // b_r - 7 of this warp's columns 32 hh + lane, shared by shuffles
      const int bl = a.bexp[static_cast<int64_t>(ei) * 128 + kPass * wk.p + 32 * hh + lane];
      const bool row_in = m >= en.dst && m < en.dst + en.nrows && m < wk.tl.rows;
      if (!ws_wait(&c->dfull, u & 1, abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tb = c->tmem + (static_cast<uint32_t>(32 * q) << 16);
      // both chunks of this warp's 32 columns out of tensor memory, each
      // reduced at once to S + C (two-sums from the smallest accumulator);
      // then the accumulators are released to the next unit's MMAs while
      // the conversion and the stores run
      float S[2][16], C[2][16];
#pragma unroll
      for (int ch = 0; ch < 2; ++ch) {
        const int c0 = 32 * hh + 16 * ch;
        if (c0 < ncol) {
          uint32_t v[kAcc][16];
#pragma unroll
          for (int g = 0; g < kAcc; ++g) tmem_ld16(tb + g * kPass + c0, v[g]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            S[ch][j] = __uint_as_float(v[4][j]);
            C[ch][j] = 0.f;
          }
#pragma unroll
          for (int g = 3; g >= 0; --g)
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float x = __uint_as_float(v[g][j]);
              const float s2 = x + S[ch][j];
              const float bp = s2 - x;
              C[ch][j] += (x - (s2 - bp)) + (S[ch][j] - bp);
              S[ch][j] = s2;
            }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&c->dempty);
#pragma unroll
      for (int ch = 0; ch < 2; ++ch) {
        const int c0 = 32 * hh + 16 * ch;
        if (c0 >= ncol) break;
        int sc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) sc[j] = am + __shfl_sync(0xffffffffu, bl, (c0 + j) & 31);
        if (!row_in) continue;
        // (S + C) 2^(a_m + b_r) as fp64 with integer operations; the first
        // entry over a row stores it into the cleared accumulator, a later
        // one adds it after loading the sixteen values at once
        double y[16];
        unsigned rare = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (!pair_to_f64_fast(S[ch][j], C[ch][j], sc[j], y[j])) rare |= 1u << j;
        if (rare)
          for (int j = 0; j < 16; ++j)
            if ((rare >> j) & 1u) y[j] = pair_to_f64_rare(S[ch][j], C[ch][j], sc[j]);
        double* out = a.acc + static_cast<int64_t>(kPass * wk.p + c0) * a.npad + wk.tl.row0 + m;
        if (!en.first) {
          double prev[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) prev[j] = c0 + j < ncol ? out[static_cast<int64_t>(j) * a.npad] : 0.0;
#pragma unroll
          for (int j = 0; j < 16; ++j) y[j] += prev[j];
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < ncol) out[static_cast<int64_t>(j) * a.npad] = y[j];
      }
      ++u;
      ok = wk.next(a);
    }
  }

  // teardown: on an abort the producer waits (bounded) for the copies it
  // issued and the MMA thread for its last MMAs; then tensor memory is freed
  __syncthreads();
  if (c->abort) {
    volatile int no = 0;
    if (tid == 0)
      for (int i = produced > kDepth ? produced - kDepth : 0; i < produced; ++i)
        ws_wait(&c->full[i % kDepth], (i / kDepth) & 1, &no);
    if (tid == 32 && mmas > 0) ws_wait(&c->empty[(mmas - 1) % kDepth], ((mmas - 1) / kDepth) & 1, &no);
    if (tid == 0) atomicOr(a.status, 8);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c->tmem), "r"(kTmemCols));
}

// Digit panels (one CTA per entry): the exponent of each tile row over the
// entry's contracted positions, then unit (k-step ks, half hc, tile row m)
// = digits of A[m][16 ks + 8 hc .. + 7] at img + en.img + ks * kTdStepBytes
// + s * 4096 + core_off(m, hc); rows outside the entry and positions past kc
// are zero.  rexp[entry][m] = e + a_m - 7 (A = 2^rexp sum_s 2^-8s d_s).
__global__ void td_pack_kernel(const TdEntry* __restrict__ entries, uint8_t* __restrict__ img,
                               int32_t* __restrict__ rexp) {
  __shared__ float part[2][128];
  __shared__ int sc[128];
  const int ei = blockIdx.x, tid = threadIdx.x;
  const TdEntry en = entries[ei];
  auto at = [&](int m, int k) -> float2 {
    const int64_t row = en.src + (m - en.dst);
    return en.trans ? en.d[row * en.ld + en.k0 + k] : en.d[static_cast<int64_t>(en.k0 + k) * en.ld + row];
  };
  auto in_rows = [&](int m) { return m >= en.dst && m < en.dst + en.nrows; };
  {
    const int m = tid & 127, half = tid >> 7;
    float mx = 0.f;
    if (in_rows(m))
      for (int k = half; k < en.kc; k += 2) mx = fmaxf(mx, fabsf(at(m, k).x));
    part[half][m] = mx;
  }
  __syncthreads();
  if (tid < 128) {
    const int am = exp_above(fmaxf(part[0][tid], part[1][tid]));
    sc[tid] = 7 - am;
    rexp[static_cast<int64_t>(ei) * 128 + tid] = en.e + am - 7;
  }
  __syncthreads();
  const int nks = (en.kc + 15) >> 4;
  for (int u = tid; u < nks * 256; u += blockDim.x) {
    const int m = u & 127, hc = (u >> 7) & 1, ks = u >> 8;
    float vh[8], vl[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = 16 * ks + 8 * hc + t;
      vh[t] = vl[t] = 0.f;
      if (in_rows(m) && k < en.kc) {
        const float2 v = at(m, k);
        vh[t] = v.x;
        vl[t] = v.y;
      }
    }
    store_digits8(vh, vl, sc[m], img + en.img + ks * kTdStepBytes + core_off(m, hc), 4096);
  }
}

// The input's digit panels (one CTA per entry, every launch): the exponent
// of each right-hand side over the entry's contracted positions, then unit
// (pass p, k-step ks, half hc, column rl of the pass) = digits of
// X[16 ks + 8 hc .. + 7][64 p + rl] at xdig + en.xoff + (p nks + ks) *
// kTdXStepBytes + s * 2048 + core_off(rl, hc); positions past kc are zero.
// bexp[entry][r] = b_r - 7 (X = 2^bexp sum_t 2^-8t c_t).
__global__ void td_prep_kernel(TdArgs a) {
  __shared__ float part[2][128];
  __shared__ int sc[128];
  const int ei = blockIdx.x, tid = threadIdx.x;
  const TdEntry en = a.entries[ei];
  {
    const int r = tid & 127, half = tid >> 7;
    float mx = 0.f;
    for (int k = half; k < en.kc; k += 2) mx = fmaxf(mx, fabsf(a.xh[static_cast<int64_t>(en.in_off + k) * 128 + r]));
    part[half][r] = mx;
  }
  __syncthreads();
  if (tid < 128) {
    const int b = exp_above(fmaxf(part[0][tid], part[1][tid]));
    sc[tid] = 7 - b;
    a.bexp[static_cast<int64_t>(ei) * 128 + tid] = b - 7;
  }
  __syncthreads();
  const int nks = (en.kc + 15) >> 4, passes = (a.nr + kPass - 1) / kPass;
  for (int u = tid; u < passes * nks * 128; u += blockDim.x) {
    const int rl = u & 63, hc = (u >> 6) & 1, rest = u >> 7, ks = rest % nks, p = rest / nks, r = kPass * p + rl;
    float vh[8], vl[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = 16 * ks + 8 * hc + t;
      vh[t] = vl[t] = 0.f;
      if (k < en.kc) {
        const int64_t o = static_cast<int64_t>(en.in_off + k) * 128 + r;
        vh[t] = a.xh[o];
        vl[t] = a.xl[o];
      }
    }
    store_digits8(vh, vl, sc[r], a.xdig + en.xoff + static_cast<int64_t>(p * nks + ks) * kBStep + core_off(rl, hc),
                  2048);
  }
}

}  // namespace

cudaError_t launch_td_prep(const TdArgs& a, int n_entries, cudaStream_t st) {
  if (n_entries <= 0) return cudaSuccess;
  if (a.nr < 1 || a.nr > kTcMaxRhs) return cudaErrorInvalidValue;
  td_prep_kernel<<<n_entries, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_td_pack(const TdEntry* entries, int n, uint8_t* img, int32_t* rexp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  td_pack_kernel<<<n, 256, 0, st>>>(entries, img, rexp);
  return cudaGetLastError();
}

cudaError_t launch_td(const TdArgs& a, int grid, cudaStream_t st) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (a.nr < 1 || a.nr > kTcMaxRhs) return cudaErrorInvalidValue;
  if (grid > a.n_tiles) grid = a.n_tiles;
  if (grid < 1) grid = 1;
  const size_t smem = kDepth * kStage + 128 + sizeof(Ctl);
  cudaError_t e = cudaFuncSetAttribute(td_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  td_kernel<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace hh
