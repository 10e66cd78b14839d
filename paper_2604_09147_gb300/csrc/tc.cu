// Tensor-core path (tcgen05, kind::f16 with bf16 operands) of the H_h product
// for many right-hand sides, for the low-rank blocks stored in fp32, fp16,
// bf16 or fp8-e4m3 whose clusters start at multiples of 16.  With R right-hand
// sides the two phases of Algorithm 4 become dense contractions,
//   phase 1  T_b = 2^(e_u+e_v) V_b^T X_J          (k_b x R, contraction over |J|)
//   phase 2  Y_I += U_b T_b                        (|I| x R, contraction over k_b)
// computed as
//   phase 1  items are (group, position range): a group is the blocks of one
//            format sharing the input cluster J (at most 128 ranks);
//            D[r][col] = sum_p X[p][r] V[p][col], M = 128 right-hand sides,
//            N = the group's ranks, K = 16 positions per MMA.  Long clusters
//            are split over several items; each writes its partial sums, and
//            per quarter of the right-hand sides the warp that arrives last
//            (an atomic counter, nothing waits) adds them in split order.
//   phase 2  items are 128-row output tiles: D[row][r] = sum over the blocks
//            covering the tile and their ranks of U[row][j] T[j][r], N = R,
//            added once into the fp64 output accumulator (fire-and-forget
//            fp64 reductions in L2: the drain warps wait on no load).
//
// Operands.  The factors are packed once per matrix and direction into bf16
// slices laid out exactly as the MMAs read them (tc_pack below): a phase-1
// group panel holds, per 16-position block, the slices of all the group's
// ranks; a phase-2 entry panel holds, per 16-rank step, the slices of the
// 128 rows of one output tile.  fp32 values are split exactly into three
// slices s0 + s1 + s2, fp16 into two, bf16 and e4m3 values are one slice.
// The input X (fp32 of the fp64 input) and T (fp32) are written as three
// slices for fp32 pieces and two for the others.  Products kept: factor slice
// i times input slice j for i + j <= 2 (fp32: six products), i + j <= 1
// (fp16: three), j <= 1 (bf16 and e4m3: two): everything above about 2^-24
// (fp32) or the unit roundoff of the 16- and 8-bit formats.
//
// Accumulation.  The tensor core's fp32 accumulation does not round to
// nearest; its error grows with the number of MMAs that add into one
// accumulator.  The main products (slice 0 x slice 0) and the correction
// products accumulate in separate tensor-memory columns, and after every
// chunk of K steps (4 for fp32 pieces, 32 for the others) the accumulators
// are drained into fp32 registers with round-to-nearest additions; two banks
// alternate so that the MMAs of the next chunk overlap the drain of the last.
//
// Kernels.  Both phases are persistent and warp-specialized, one CTA per SM
// (192 threads, ~193 KB of shared memory, all 512 tensor-memory columns):
//   warp 0     lane 0 fills a 4-deep ring of 48 KB stages, two K steps each,
//              with bulk copies (input or T slices, factor panel slices);
//   warp 1     lane 0 issues the MMAs of a stage once its copies landed and,
//              for a chunk's first stage, once its bank has been drained;
//              tcgen05.commit frees the stage and hands a bank over (an MMA
//              instruction costs its issuing thread tens of cycles whatever
//              its size, so a stage carries two K steps and the descriptors
//              are advanced by additions);
//   warps 2-5  drain the banks (tensor-memory lane quarter w mod 4) into fp32
//              registers and write each item's result.
// Items are cost-sorted on the host and taken dynamically from a work
// counter by each CTA's producer, which passes their indices to the other
// roles through a small shared-memory queue.  Shared-memory operands use the K-major
// layout without swizzling: 8-row by 16-byte core matrices, the two core
// matrices of one K step 128 bytes apart (leading byte offset), successive
// 8-row groups 256 bytes apart (stride byte offset).  Every mbarrier wait has
// a clock limit; an expired wait sets an abort flag that the other roles see,
// sets bit 3 of the status word, and the CTA ends after its copies and MMAs
// have completed and its tensor memory has been released.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "hh_device.h"

namespace hh {
namespace dev {

namespace {

constexpr long long kWaitCycles = 4000000000LL;
constexpr int kThreads = 192;
constexpr int kKS = kTcKSteps;           // K steps per stage
constexpr int kDepth = 2;         // stages per CTA
constexpr int kCtasPerSm = 2;     // two CTAs per SM: two bulk-copy queues, two MMA issuers
constexpr int kBanks = 1;         // accumulator banks per CTA (256 tensor-memory columns each)
// a stage: kKS K steps of the A operand (phase 1: X slices [3][128 x 32 B]
// per step; phase 2: U slices [sf][128 x 32 B] per step), then kKS K steps of
// the B operand (phase 1: V slices [sf][nk x 32 B]; phase 2: T slices
// [sx][rp x 32 B])
constexpr int kOpA = kKS * 3 * 4096;
constexpr int kOpB = kKS * 3 * 4096;
constexpr int kStage = kOpA + kOpB;
constexpr uint32_t kTmemCols = 256 * kBanks;  // bank b: main at 256 b, corrections at 256 b + 128
// Stages whose K steps add into one bank before it is drained
// (kTcChunkF32 / kTcChunk16).  Each MMA's addition into an fp32 accumulator
// truncates (at most one unit in the last place of the running sum), so over
// n steps the error is at most about n * 2^-24 of the absolute sum of the
// chunk's products: fp32 pieces drain after 2 stages (4 steps: 2^-22, below
// what their 2^-24 unit roundoff and the three-slice products leave), the
// 16- and 8-bit pieces after 16 (32 steps: 2^-19, far below their unit
// roundoff).
constexpr int kChunkF32 = kTcChunkF32;
constexpr int kChunk16 = kTcChunk16;

constexpr int kF32 = 1, kF16 = 2, kBF16 = 3, kE4M3 = 4;

__device__ __forceinline__ int n_products(int f) { return f == kF32 ? 6 : (f == kF16 ? 3 : 2); }
__device__ __forceinline__ int chunk_of(int f) { return f == kF32 ? kChunkF32 : kChunk16; }
// product p: factor slice fpf(p) times input slice fpx(p): (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
__device__ __forceinline__ int fpf(int p) { return (0x210100 >> (4 * p)) & 0xf; }
__device__ __forceinline__ int fpx(int p) { return (0x012010 >> (4 * p)) & 0xf; }

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, no swizzle: leading byte offset 128 (next core matrix along K),
// stride byte offset 256 (next 8-row group)
__device__ __forceinline__ uint64_t op_desc(const void* p) {
  const uint32_t a = saddr(p);
  uint64_t d = static_cast<uint64_t>((a >> 4) & 0x3fff);
  d |= static_cast<uint64_t>(128 >> 4) << 16;
  d |= static_cast<uint64_t>(256 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

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

// The np products of one K step into the bank at tmem (main at +0, corrections
// at +128).  Descriptors are advanced by adding to the start-address field
// (bits 0-13, address / 16): da / db address slice 0 of the A and B operands,
// a_step / b_step are the slice strides / 16.  Phase 1: A = input slices
// fpx(p), B = factor slices fpf(p); phase 2: A = factor slices, B = input
// (T) slices.  acc0: whether the main and first correction products add to
// the bank (later corrections always do).
template <int NP, bool PH2>
__device__ __forceinline__ void issue_products(uint32_t tmem, uint64_t da, uint64_t db, uint32_t a_step,
                                               uint32_t b_step, uint32_t idesc, uint32_t acc0) {
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int ia = PH2 ? fpf(p) : fpx(p), ib = PH2 ? fpx(p) : fpf(p);
    mma(tmem + (p ? 128 : 0), da + ia * a_step, db + ib * b_step, idesc, p >= 2 ? 1u : acc0);
  }
}

template <bool PH2>
__device__ __forceinline__ void issue_step(int np, uint32_t tmem, uint64_t da, uint64_t db, uint32_t a_step,
                                           uint32_t b_step, uint32_t idesc, uint32_t acc0) {
  if (np == 6)
    issue_products<6, PH2>(tmem, da, db, a_step, b_step, idesc, acc0);
  else if (np == 3)
    issue_products<3, PH2>(tmem, da, db, a_step, b_step, idesc, acc0);
  else
    issue_products<2, PH2>(tmem, da, db, a_step, b_step, idesc, acc0);
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
// streamed once: evict-first in L2
__device__ __forceinline__ void bulk_copy_once(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                               uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 16 columns of this warp's 32 lanes, without waiting (tcgen05.wait::ld follows)
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// eight values -> their first ns (1..3) bf16 slices (s0 = bf16(v), s1 =
// bf16(v - s0), s2 = bf16(v - s0 - s1); the differences are exact in fp32),
// 16 bytes each, at dst + s * sstride
__device__ __forceinline__ void store_slices(const float* v, int ns, uint8_t* dst, int64_t sstride) {
  __align__(16) __nv_bfloat16 s[3][8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    s[0][t] = __float2bfloat16_rn(v[t]);
    const float r1 = v[t] - __bfloat162float(s[0][t]);
    s[1][t] = __float2bfloat16_rn(r1);
    s[2][t] = __float2bfloat16_rn(r1 - __bfloat162float(s[1][t]));
  }
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(s[0]);
  if (ns > 1) *reinterpret_cast<uint4*>(dst + sstride) = *reinterpret_cast<const uint4*>(s[1]);
  if (ns > 2) *reinterpret_cast<uint4*>(dst + 2 * sstride) = *reinterpret_cast<const uint4*>(s[2]);
}

// stored factor element i of a column (format fmt) as fp32
__device__ __forceinline__ float load_factor(const uint8_t* f, int fmt, int64_t i) {
  if (fmt == kF32) return reinterpret_cast<const float*>(f)[i];
  if (fmt == kE4M3) {
    __half_raw h = __nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(f[i]), __NV_E4M3);
    return __half2float(__half(h));
  }
  const uint16_t b = reinterpret_cast<const uint16_t*>(f)[i];
  if (fmt == kBF16) return __uint_as_float(static_cast<uint32_t>(b) << 16);
  __half_raw h;
  h.x = b;
  return __half2float(__half(h));
}

// byte offset of (row, 8-element group c of the K step) in a K-major operand tile
__device__ __forceinline__ int core_off(int row, int c) { return (row >> 3) * 256 + c * 128 + (row & 7) * 16; }

__device__ __forceinline__ uint8_t* align128(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 127) & ~static_cast<uintptr_t>(127));
}

constexpr int kQ = 4;  // item queue slots between the producer and the other roles

struct Ctl {
  uint64_t full[kDepth], empty[kDepth];
  uint64_t bfull[kBanks], bempty[kBanks];
  uint64_t qfull[kQ], qempty[kQ];  // item index published / read by the MMA thread and the 4 drain warps
  int qid[kQ];
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

__device__ __forceinline__ void ws_setup(Ctl* c) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kDepth; ++s) {
      mbar_init(&c->full[s], 1);
      mbar_init(&c->empty[s], 1);
    }
    for (int b = 0; b < kBanks; ++b) {
      mbar_init(&c->bfull[b], 1);
      mbar_init(&c->bempty[b], 4);
    }
    for (int q = 0; q < kQ; ++q) {
      mbar_init(&c->qfull[q], 1);
      mbar_init(&c->qempty[q], 5);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    c->abort = 0;
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&c->tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Items are taken dynamically, in the host's cost order, from a work counter
// in global memory (cleared by the input-image launch): the producer takes
// the index of its k-th item and publishes it in queue slot k mod kQ; the MMA
// thread and the drain warps read it there.  Returns the item, -1 when the
// list is exhausted, -2 when a bounded wait gave up.
__device__ __forceinline__ int q_publish(Ctl* c, int k, int* counter, int n, volatile int* abort) {
  const int slot = k % kQ;
  if (k >= kQ && !ws_wait(&c->qempty[slot], ((k / kQ) - 1) & 1, abort)) return -2;
  int it = atomicAdd(counter, 1);
  if (it >= n) it = -1;
  c->qid[slot] = it;
  mbar_arrive(&c->qfull[slot]);
  return it;
}
// whole_warp: a drain warp (all lanes read, lane 0 releases the slot);
// otherwise the single MMA-issuing thread
__device__ __forceinline__ int q_take(Ctl* c, int k, volatile int* abort, bool whole_warp) {
  const int slot = k % kQ;
  if (!ws_wait(&c->qfull[slot], (k / kQ) & 1, abort)) return -2;
  const int it = *reinterpret_cast<volatile int*>(&c->qid[slot]);
  if (whole_warp) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&c->qempty[slot]);
  } else {
    mbar_arrive(&c->qempty[slot]);
  }
  return it;
}

// after the role loops: on an abort the producer waits (bounded) for the
// copies it issued and the MMA thread for its last MMAs; then tensor memory
// is freed.  produced / mmas: stages issued by the producer / the MMA thread.
__device__ __forceinline__ void ws_teardown(Ctl* c, int produced, int mmas, int* status) {
  __syncthreads();
  if (c->abort) {
    volatile int no = 0;
    if (threadIdx.x == 0)
      for (int i = produced > kDepth ? produced - kDepth : 0; i < produced; ++i)
        ws_wait(&c->full[i % kDepth], (i / kDepth) & 1, &no);
    if (threadIdx.x == 32 && mmas > 0) ws_wait(&c->empty[(mmas - 1) % kDepth], ((mmas - 1) / kDepth) & 1, &no);
    if (threadIdx.x == 0) atomicOr(status, 8);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c->tmem), "r"(kTmemCols));
}

// drain warps: add bank b (this warp's lane quarter, columns 0 .. ncols) into
// acc, 16 columns (main and corrections) per tcgen05.wait::ld
__device__ __forceinline__ void drain(const Ctl* c, int bank, int ncols, float* acc) {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int w = threadIdx.x >> 5;
  const uint32_t t = c->tmem + (static_cast<uint32_t>(32 * (w & 3)) << 16) + 256 * bank;
#pragma unroll
  for (int cb = 0; cb < 8; ++cb) {
    if (16 * cb < ncols) {
      uint32_t h0[16], l0[16];
      tmem_ld16_nowait(t + 16 * cb, h0);
      tmem_ld16_nowait(t + 128 + 16 * cb, l0);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[16 * cb + j] += __uint_as_float(h0[j]) + __uint_as_float(l0[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// T = 2^e D of 16 ranks (group columns cb16 ..) of right-hand side r, as the
// slices of the phase-2 operand image of its piece
__device__ __forceinline__ void write_t(const TcArgs& a, const TcPiece& q, int cb16, int r, float* v) {
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = ldexpf(v[j], q.e);
  const int sx = tc_input_slices(q.fmt);
  const int step = (cb16 - q.col) >> 4;
  uint8_t* dst = a.timg + q.toff + static_cast<int64_t>(step) * sx * 4096 + core_off(r, 0);
  store_slices(v, sx, dst, 4096);
  store_slices(v + 8, sx, dst + 128, 4096);
}

// piece of a group that holds group column col
__device__ __forceinline__ const TcPiece& piece_at(const TcArgs& a, const TcGroup& g, int col) {
  int i = g.first;
  for (int t = 1; t < g.count; ++t)
    if (a.pieces[g.first + t].col <= col) i = g.first + t;
  return a.pieces[i];
}

// ------------------------------------------------------------------ phase 1
__global__ void __launch_bounds__(kThreads, kCtasPerSm) tc_phase1(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align128(smem_raw);
  Ctl* c = reinterpret_cast<Ctl*>(base + kDepth * kStage);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  ws_setup(c);
  volatile int* abort = &c->abort;
  int produced = 0, mmas = 0;

  if (w == 0) {  // producer
    if (lane == 0) {
      const uint64_t pol = evict_first();
      int gs = 0;
      bool ok = true;
      int itn = q_publish(c, 0, a.work, a.n_groups, abort);
      TcGroup gn{};
      if (itn >= 0) gn = a.groups[itn];  // the next item, loaded one ahead
      for (int k = 0; ok && itn >= 0; ++k) {
        const TcGroup g = gn;
        itn = q_publish(c, k + 1, a.work, a.n_groups, abort);
        if (itn == -2) break;
        if (itn >= 0) gn = a.groups[itn];
        const uint32_t vbytes = tc_factor_slices(g.fmt) * static_cast<uint32_t>(g.nk) * 32u;
        const int nblk = (g.p1 - g.p0 + 15) >> 4, nst = (nblk + kKS - 1) / kKS;
        for (int i = 0; i < nst; ++i, ++gs) {
          const int s = gs % kDepth;
          if (gs >= kDepth && !ws_wait(&c->empty[s], ((gs / kDepth) - 1) & 1, abort)) {
            ok = false;
            break;
          }
          uint8_t* st = base + s * kStage;
          // 16-position blocks b0 .. b0 + nb - 1 of the cluster
          const int b0 = (g.p0 >> 4) + kKS * i, nb = min(kKS, nblk - kKS * i);
          const int64_t blk = (static_cast<int64_t>(g.in_off) >> 4) + b0;
          // the stage's input blocks with all three slices in one copy (the
          // 16- and 8-bit groups read two of them): a CTA's bulk copies run
          // one after another, so fewer and larger copies fill faster
          mbar_expect_tx(&c->full[s], nb * (3u * 4096u + vbytes));
          bulk_copy(st, a.ximg + blk * (3 * 4096), nb * (3u * 4096u), &c->full[s]);
          bulk_copy_once(st + kOpA, a.img + g.img + static_cast<int64_t>(b0) * vbytes, nb * vbytes, &c->full[s], pol);
          produced = gs + 1;
        }
      }
    }
  } else if (w == 1) {  // MMA issuer
    if (lane == 0) {
      const uint64_t d0 = op_desc(base);
      int gs = 0, gp = 0;
      bool ok = true;
      int itn = q_take(c, 0, abort, false);
      TcGroup gn{};
      if (itn >= 0) gn = a.groups[itn];  // the next item, loaded one ahead
      for (int k = 0; ok && itn >= 0; ++k) {
        const TcGroup g = gn;
        itn = q_take(c, k + 1, abort, false);
        if (itn == -2) break;
        if (itn >= 0) gn = a.groups[itn];
        const int np = n_products(g.fmt), nblk = (g.p1 - g.p0 + 15) >> 4, nst = (nblk + kKS - 1) / kKS;
        const int L = chunk_of(g.fmt);
        const uint32_t idesc = idesc_bf16(g.nk), vstep = static_cast<uint32_t>(g.nk) * 2u;
        const uint32_t vstage = tc_factor_slices(g.fmt) * vstep;  // V bytes of one K step / 16
        int s = gs % kDepth, par = (gs / kDepth) & 1;
        for (int i = 0, j = 0; i < nst; ++i, ++gs) {
          // chunks of L stages alternate between the banks: a chunk's first
          // K step starts fresh accumulators, the others add to them, then
          // the bank is handed to the drain warps
          const int b = gp % kBanks;
          if (!ws_wait(&c->full[s], par, abort)) {
            ok = false;
            break;
          }
          if (j == 0) {
            if (gp >= kBanks && !ws_wait(&c->bempty[b], ((gp / kBanks) - 1) & 1, abort)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          }
          const uint64_t da = d0 + static_cast<uint32_t>(s * (kStage >> 4));
          const int nb = min(kKS, nblk - kKS * i);
          for (int t = 0; t < nb; ++t)
            issue_step<false>(np, c->tmem + 256 * b, da + t * (3 * 256), da + (kOpA >> 4) + t * vstage, 256u, vstep,
                              idesc, (j != 0 || t != 0));
          mma_commit(&c->empty[s]);
          if (++j == L || i == nst - 1) {
            mma_commit(&c->bfull[b]);
            ++gp;
            j = 0;
          }
          mmas = gs + 1;
          if (++s == kDepth) {
            s = 0;
            par ^= 1;
          }
        }
      }
    }
  } else {  // drain warps: right-hand side r of this lane, group columns 0 .. nk
    const int quarter = w & 3, r = 32 * quarter + lane;
    float acc[128];
    int gp = 0;
    bool ok = true;
    int itn = q_take(c, 0, abort, true);
    TcGroup gn{};
    if (itn >= 0) gn = a.groups[itn];
    for (int k = 0; ok && itn >= 0; ++k) {
      const TcGroup g = gn;
      itn = q_take(c, k + 1, abort, true);
      if (itn == -2) break;
      if (itn >= 0) gn = a.groups[itn];
      const int L = chunk_of(g.fmt), nk = g.nk, nst = (((g.p1 - g.p0 + 15) >> 4) + kKS - 1) / kKS;
      const int nchunks = (nst + L - 1) / L;
#pragma unroll
      for (int j = 0; j < 128; ++j) acc[j] = 0.f;
      for (int q = 0; q < nchunks; ++q, ++gp) {
        const int b = gp % kBanks;
        if (!ws_wait(&c->bfull[b], (gp / kBanks) & 1, abort)) {
          ok = false;
          break;
        }
        drain(c, b, nk, acc);
        __syncwarp();
        if (lane == 0) mbar_arrive(&c->bempty[b]);
      }
      if (!ok) break;
      if (g.nsplit == 1) {
#pragma unroll
        for (int cb = 0; cb < 8; ++cb) {
          if (16 * cb >= nk) break;
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = acc[16 * cb + j];
          write_t(a, piece_at(a, g, 16 * cb), 16 * cb, r, v);
        }
        continue;
      }
      // split group: partial sums, then the quarter's last arrival adds them
      const int64_t pstride = static_cast<int64_t>(128) * nk;
#pragma unroll
      for (int cb = 0; cb < 8; ++cb) {
        if (16 * cb >= nk) break;
        float4* dst = reinterpret_cast<float4*>(a.part + g.poff + static_cast<int64_t>(r) * nk + 16 * cb);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          dst[j] = make_float4(acc[16 * cb + 4 * j], acc[16 * cb + 4 * j + 1], acc[16 * cb + 4 * j + 2],
                               acc[16 * cb + 4 * j + 3]);
      }
      __threadfence();
      __syncwarp();
      int last = 0;
      if (lane == 0) last = atomicAdd(a.cnt + 4 * g.gid + quarter, 1) == g.nsplit - 1;
      last = __shfl_sync(0xffffffffu, last, 0);
      if (!last) continue;
      __threadfence();
      const float* p0 = a.part + g.poff - static_cast<int64_t>(g.split) * pstride;
      for (int cb = 0; cb < 8; ++cb) {
        if (16 * cb >= nk) break;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
        for (int sp = 0; sp < g.nsplit; ++sp) {
          const float4* src =
              reinterpret_cast<const float4*>(p0 + sp * pstride + static_cast<int64_t>(r) * nk + 16 * cb);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 f = __ldcg(src + j);
            v[4 * j] += f.x;
            v[4 * j + 1] += f.y;
            v[4 * j + 2] += f.z;
            v[4 * j + 3] += f.w;
          }
        }
        write_t(a, piece_at(a, g, 16 * cb), 16 * cb, r, v);
      }
      if (lane == 0) a.cnt[4 * g.gid + quarter] = 0;
    }
  }
  ws_teardown(c, produced, mmas, a.status);
}

// ------------------------------------------------------------------ phase 2
__global__ void __launch_bounds__(kThreads, kCtasPerSm) tc_phase2(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align128(smem_raw);
  Ctl* c = reinterpret_cast<Ctl*>(base + kDepth * kStage);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, rp = a.rp;
  ws_setup(c);
  volatile int* abort = &c->abort;
  int produced = 0, mmas = 0;

  if (w == 0) {  // producer: U panel slices and T slices of up to kKS 16-rank steps of one entry
    if (lane == 0) {
      const uint64_t pol = evict_first();
      int gs = 0;
      bool ok = true;
      int itn = q_publish(c, 0, a.work + 1, a.n_tiles, abort);
      TcTile tn{};
      if (itn >= 0) tn = a.tiles[itn];  // the next item, loaded one ahead
      for (int k = 0; ok && itn >= 0; ++k) {
        const TcTile tl = tn;
        itn = q_publish(c, k + 1, a.work + 1, a.n_tiles, abort);
        if (itn == -2) break;
        if (itn >= 0) tn = a.tiles[itn];
        TcEntry nx = a.entries[tl.first];  // the next entry, loaded one ahead
        for (int e = 0; e < tl.count && ok; ++e) {
          const TcEntry en = nx;
          if (e + 1 < tl.count) nx = a.entries[tl.first + e + 1];
          const uint32_t ub = tc_factor_slices(en.fmt) * 4096u, tb = tc_input_slices(en.fmt) * 4096u;
          const int nks = en.nks;
          for (int ks = 0; ks < nks; ks += kKS, ++gs) {
            const int s = gs % kDepth, nb = min(kKS, nks - ks);
            if (gs >= kDepth && !ws_wait(&c->empty[s], ((gs / kDepth) - 1) & 1, abort)) {
              ok = false;
              break;
            }
            uint8_t* st = base + s * kStage;
            mbar_expect_tx(&c->full[s], nb * (ub + tb));
            bulk_copy_once(st, a.img + en.img + static_cast<int64_t>(ks) * ub, nb * ub, &c->full[s], pol);
            bulk_copy(st + kOpA, a.timg + en.toff + static_cast<int64_t>(ks) * tb, nb * tb, &c->full[s]);
            produced = gs + 1;
          }
        }
      }
    }
  } else if (w == 1) {  // MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(rp);
      const uint64_t d0 = op_desc(base);
      int gs = 0, gp = 0;
      bool ok = true;
      int itn = q_take(c, 0, abort, false);
      TcTile tn{};
      if (itn >= 0) tn = a.tiles[itn];  // the next item, loaded one ahead
      for (int k = 0; ok && itn >= 0; ++k) {
        const TcTile tl = tn;
        itn = q_take(c, k + 1, abort, false);
        if (itn == -2) break;
        if (itn >= 0) tn = a.tiles[itn];
        const int nst = tl.nst, L = tl.chunk;
        int i = 0, j = 0, s = gs % kDepth, par = (gs / kDepth) & 1;
        int2 nx = *reinterpret_cast<const int2*>(&a.entries[tl.first].nks);  // {nks, fmt} of the next entry
        for (int e = 0; e < tl.count && ok; ++e) {
          const int nks = nx.x, fmt = nx.y;
          if (e + 1 < tl.count) nx = *reinterpret_cast<const int2*>(&a.entries[tl.first + e + 1].nks);
          const int np = n_products(fmt);
          const uint32_t ustep = tc_factor_slices(fmt) * 256u, tstep = tc_input_slices(fmt) * 256u;
          for (int ks = 0; ks < nks; ks += kKS, ++i, ++gs) {
            const int b = gp % kBanks;
            if (!ws_wait(&c->full[s], par, abort)) {
              ok = false;
              break;
            }
            if (j == 0) {
              if (gp >= kBanks && !ws_wait(&c->bempty[b], ((gp / kBanks) - 1) & 1, abort)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            const uint64_t da = d0 + static_cast<uint32_t>(s * (kStage >> 4));
            const int nb = min(kKS, nks - ks);
            for (int t = 0; t < nb; ++t)
              issue_step<true>(np, c->tmem + 256 * b, da + t * ustep, da + (kOpA >> 4) + t * tstep, 256u, 256u, idesc,
                               (j != 0 || t != 0));
            mma_commit(&c->empty[s]);
            if (++j == L || i == nst - 1) {
              mma_commit(&c->bfull[b]);
              ++gp;
              j = 0;
            }
            mmas = gs + 1;
            if (++s == kDepth) {
              s = 0;
              par ^= 1;
            }
          }
        }
      }
    }
  } else {  // drain warps: tile row of this lane, right-hand sides 0 .. rp
    const int row = 32 * (w & 3) + lane;
    float acc[128];
    int gp = 0;
    bool ok = true;
    int itn = q_take(c, 0, abort, true);
    TcTile tn{};
    if (itn >= 0) tn = a.tiles[itn];
    for (int k = 0; ok && itn >= 0; ++k) {
      const TcTile tl = tn;
      itn = q_take(c, k + 1, abort, true);
      if (itn == -2) break;
      if (itn >= 0) tn = a.tiles[itn];
      const int nst = tl.nst, L = tl.chunk;
#pragma unroll
      for (int j = 0; j < 128; ++j) acc[j] = 0.f;
      for (int q = 0; q < (nst + L - 1) / L; ++q, ++gp) {
        const int b = gp % kBanks;
        if (!ws_wait(&c->bfull[b], (gp / kBanks) & 1, abort)) {
          ok = false;
          break;
        }
        drain(c, b, rp, acc);
        __syncwarp();
        if (lane == 0) mbar_arrive(&c->bempty[b]);
      }
      if (!ok || nst == 0 || row >= tl.rows) continue;
#pragma unroll
      for (int j = 0; j < 128; ++j)
        if (j < a.nr) atomicAdd(a.acc + static_cast<int64_t>(j) * a.npad + tl.row0 + row, f32_to_f64(acc[j], 0));
    }
  }
  ws_teardown(c, produced, mmas, a.status);
}

// ------------------------------------------------------------- packing
// Phase-1 group panels (one CTA per group item, over the item's positions):
// unit (column j, 16-position block pb, half cc) holds positions
// 16 pb + 8 cc .. + 7 of group column j as factor slices at
// img + g.img + pb * (sf * nk * 32) + s * nk * 32 + core_off(j, cc); ranks
// past a piece's k and positions past the cluster are zero.
__global__ void tc_pack1_kernel(const TcPiece* __restrict__ pieces, const TcGroup* __restrict__ groups,
                                uint8_t* __restrict__ img) {
  const TcGroup g = groups[blockIdx.x];
  const int sf = tc_factor_slices(g.fmt), pb0 = g.p0 >> 4, nb = ((g.p1 + 15) >> 4) - pb0, nk = g.nk;
  const int64_t units = static_cast<int64_t>(nk) * nb * 2;
  for (int64_t u = threadIdx.x; u < units; u += blockDim.x) {
    const int j = static_cast<int>(u / (2 * nb)), rest = static_cast<int>(u % (2 * nb));
    const int pb = pb0 + (rest >> 1), cc = rest & 1;
    int pi = g.first;
    for (int t = 1; t < g.count; ++t)
      if (pieces[g.first + t].col <= j) pi = g.first + t;
    const TcPiece& q = pieces[pi];
    const int rk = j - q.col;
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int pos = 16 * pb + 8 * cc + t;
      v[t] = (rk < q.k && pos < g.rows) ? load_factor(q.f1, q.fmt, static_cast<int64_t>(rk) * q.ld1 + pos) : 0.f;
    }
    store_slices(v, sf, img + g.img + static_cast<int64_t>(pb) * sf * nk * 32 + core_off(j, cc),
                 static_cast<int64_t>(nk) * 32);
  }
}

// Phase-2 entry panels (one CTA per entry): unit (step ks, half cc, tile row
// m) holds ranks 16 ks + 8 cc .. + 7 of tile row m as factor slices at
// img + en.img + ks * sf * 4096 + s * 4096 + core_off(m, cc); rows outside
// the entry and ranks past k are zero.
__global__ void tc_pack2_kernel(const TcPiece* __restrict__ pieces, const TcEntry* __restrict__ entries,
                                uint8_t* __restrict__ img) {
  const TcEntry en = entries[blockIdx.x];
  const TcPiece& q = pieces[en.piece];
  const int sf = tc_factor_slices(q.fmt), nks = q.kp >> 4;
  const int units = nks * 2 * 128;
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int m = u & 127, cc = (u >> 7) & 1, ks = u >> 8;
    const bool in = m >= en.dst && m < en.dst + en.nrows;
    const int64_t row = en.src + (m - en.dst);
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int rk = 16 * ks + 8 * cc + t;
      v[t] = (in && rk < q.k) ? load_factor(q.f2, q.fmt, static_cast<int64_t>(rk) * q.ld2 + row) : 0.f;
    }
    store_slices(v, sf, img + en.img + static_cast<int64_t>(ks) * sf * 4096 + core_off(m, cc), 4096);
  }
}

// X (caller's order, column-major, ld) -> xt (tree order, [nr][npad] fp64),
// column by column: consecutive threads take consecutive tree positions of
// the same column, so the gathered reads of the threads in flight stay in a
// few columns of X (L2) and the writes are coalesced
__global__ void tc_gather_kernel(const double* __restrict__ x, int64_t ld, int nr, const int32_t* __restrict__ perm,
                                 int64_t n, int64_t npad, double* __restrict__ xt) {
  const int64_t total = static_cast<int64_t>(nr) * npad;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total; q += stride) {
    const int64_t r = q / npad, p = q - r * npad;
    xt[q] = p < n ? x[static_cast<int64_t>(perm[p]) + r * ld] : 0.0;
  }
}

// the input in tree order (xt, or X read through the permutation when xt is
// null) -> the images, once per product:
//   * fp32 of each value as three bf16 slices in the phase-1 operand image
//     [16-position block][slice][128 rows x 32 B] (rows r >= nr and positions
//     >= n are zero);
//   * its fp32 leading and trailing halves [npos][128] for the CUDA-core
//     kernels (mr.cu);
// and clears the output accumulator, the arrival counters of the split
// groups and the T arena of the CUDA-core pieces.  One gather of X feeds
// both images; each value is split into fp32 halves with integer operations.
__global__ void tc_prep_kernel(const double* __restrict__ x, int64_t ld, const int32_t* __restrict__ perm,
                               const double* __restrict__ xt, int nr, int64_t n, int64_t nblk,
                               uint8_t* __restrict__ ximg, double* __restrict__ acc, int64_t npad,
                               int* __restrict__ cnt, int n_cnt, float* __restrict__ xh, float* __restrict__ xl,
                               int64_t npos, float* __restrict__ t32, int64_t t_floats) {
  const int64_t total = nblk * 256;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  for (int64_t q = t0; q < total; q += stride) {
    const int64_t blk = q >> 8;
    const int c = static_cast<int>(q >> 7) & 1, r = static_cast<int>(q & 127);
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int64_t p = 16 * blk + 8 * c + t;
      double d = 0.0;
      if (r < nr && p < n) d = xt ? xt[static_cast<int64_t>(r) * npad + p] : x[static_cast<int64_t>(perm[p]) + r * ld];
      float lo;
      split_f64(d, v[t], lo);
      if (p < npos) {
        xh[p * 128 + r] = v[t];
        xl[p * 128 + r] = lo;
      }
    }
    store_slices(v, 3, ximg + blk * (3 * 4096) + core_off(r, c), 4096);
  }
  const int64_t ntot = static_cast<int64_t>(nr) * npad;
  for (int64_t q = t0; q < ntot; q += stride) acc[q] = 0.0;
  for (int64_t q = t0; q < n_cnt; q += stride) cnt[q] = 0;
  for (int64_t q = t0; q < t_floats; q += stride) t32[q] = 0.f;
}

}  // namespace

cudaError_t launch_tc_prep(const double* x, int64_t ld, int nr, const int32_t* perm, int64_t n, int64_t nblk,
                           uint8_t* ximg, double* acc, int64_t npad, int* cnt, int n_cnt, float* xh, float* xl,
                           int64_t npos, float* t32, int64_t t_floats, double* xt, cudaStream_t st) {
  if (16 * nblk < npos) return cudaErrorInvalidValue;  // the fp32 images must be covered
  // the input's columns read through the permutation stay in L2 up to about
  // 100 MB; beyond that they are first gathered column by column into xt
  const bool gather = static_cast<int64_t>(nr) * n * 8 > (int64_t(100) << 20);
  if (gather) {
    int64_t gb = (static_cast<int64_t>(nr) * npad + 255) / 256;
    if (gb > 8192) gb = 8192;
    if (gb < 1) gb = 1;
    tc_gather_kernel<<<static_cast<int>(gb), 256, 0, st>>>(x, ld, nr, perm, n, npad, xt);
  }
  int64_t blocks = (nblk * 256 + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  tc_prep_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(x, ld, perm, gather ? xt : nullptr, nr, n, nblk, ximg, acc,
                                                          npad, cnt, n_cnt, xh, xl, npos, t32, t_floats);
  return cudaGetLastError();
}

cudaError_t launch_tc_pack(const TcPiece* pieces, const TcGroup* groups, int n_groups, const TcEntry* entries,
                           int n_entries, uint8_t* img, cudaStream_t st) {
  if (n_groups > 0) tc_pack1_kernel<<<n_groups, 256, 0, st>>>(pieces, groups, img);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (n_entries > 0) tc_pack2_kernel<<<n_entries, 256, 0, st>>>(pieces, entries, img);
  return cudaGetLastError();
}

cudaError_t launch_tc(int phase, const TcArgs& a, int grid, cudaStream_t st) {
  if (a.rp < 16 || a.rp > 128 || (a.rp & 15)) return cudaErrorInvalidValue;
  const int n = phase == 1 ? a.n_groups : a.n_tiles;
  if (n <= 0) return cudaSuccess;
  grid *= kCtasPerSm;  // grid: SMs
  if (grid > n) grid = n;
  if (grid < 1) grid = 1;
  const size_t smem = kDepth * kStage + 128 + sizeof(Ctl);
  auto k = phase == 1 ? tc_phase1 : tc_phase2;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace hh
