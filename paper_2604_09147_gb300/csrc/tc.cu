// Tensor-core path (tcgen05, kind::f16 with bf16 operands) of the H_h product
// for many right-hand sides: low-rank blocks stored in fp16, bf16 or fp8-e4m3
// (the kernels also take fp32 factors as three slices; the host keeps fp32
// blocks on the streaming passes, see below).  With R right-hand sides the two phases of Algorithm 4 become
// dense contractions,
//   phase 1  T_b = 2^(e_u+e_v) V_b^T X_J          (k_b x R, contraction over |J|)
//   phase 2  Y_I += U_b T_b                        (|I| x R, contraction over k_b)
// computed as
//   phase 1  one CTA per group of blocks sharing the input cluster J and the
//            format: D[r][col] = sum_p X[p][r] V[p][col], M = 128 right-hand
//            sides, N = the group's ranks, K = positions of J (16 per MMA);
//   phase 2  one CTA per 256-row output tile: two 128-row accumulators
//            D[row][r] = sum over the blocks covering the tile and their ranks
//            of U[row][j] T[j][r], N = R, then added once into the fp64 output.
//
// Precision.  The operands are bf16 slices: a value v of a format with more
// than 8 significant bits is written exactly as s0 + s1 (+ s2), s_i =
// bf16(v - s0 - ... - s_{i-1}).  Factors: fp32 3 slices, fp16 2, bf16 and
// e4m3 1 (all exact).  The input X (fp32 of the fp64 input) and T (fp32) are
// sliced in the same way.  The products kept are those with slice indices
// i + j < 3 (fp32 blocks: 6 MMAs per K step) or i + j < 2 (2 or 3 MMAs),
// which leaves a slicing error of about 2^-24 (fp32) or 2^-17 (other formats,
// whose own unit roundoff is 2^-11 or larger).  Accumulation is fp32 in tensor
// memory; the output accumulator is fp64.  The tensor core's accumulation
// does not round to nearest: measured against the exact sums, the error grows
// with the number of MMAs that add into one accumulator, to about 2^-17 of a
// block's product over a few hundred MMAs.  That is far below the unit
// roundoff of the 16- and 8-bit formats, but not below fp32's, so fp32 blocks
// keep the CUDA-core passes, whose sums round to nearest.  The main products
// (slice 0 times slice 0) and the correction products accumulate in separate
// tensor-memory columns (0.. and 256..), so the many small additions do not
// land on the large accumulator.
//
// Shared-memory operands use the K-major layout without swizzling: 8-row by
// 16-byte core matrices, the two core matrices of one 16-element K step 128
// bytes apart (leading byte offset) and successive 8-row groups 256 bytes apart
// (stride byte offset).  Stages are filled with cp.async (16-byte copies into
// shared memory) several stages ahead; formats other than bf16 land raw and are
// converted into slices by the CTA's threads.  One thread issues the MMAs;
// tcgen05.commit on a per-stage mbarrier frees the stage.  Every mbarrier wait
// is bounded by a clock limit that sets bit 3 of the status word; an expired
// wait ends the CTA after its copies have landed and its tensor memory has been
// released.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "hh_device.h"

namespace hh {
namespace dev {

namespace {

constexpr int kThreads = 256;
constexpr long long kWaitCycles = 4000000000LL;
constexpr int kTmemCols = 512;
constexpr int kLoCol = 256;  // accumulator of the correction products (slice index sum > 0)

// phase 1 stage: 2 K steps (32 positions)
constexpr int kP1Steps = 2;
constexpr int kP1XOp = 3 * kP1Steps * 4096;  // X slices [slice][step][128 rows x 32 B]
constexpr int kP1VOp = 32768;                // V slices [slice][step][nk rows x 32 B]
constexpr int kP1Raw = 16384;                // raw factor bytes [nk ranks][32 positions]
constexpr int kP1Stage = kP1XOp + kP1VOp + kP1Raw;
constexpr int kP1Depth = 3;
// phase 2 stage: 1 K step (16 ranks) of a 256-row tile
constexpr int kP2Rows = 256;
constexpr int kP2Raw = 16 * kP2Rows * 4;  // raw factor bytes [16 ranks][256 rows]
constexpr int kP2UOp = 3 * kP2Rows * 32;  // U slices [slice][256 rows x 32 B]
constexpr int kP2TOp = 3 * 128 * 32;      // T slices [slice][rp rows x 32 B]
constexpr int kP2Stage = kP2Raw + kP2UOp + kP2TOp;
constexpr int kP2Depth = 4;

// format codes (hh_fmt order)
constexpr int kF32 = 1, kF16 = 2, kBF16 = 3, kE4M3 = 4;

__device__ __forceinline__ int fmt_size(int f) { return f == kF32 ? 4 : (f == kE4M3 ? 1 : 2); }
__device__ __forceinline__ int factor_slices(int f) { return f == kF32 ? 3 : (f == kF16 ? 2 : 1); }
__device__ __forceinline__ int input_slices(int f) { return f == kF32 ? 3 : 2; }
__device__ __forceinline__ int n_products(int f) { return f == kF32 ? 6 : (f == kF16 ? 3 : 2); }
// product p multiplies factor slice pf(p) with input slice px(p):
// (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
__device__ __forceinline__ int pf(int p) { return (0x210100 >> (4 * p)) & 0xf; }
__device__ __forceinline__ int px(int p) { return (0x012010 >> (4 * p)) & 0xf; }

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
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

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// exact split of an fp32 value into three bf16 slices
__device__ __forceinline__ void slice3(float v, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b);
  c = __float2bfloat16_rn(r2);
}

// eight values -> their first ns slices, 16 bytes each, at dst + s * sstride
__device__ __forceinline__ void store_slices(const float* v, int ns, uint8_t* dst, int64_t sstride) {
  __align__(16) __nv_bfloat16 s[3][8];
#pragma unroll
  for (int t = 0; t < 8; ++t) slice3(v[t], s[0][t], s[1][t], s[2][t]);
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(s[0]);
  if (ns > 1) *reinterpret_cast<uint4*>(dst + sstride) = *reinterpret_cast<const uint4*>(s[1]);
  if (ns > 2) *reinterpret_cast<uint4*>(dst + 2 * sstride) = *reinterpret_cast<const uint4*>(s[2]);
}

__device__ __forceinline__ float elem(const uint8_t* p, int fmt) {
  if (fmt == kF32) return *reinterpret_cast<const float*>(p);
  if (fmt == kF16) return __half2float(*reinterpret_cast<const __half*>(p));
  if (fmt == kBF16) return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
  __half_raw h = __nv_cvt_fp8_to_halfraw(*reinterpret_cast<const __nv_fp8_storage_t*>(p), __NV_E4M3);
  return __half2float(__half(h));
}

// byte offset of (row, 8-element group c of the K step) in a K-major operand tile
__device__ __forceinline__ int core_off(int row, int c) { return (row >> 3) * 256 + c * 128 + (row & 7) * 16; }

struct Ctl {
  uint64_t bar[4];
  uint32_t tmem;
  int abort;
  int inited[4];  // phase 2: [sub] main products, [2 + sub] correction products
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~static_cast<uintptr_t>(1023));
}

__device__ __forceinline__ void tc_begin(Ctl* c, int depth) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < depth; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&c->bar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    c->abort = 0;
    c->inited[0] = c->inited[1] = c->inited[2] = c->inited[3] = 0;
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

__device__ __forceinline__ void tc_end(Ctl* c) {
  cp_wait<0>();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c->tmem), "r"(kTmemCols));
}

// ------------------------------------------------------------------ phase 1
__global__ void __launch_bounds__(kThreads, 1) tc_phase1(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + kP1Depth * kP1Stage);
  const uint8_t** colp = reinterpret_cast<const uint8_t**>(ctl + 1);  // [256] column of each operand row
  int* rowpiece = reinterpret_cast<int*>(colp + 256);                 // [256] piece of each operand row
  const TcGroup g = a.groups[blockIdx.x];
  const int tid = threadIdx.x;
  for (int j = tid; j < 256; j += kThreads) {
    colp[j] = nullptr;
    rowpiece[j] = -1;
  }
  __syncthreads();
  if (tid < g.count) {
    const TcPiece& q = a.pieces[g.first + tid];
    const int sz = fmt_size(q.fmt);
    for (int j = 0; j < q.kp; ++j) {
      rowpiece[q.col + j] = g.first + tid;
      colp[q.col + j] = j < q.k ? q.f1 + static_cast<int64_t>(j) * q.ld1 * sz : nullptr;
    }
  }
  tc_begin(ctl, kP1Depth);
  const int fmt = g.fmt, sz = fmt_size(fmt), sf = factor_slices(fmt), sx = input_slices(fmt);
  const int np = n_products(fmt), nk = g.nk, rows = g.rows;
  const int nst = (rows + 31) / 32;
  const uint32_t idesc = idesc_bf16(nk);
  const int vslice = kP1Steps * nk * 32;  // bytes of one V slice (both steps)

  auto issue_loads = [&](int i) {
    if (i < nst) {
      uint8_t* st = base + (i % kP1Depth) * kP1Stage;
      const int p0 = 32 * i;
      const int64_t b0 = (static_cast<int64_t>(g.in_off) + p0) >> 4;
      for (int q = tid; q < sx * 2 * 256; q += kThreads) {
        const int sl = q >> 9, step = (q >> 8) & 1, pc = q & 255;
        cp16(st + (sl * 2 + step) * 4096 + pc * 16,
             a.ximg + ((static_cast<int64_t>(sl) * a.nblk + b0 + step) << 12) + pc * 16);
      }
      if (fmt == kBF16) {
        uint8_t* vop = st + kP1XOp;
        for (int q = tid; q < nk * 4; q += kThreads) {
          const int j = q >> 2, u = q & 3, pos = p0 + 8 * u;
          if (colp[j] && pos + 8 <= rows)
            cp16(vop + (u >> 1) * (nk * 32) + core_off(j, u & 1), colp[j] + 2 * pos);
        }
      } else {
        uint8_t* raw = st + kP1XOp + kP1VOp;
        const int per = 16 / sz, units = 2 * sz;  // positions per copy, copies per rank row
        for (int q = tid; q < nk * units; q += kThreads) {
          const int j = q / units, u = q - j * units, pos = p0 + u * per;
          if (colp[j] && pos < rows) cp16(raw + j * (32 * sz) + u * 16, colp[j] + static_cast<int64_t>(pos) * sz);
        }
      }
    }
    cp_commit();
  };

  for (int i = 0; i < kP1Depth - 1; ++i) issue_loads(i);
  bool ok = true;
  for (int i = 0; i < nst; ++i) {
    const int s = i % kP1Depth;
    uint8_t* st = base + s * kP1Stage;
    cp_wait<kP1Depth - 2>();
    __syncthreads();
    const int p0 = 32 * i;
    uint8_t* vop = st + kP1XOp;
    if (fmt == kBF16) {
      // rank rows and position groups that were not copied: zeros or the masked tail
      for (int q = tid; q < nk * 4; q += kThreads) {
        const int j = q >> 2, u = q & 3, pos = p0 + 8 * u;
        if (colp[j] && pos + 8 <= rows) continue;
        __align__(16) uint16_t e[8];
        const uint16_t* src = colp[j] ? reinterpret_cast<const uint16_t*>(colp[j]) + pos : nullptr;
#pragma unroll
        for (int t = 0; t < 8; ++t) e[t] = (src && pos + t < rows) ? src[t] : static_cast<uint16_t>(0);
        *reinterpret_cast<uint4*>(vop + (u >> 1) * (nk * 32) + core_off(j, u & 1)) =
            *reinterpret_cast<const uint4*>(e);
      }
    } else {
      const uint8_t* raw = st + kP1XOp + kP1VOp;
      for (int q = tid; q < nk * 4; q += kThreads) {
        const int j = q >> 2, u = q & 3, pos = p0 + 8 * u;
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t)
          v[t] = (colp[j] && pos + t < rows) ? elem(raw + j * (32 * sz) + (8 * u + t) * sz, fmt) : 0.f;
        store_slices(v, sf, vop + (u >> 1) * (nk * 32) + core_off(j, u & 1), vslice);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int step = 0; step < kP1Steps; ++step) {
        if (p0 + 16 * step >= rows) break;
        for (int p = 0; p < np; ++p) {
          const uint64_t da = op_desc(st + (px(p) * 2 + step) * 4096);
          const uint64_t db = op_desc(vop + pf(p) * vslice + step * (nk * 32));
          const uint32_t acc = p == 0 ? ((i | step) ? 1u : 0u) : ((i | step | (p - 1)) ? 1u : 0u);
          mma(ctl->tmem + (p ? kLoCol : 0), da, db, idesc, acc);
        }
      }
      mma_commit(&ctl->bar[s]);
    }
    // refill the stage that the previous iteration's MMAs read
    if (i >= 1 && i + kP1Depth - 1 < nst) {
      const int sp = (i - 1) % kP1Depth;
      if (!bar_wait(&ctl->bar[sp], ((i - 1) / kP1Depth) & 1)) ok = false;
    }
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    issue_loads(i + kP1Depth - 1);
  }
  if (ok && nst > 0 && !bar_wait(&ctl->bar[(nst - 1) % kP1Depth], ((nst - 1) / kP1Depth) & 1)) ok = false;
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicOr(a.status, 8);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: TMEM lane = right-hand side r, column = rank row of the group;
    // T = 2^e D in slices, written as the phase-2 operand image of the piece
    const int w = tid >> 5, lane = tid & 31;
    const int r = 32 * (w & 3) + lane;
    const uint32_t tbase = ctl->tmem + (static_cast<uint32_t>(32 * (w & 3)) << 16);
    for (int cb = (w >> 2); 16 * cb < nk; cb += 2) {
      float v[16], vl[16];
      tmem_ld16(tbase + 16 * cb, v);
      tmem_ld16(tbase + kLoCol + 16 * cb, vl);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] += vl[j];
      const TcPiece& q = a.pieces[rowpiece[16 * cb]];
      const int step = (16 * cb - q.col) >> 4;
      const int nsl = input_slices(q.fmt);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = ldexpf(v[j], q.e);
      uint8_t* dst = a.timg + q.toff + static_cast<int64_t>(step) * 4096 + core_off(r, 0);
      const int64_t sstride = static_cast<int64_t>(q.kp >> 4) * 4096;
      store_slices(v, nsl, dst, sstride);
      store_slices(v + 8, nsl, dst + 128, sstride);
    }
  }
  tc_end(ctl);
}

// ------------------------------------------------------------------ phase 2
struct Cursor {
  int e, step;
};

__global__ void __launch_bounds__(kThreads, 1) tc_phase2(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + kP2Depth * kP2Stage);
  const TcTile tl = a.tiles[blockIdx.x];
  const int tid = threadIdx.x, rp = a.rp;
  tc_begin(ctl, kP2Depth);
  int nst = 0;
  for (int e = 0; e < tl.count; ++e) nst += a.pieces[a.entries[tl.first + e].piece].kp >> 4;
  const uint32_t idesc = idesc_bf16(rp);

  Cursor ld_cur{0, 0};
  auto advance = [&](Cursor& c) {
    if (++c.step == (a.pieces[a.entries[tl.first + c.e].piece].kp >> 4)) {
      c.step = 0;
      ++c.e;
    }
  };
  auto issue_loads = [&](int i) {
    if (i < nst) {
      const TcEntry en = a.entries[tl.first + ld_cur.e];
      const TcPiece& q = a.pieces[en.piece];
      uint8_t* st = base + (i % kP2Depth) * kP2Stage;
      const int sz = fmt_size(q.fmt), nsl = input_slices(q.fmt);
      // T slices of this K step: the first rp rows (rp * 32 bytes) of each slice tile
      const uint8_t* tsrc = a.timg + q.toff + static_cast<int64_t>(ld_cur.step) * 4096;
      const int tunits = rp * 2;
      for (int u = tid; u < nsl * tunits; u += kThreads) {
        const int sl = u / tunits, w = u - sl * tunits;
        cp16(st + kP2Raw + kP2UOp + sl * 4096 + w * 16,
             tsrc + static_cast<int64_t>(sl) * (q.kp >> 4) * 4096 + w * 16);
      }
      // factor rows [src, src + nrows) of ranks 16*step .. +15: raw [rank][tile row]
      const int per = 16 / sz, units = (en.nrows + per - 1) / per;
      const int j0 = 16 * ld_cur.step;
      for (int u = tid; u < 16 * units; u += kThreads) {
        const int j = u / units, c = u - j * units;
        if (j0 + j < q.k)
          cp16(st + j * (kP2Rows * sz) + (en.dst + c * per) * sz,
               q.f2 + (static_cast<int64_t>(j0 + j) * q.ld2 + en.src + c * per) * sz);
      }
      advance(ld_cur);
    }
    cp_commit();
  };

  for (int i = 0; i < kP2Depth - 1; ++i) issue_loads(i);
  Cursor cu{0, 0};
  bool ok = true;
  int ini[4] = {0, 0, 0, 0};  // meaningful in thread 0
  for (int i = 0; i < nst; ++i) {
    const int s = i % kP2Depth;
    uint8_t* st = base + s * kP2Stage;
    const TcEntry en = a.entries[tl.first + cu.e];
    const TcPiece& q = a.pieces[en.piece];
    const int sz = fmt_size(q.fmt), sf = factor_slices(q.fmt), np = n_products(q.fmt);
    cp_wait<kP2Depth - 2>();
    __syncthreads();
    // convert: tile row m, ranks 16*step + 8c .. +7 -> slices of the K-major operand
    uint8_t* uop = st + kP2Raw;
    const int j0 = 16 * cu.step;
    for (int u = tid; u < 2 * kP2Rows; u += kThreads) {
      const int m = u >> 1, c = u & 1;
      const bool in = m >= en.dst && m < en.dst + en.nrows;
      float v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t)
        v[t] = (in && j0 + 8 * c + t < q.k) ? elem(st + (8 * c + t) * (kP2Rows * sz) + m * sz, q.fmt) : 0.f;
      store_slices(v, sf, uop + core_off(m, c), kP2Rows * 32);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int sub = 0; sub < 2; ++sub) {
        if (en.dst >= 128 * (sub + 1) || en.dst + en.nrows <= 128 * sub) continue;
        for (int p = 0; p < np; ++p) {
          const uint64_t da = op_desc(uop + pf(p) * (kP2Rows * 32) + sub * 4096);
          const uint64_t db = op_desc(st + kP2Raw + kP2UOp + px(p) * 4096);
          const int slot = (p ? 2 : 0) + sub;
          mma(ctl->tmem + (p ? kLoCol : 0) + 128 * sub, da, db, idesc, ini[slot] ? 1u : 0u);
          ini[slot] = 1;
        }
      }
      mma_commit(&ctl->bar[s]);
    }
    advance(cu);
    if (i >= 1 && i + kP2Depth - 1 < nst) {
      const int sp = (i - 1) % kP2Depth;
      if (!bar_wait(&ctl->bar[sp], ((i - 1) / kP2Depth) & 1)) ok = false;
    }
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    issue_loads(i + kP2Depth - 1);
  }
  if (tid == 0)
    for (int q = 0; q < 4; ++q) ctl->inited[q] = ini[q];
  if (ok && nst > 0 && !bar_wait(&ctl->bar[(nst - 1) % kP2Depth], ((nst - 1) / kP2Depth) & 1)) ok = false;
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicOr(a.status, 8);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warps 0-3 hold rows 0-127 of the tile, warps 4-7 rows 128-255
    const int w = tid >> 5, lane = tid & 31, sub = w >> 2;
    const int row = 128 * sub + 32 * (w & 3) + lane;
    const bool has_lo = ctl->inited[2 + sub] != 0;
    if (ctl->inited[sub]) {
      const uint32_t tbase = ctl->tmem + (static_cast<uint32_t>(32 * (w & 3)) << 16) + 128 * sub;
      for (int cb = 0; 16 * cb < rp; ++cb) {
        float v[16], vl[16];
        tmem_ld16(tbase + 16 * cb, v);
        if (has_lo) {
          tmem_ld16(tbase + kLoCol + 16 * cb, vl);
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] += vl[j];
        }
        if (row < tl.rows) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int rr = 16 * cb + j;
            if (rr < a.nr) a.acc[static_cast<int64_t>(rr) * a.npad + tl.row0 + row] += static_cast<double>(v[j]);
          }
        }
      }
    }
  }
  tc_end(ctl);
}

// X (caller's order, column-major, ld) -> tree order, fp32, bf16 slices in the
// phase-1 operand image [slice][16-position block][128 rows x 32 B]; rows
// r >= nr and positions >= n are zero.  Also clears the output accumulator.
__global__ void tc_prep_kernel(const double* __restrict__ x, int64_t ld, int nr, const int32_t* __restrict__ perm,
                               int64_t n, int64_t nblk, uint8_t* __restrict__ ximg, double* __restrict__ acc,
                               int64_t npad) {
  const int64_t total = nblk * 256;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total; q += stride) {
    const int64_t blk = q >> 8;
    const int c = static_cast<int>(q >> 7) & 1, r = static_cast<int>(q & 127);
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int64_t p = 16 * blk + 8 * c + t;
      v[t] = (r < nr && p < n) ? __double2float_rn(x[static_cast<int64_t>(perm[p]) + r * ld]) : 0.f;
    }
    store_slices(v, 3, ximg + (blk << 12) + core_off(r, c), nblk << 12);
  }
  const int64_t ntot = static_cast<int64_t>(nr) * npad;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < ntot; q += stride) acc[q] = 0.0;
}

}  // namespace

size_t tc_smem_bytes(int phase) {
  return (phase == 1 ? kP1Depth * kP1Stage : kP2Depth * kP2Stage) + 1024 + sizeof(Ctl) + 256 * 12;
}

cudaError_t launch_tc_prep(const double* x, int64_t ld, int nr, const int32_t* perm, int64_t n, int64_t nblk,
                           uint8_t* ximg, double* acc, int64_t npad, cudaStream_t st) {
  int64_t blocks = (nblk * 256 + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  tc_prep_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(x, ld, nr, perm, n, nblk, ximg, acc, npad);
  return cudaGetLastError();
}

cudaError_t launch_tc(int phase, const TcArgs& a, cudaStream_t st) {
  const size_t smem = tc_smem_bytes(phase);
  if (smem > 232448) return cudaErrorInvalidConfiguration;
  if (phase == 1) {
    if (a.n_groups <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(tc_phase1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_phase1<<<a.n_groups, kThreads, smem, st>>>(a);
  } else {
    if (a.n_tiles <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(tc_phase2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_phase2<<<a.n_tiles, kThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace hh
