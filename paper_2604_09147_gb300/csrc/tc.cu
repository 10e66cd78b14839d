// Tensor-core path (tcgen05, kind::f16 with bf16 operands) of the H_h product
// for many right-hand sides, for the low-rank blocks stored in fp16, bf16 or
// fp8-e4m3.  With R right-hand sides the two phases of Algorithm 4 become
// dense contractions,
//   phase 1  T_b = 2^(e_u+e_v) V_b^T X_J          (k_b x R, contraction over |J|)
//   phase 2  Y_I += U_b T_b                        (|I| x R, contraction over k_b)
// computed as
//   phase 1  one CTA per (group, position range): a group is the blocks of
//            one format sharing the input cluster J (at most 128 ranks);
//            D[r][col] = sum_p X[p][r] V[p][col], M = 128 right-hand sides,
//            N = the group's ranks, K = 16 positions per MMA.  Clusters longer
//            than 1,024 positions are split over several CTAs; each writes
//            its partial sums, and the CTA that arrives last (an atomic
//            counter, nothing waits) adds them in split order.
//   phase 2  one CTA per 128-row output tile: D[row][r] = sum over the blocks
//            covering the tile and their ranks of U[row][j] T[j][r], N = R,
//            added once into the fp64 output accumulator.
//
// Precision.  Operands are bf16 slices: fp16 factors are written exactly as
// s0 + s1 (s0 = bf16(v), s1 = bf16(v - s0)), bf16 and e4m3 factors as one
// slice; the input X (fp32 of the fp64 input) and T (fp32) as two slices,
// leaving about 2^-17 of the value.  Products kept: slice 0 x slice 0 (the
// main product) and 0 x 1 (and 1 x 0 for fp16).  Accumulation is fp32 in
// tensor memory, and it does not round to nearest: measured against exact
// sums its error grows with the number of MMAs that add into one
// accumulator, to about 2^-17 of a block's product over a few hundred MMAs.
// That is far below the unit roundoff of these formats (2^-11 and larger);
// fp32 blocks, whose unit roundoff is 2^-24, stay on the CUDA-core passes.
// The main products and the correction products accumulate in separate
// tensor-memory columns (0.. and 128..), so the small additions do not land
// on the large accumulator.
//
// Shared-memory operands use the K-major layout without swizzling: 8-row by
// 16-byte core matrices, the two core matrices of one 16-element K step 128
// bytes apart (leading byte offset) and successive 8-row groups 256 bytes
// apart (stride byte offset).  A stage is one K step; a ring of kDepth stages
// is filled with cp.async (16-byte copies) kDepth - 1 stages ahead.  In phase
// 1 every thread converts exactly the bytes it copied (raw factor bytes into
// bf16 slices); in phase 2, where U is transposed from columns to rows on the
// way, a stage's copies are complete one barrier before its conversion.
// Either way one barrier per stage publishes a stage to the thread that
// issues its MMAs;
// tcgen05.commit on the stage's mbarrier frees it.  About 100 KB of shared
// memory and 256 tensor-memory columns per CTA let two CTAs share an SM.
// Every mbarrier wait has a clock limit that sets bit 3 of the status word;
// an expired wait ends the CTA after its copies have landed and its tensor
// memory has been released.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "hh_device.h"

namespace hh {
namespace dev {

namespace {

constexpr int kThreads = 256;
constexpr long long kWaitCycles = 4000000000LL;
constexpr int kTmemCols = 256;
constexpr int kLoCol = 128;  // accumulator of the correction products
constexpr int kDepth = 5;

// phase 1 stage: one K step (16 positions)
constexpr int kP1XOp = 2 * 4096;                // X slices [slice][128 rows x 32 B]
constexpr int kP1VOp = 2 * kTcGroupRanks * 32;  // V slices [slice][nk rows x 32 B]
constexpr int kP1Raw = kTcGroupRanks * 32;      // raw factor bytes [nk ranks][16 positions]
constexpr int kP1Stage = kP1XOp + kP1VOp + kP1Raw;
// phase 2 stage: one K step (16 ranks) of a 128-row tile
constexpr int kP2Raw = 16 * kTcRows * 2;  // raw factor bytes [16 ranks][128 rows]
constexpr int kP2UOp = 2 * kTcRows * 32;  // U slices [slice][128 rows x 32 B]
constexpr int kP2TOp = 2 * 128 * 32;      // T slices [slice][rp rows x 32 B]
constexpr int kP2Stage = kP2Raw + kP2UOp + kP2TOp;

// format codes (hh_fmt order)
constexpr int kF16 = 2, kBF16 = 3, kE4M3 = 4;

__device__ __forceinline__ int fmt_size(int f) { return f == kE4M3 ? 1 : 2; }
__device__ __forceinline__ int factor_slices(int f) { return f == kF16 ? 2 : 1; }
__device__ __forceinline__ int n_products(int f) { return f == kF16 ? 3 : 2; }
// product p: factor slice pf(p) times input slice px(p): (0,0) (0,1) (1,0)
__device__ __forceinline__ int pf(int p) { return p == 2 ? 1 : 0; }
__device__ __forceinline__ int px(int p) { return p == 1 ? 1 : 0; }

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

// eight values -> their first ns (<= 2) bf16 slices, 16 bytes each, at dst + s * sstride
__device__ __forceinline__ void store_slices(const float* v, int ns, uint8_t* dst, int64_t sstride) {
  __align__(16) __nv_bfloat16 s[2][8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    s[0][t] = __float2bfloat16_rn(v[t]);
    s[1][t] = __float2bfloat16_rn(v[t] - __bfloat162float(s[0][t]));
  }
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(s[0]);
  if (ns > 1) *reinterpret_cast<uint4*>(dst + sstride) = *reinterpret_cast<const uint4*>(s[1]);
}

__device__ __forceinline__ float e4m3_to_float(uint8_t b) {
  __half_raw h = __nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(b), __NV_E4M3);
  return __half2float(__half(h));
}

__device__ __forceinline__ float f16_or_bf16(uint16_t b, int fmt) {
  if (fmt == kBF16) return __uint_as_float(static_cast<uint32_t>(b) << 16);
  __half_raw h;
  h.x = b;
  return __half2float(__half(h));
}

// byte offset of (row, 8-element group c of the K step) in a K-major operand tile
__device__ __forceinline__ int core_off(int row, int c) { return (row >> 3) * 256 + c * 128 + (row & 7) * 16; }

struct Ctl {
  uint64_t bar[kDepth];
  uint32_t tmem;
  int last;
  int inited[2];  // phase 2: main and correction accumulators written
};

__device__ __forceinline__ uint8_t* align128(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 127) & ~static_cast<uintptr_t>(127));
}

__device__ __forceinline__ void tc_begin(Ctl* c, uint32_t cols = kTmemCols) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kDepth; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&c->bar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    c->last = 0;
    c->inited[0] = c->inited[1] = 0;
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&c->tmem)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_end(Ctl* c, uint32_t cols = kTmemCols) {
  cp_wait<0>();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c->tmem), "r"(cols));
}

// T = 2^e D of 16 ranks of one right-hand side, as the two slices of the
// phase-2 operand image of its piece
// 16 columns of this warp's 32 lanes, without waiting (tcgen05.wait::ld follows)
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// exact split of an fp32 value into three bf16 slices
__device__ __forceinline__ void store_slices3(const float* v, uint8_t* dst, int64_t sstride) {
  __align__(16) __nv_bfloat16 s[3][8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    s[0][t] = __float2bfloat16_rn(v[t]);
    const float r1 = v[t] - __bfloat162float(s[0][t]);
    s[1][t] = __float2bfloat16_rn(r1);
    s[2][t] = __float2bfloat16_rn(r1 - __bfloat162float(s[1][t]));
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) *reinterpret_cast<uint4*>(dst + k * sstride) = *reinterpret_cast<const uint4*>(s[k]);
}

__device__ __forceinline__ void write_t(const TcArgs& a, const TcPiece& q, int cb16, int r, float* v) {
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = ldexpf(v[j], q.e);
  const int step = (cb16 - q.col) >> 4;
  uint8_t* dst = a.timg + q.toff + static_cast<int64_t>(step) * 4096 + core_off(r, 0);
  const int64_t sstride = static_cast<int64_t>(q.kp >> 4) * 4096;
  if (q.fmt == 1) {  // fp32 pieces: three slices
    store_slices3(v, dst, sstride);
    store_slices3(v + 8, dst + 128, sstride);
  } else {
    store_slices(v, 2, dst, sstride);
    store_slices(v + 8, 2, dst + 128, sstride);
  }
}

// ------------------------------------------------------------------ phase 1
__global__ void __launch_bounds__(kThreads, 2) tc_phase1(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align128(smem_raw);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + kDepth * kP1Stage);
  const uint8_t** colp = reinterpret_cast<const uint8_t**>(ctl + 1);  // [nk] column of each operand row
  int* rowpiece = reinterpret_cast<int*>(colp + kTcGroupRanks);       // [nk] piece of each operand row
  const TcGroup g = a.groups[blockIdx.x];
  const int tid = threadIdx.x;
  if (tid < g.count) {
    const TcPiece& q = a.pieces[g.first + tid];
    const int sz = fmt_size(q.fmt);
    for (int j = 0; j < q.kp; ++j) {
      rowpiece[q.col + j] = g.first + tid;
      colp[q.col + j] = j < q.k ? q.f1 + static_cast<int64_t>(j) * q.ld1 * sz : nullptr;
    }
  }
  tc_begin(ctl);  // its barrier also publishes colp / rowpiece
  const int fmt = g.fmt, sf = factor_slices(fmt), np = n_products(fmt), nk = g.nk;
  const int nst = (g.p1 - g.p0 + 15) >> 4;
  const uint32_t idesc = idesc_bf16(nk);
  // this thread's factor unit: 16-bit formats (rank j, 8 positions at 8c), e4m3 (rank j, 16 positions)
  const bool e4 = fmt == kE4M3;
  // consecutive threads take consecutive ranks: the 16-byte operand stores of a
  // quarter warp then fill one 128-byte line
  const int vj = e4 ? tid : (tid & 127), vc = e4 ? 0 : (tid >> 7);
  const bool vown = vj < nk && (e4 || true);
  const uint8_t* vcol = vown ? colp[vj] : nullptr;

  auto issue_loads = [&](int i) {
    if (i < nst) {
      uint8_t* st = base + (i % kDepth) * kP1Stage;
      const int p = g.p0 + 16 * i;
      const int64_t blk = (static_cast<int64_t>(g.in_off) + p) >> 4;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int u = tid + h * kThreads, sl = u >> 8, pc = u & 255;
        cp16(st + sl * 4096 + pc * 16, a.ximg + ((static_cast<int64_t>(sl) * a.nblk + blk) << 12) + pc * 16);
      }
      if (vcol) {
        if (fmt == kBF16) {
          const int pos = p + 8 * vc;
          if (pos + 8 <= g.p1) cp16(st + kP1XOp + core_off(vj, vc), vcol + 2 * pos);
        } else if (!e4) {
          const int pos = p + 8 * vc;
          if (pos < g.p1) cp16(st + kP1XOp + kP1VOp + vj * 32 + vc * 16, vcol + 2 * pos);
        } else {
          if (p < g.p1) cp16(st + kP1XOp + kP1VOp + vj * 16, vcol + p);
        }
      }
    }
    cp_commit();
  };
  // the operand bytes of this thread's factor unit for stage i: converted
  // slices, zeros, or the masked tail
  auto convert = [&](int i) {
    if (!vown) return;
    uint8_t* st = base + (i % kDepth) * kP1Stage;
    uint8_t* vop = st + kP1XOp;
    const int p = g.p0 + 16 * i;
    if (fmt == kBF16) {
      const int pos = p + 8 * vc;
      if (vcol && pos + 8 <= g.p1) return;  // copied in place
      __align__(16) uint16_t e[8];
      const uint16_t* src = vcol ? reinterpret_cast<const uint16_t*>(vcol) + pos : nullptr;
#pragma unroll
      for (int t = 0; t < 8; ++t) e[t] = (src && pos + t < g.p1) ? src[t] : static_cast<uint16_t>(0);
      *reinterpret_cast<uint4*>(vop + core_off(vj, vc)) = *reinterpret_cast<const uint4*>(e);
    } else if (!e4) {
      const int pos = p + 8 * vc;
      float v[8];
      const uint16_t* raw = reinterpret_cast<const uint16_t*>(st + kP1XOp + kP1VOp + vj * 32 + vc * 16);
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = (vcol && pos + t < g.p1) ? f16_or_bf16(raw[t], fmt) : 0.f;
      store_slices(v, sf, vop + core_off(vj, vc), nk * 32);
    } else {
      const uint8_t* raw = st + kP1XOp + kP1VOp + vj * 16;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = (vcol && p + 8 * c + t < g.p1) ? e4m3_to_float(raw[8 * c + t]) : 0.f;
        store_slices(v, 1, vop + core_off(vj, c), nk * 32);
      }
    }
  };

  for (int i = 0; i < kDepth - 1; ++i) issue_loads(i);
  bool ok = true;
  for (int i = 0; i < nst; ++i) {
    const int s = i % kDepth;
    uint8_t* st = base + s * kP1Stage;
    cp_wait<kDepth - 2>();
    convert(i);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int p = 0; p < np; ++p) {
        const uint64_t da = op_desc(st + px(p) * 4096);
        const uint64_t db = op_desc(st + kP1XOp + pf(p) * (nk * 32));
        const uint32_t acc = p == 0 ? (i ? 1u : 0u) : ((i || p > 1) ? 1u : 0u);
        mma(ctl->tmem + (p ? kLoCol : 0), da, db, idesc, acc);
      }
      mma_commit(&ctl->bar[s]);
    }
    // refill the stage the previous iteration's MMAs read
    if (i >= 1 && i + kDepth - 1 < nst && !bar_wait(&ctl->bar[(i - 1) % kDepth], ((i - 1) / kDepth) & 1))
      ok = false;
    issue_loads(i + kDepth - 1);
  }
  if (ok && nst > 0 && !bar_wait(&ctl->bar[(nst - 1) % kDepth], ((nst - 1) / kDepth) & 1)) ok = false;
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicOr(a.status, 8);
    tc_end(ctl);
    return;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: TMEM lane = right-hand side r, column = rank row of the group
  const int w = tid >> 5, lane = tid & 31;
  const int r = 32 * (w & 3) + lane;
  const uint32_t tbase = ctl->tmem + (static_cast<uint32_t>(32 * (w & 3)) << 16);
  const int64_t pstride = static_cast<int64_t>(128) * nk;  // floats of one split's partial sums
  for (int cb = (w >> 2); 16 * cb < nk; cb += 2) {
    float v[16], vl[16];
    tmem_ld16(tbase + 16 * cb, v);
    tmem_ld16(tbase + kLoCol + 16 * cb, vl);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] += vl[j];
    if (g.nsplit == 1) {
      write_t(a, a.pieces[rowpiece[16 * cb]], 16 * cb, r, v);
    } else {
      float4* dst = reinterpret_cast<float4*>(a.part + g.poff + static_cast<int64_t>(r) * nk + 16 * cb);
#pragma unroll
      for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
  }
  if (g.nsplit > 1) {
    __threadfence();
    __syncthreads();
    if (tid == 0) ctl->last = atomicAdd(a.cnt + g.gid, 1) == g.nsplit - 1;
    __syncthreads();
    if (ctl->last) {
      __threadfence();
      const float* p0 = a.part + g.poff - static_cast<int64_t>(g.split) * pstride;
      for (int cb = (w >> 2); 16 * cb < nk; cb += 2) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
        for (int sp = 0; sp < g.nsplit; ++sp) {
          const float4* src = reinterpret_cast<const float4*>(p0 + sp * pstride + static_cast<int64_t>(r) * nk + 16 * cb);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 f = __ldcg(src + j);
            v[4 * j] += f.x;
            v[4 * j + 1] += f.y;
            v[4 * j + 2] += f.z;
            v[4 * j + 3] += f.w;
          }
        }
        write_t(a, a.pieces[rowpiece[16 * cb]], 16 * cb, r, v);
      }
      if (tid == 0) a.cnt[g.gid] = 0;
    }
  }
  tc_end(ctl);
}

// ------------------------------------------------------------------ phase 2
// position in a tile's list of (entry, K step), with the current entry and
// the fields of its piece held in registers (reloaded when the entry changes)
struct Cursor {
  int e, step;
  TcEntry en;
  const uint8_t* f2;
  int64_t ld2, toff;
  int k, steps, fmt;
};

__device__ __forceinline__ void cursor_load(Cursor& c, const TcArgs& a, const TcTile& tl) {
  if (c.e >= tl.count) return;
  c.en = a.entries[tl.first + c.e];
  const TcPiece& q = a.pieces[c.en.piece];
  c.f2 = q.f2;
  c.ld2 = q.ld2;
  c.toff = q.toff;
  c.k = q.k;
  c.steps = q.kp >> 4;
  c.fmt = q.fmt;
}

__device__ __forceinline__ void cursor_advance(Cursor& c, const TcArgs& a, const TcTile& tl) {
  if (++c.step == c.steps) {
    c.step = 0;
    ++c.e;
    cursor_load(c, a, tl);
  }
}

__global__ void __launch_bounds__(kThreads, 2) tc_phase2(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align128(smem_raw);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + kDepth * kP2Stage);
  const TcTile tl = a.tiles[blockIdx.x];
  const int tid = threadIdx.x, rp = a.rp;
  tc_begin(ctl);
  int nst = 0;
  for (int e = 0; e < tl.count; ++e) nst += a.pieces[a.entries[tl.first + e].piece].kp >> 4;
  const uint32_t idesc = idesc_bf16(rp);

  Cursor ld{}, cv{}, mc{};
  cursor_load(ld, a, tl);
  cv = ld;
  mc = ld;
  // copies of stage i: the T slices (straight into the operand) and the raw
  // factor rows [src, src + nrows) of the 16 ranks of the K step, laid out
  // [rank][tile row]; thread = (rank, 16-byte piece of the rows)
  auto issue_loads = [&](int i) {
    if (i < nst) {
      const TcEntry& en = ld.en;
      uint8_t* st = base + (i % kDepth) * kP2Stage;
      const uint8_t* tsrc = a.timg + ld.toff + static_cast<int64_t>(ld.step) * 4096;
      const int tunits = rp * 2;
      for (int u = tid; u < 2 * tunits; u += kThreads) {
        const int sl = u >= tunits, w = u - sl * tunits;
        cp16(st + kP2Raw + kP2UOp + sl * 4096 + w * 16, tsrc + static_cast<int64_t>(sl) * ld.steps * 4096 + w * 16);
      }
      const int sz = fmt_size(ld.fmt), per = 16 / sz;  // rows per 16-byte piece
      const int pieces = kTcRows / per;                  // pieces per rank row of the tile
      const int j = tid / pieces, c = tid - j * pieces, m0 = c * per;
      const int jj = 16 * ld.step + j;
      if (j < 16 && jj < ld.k && m0 >= en.dst && m0 < en.dst + en.nrows)
        cp16(st + j * (kTcRows * sz) + m0 * sz, ld.f2 + (static_cast<int64_t>(jj) * ld.ld2 + en.src + (m0 - en.dst)) * sz);
      cursor_advance(ld, a, tl);
    }
    cp_commit();
  };
  // the U operand of stage i: thread = (tile row m, 8 ranks uo); slices, zeros
  // or the masked tail (every thread's copies of the stage have landed)
  auto convert = [&](int i) {
    if (i >= nst) return;
    const TcEntry& en = cv.en;
    uint8_t* st = base + (i % kDepth) * kP2Stage;
    const int m = tid & 127, uo = tid >> 7, sz = fmt_size(cv.fmt);
    const bool in = m >= en.dst && m < en.dst + en.nrows;
    const int j0 = 16 * cv.step + 8 * uo;
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const uint8_t* src = st + (8 * uo + t) * (kTcRows * sz) + m * sz;
      float x = 0.f;
      if (in && j0 + t < cv.k)
        x = cv.fmt == kE4M3 ? e4m3_to_float(*src) : f16_or_bf16(*reinterpret_cast<const uint16_t*>(src), cv.fmt);
      v[t] = x;
    }
    store_slices(v, factor_slices(cv.fmt), st + kP2Raw + core_off(m, uo), kTcRows * 32);
    cursor_advance(cv, a, tl);
  };

  for (int i = 0; i < kDepth - 1; ++i) issue_loads(i);
  cp_wait<kDepth - 2>();
  __syncthreads();
  convert(0);
  bool ok = true;
  int ini_hi = 0, ini_lo = 0;  // meaningful in thread 0
  for (int i = 0; i < nst; ++i) {
    const int s = i % kDepth;
    uint8_t* st = base + s * kP2Stage;
    cp_wait<kDepth - 3>();  // this thread's copies of stages <= i + 1
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      const int np = n_products(mc.fmt);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int p = 0; p < np; ++p) {
        const uint64_t da = op_desc(st + kP2Raw + pf(p) * (kTcRows * 32));
        const uint64_t db = op_desc(st + kP2Raw + kP2UOp + px(p) * 4096);
        int& ini = p ? ini_lo : ini_hi;
        mma(ctl->tmem + (p ? kLoCol : 0), da, db, idesc, ini ? 1u : 0u);
        ini = 1;
      }
      mma_commit(&ctl->bar[s]);
    }
    cursor_advance(mc, a, tl);
    if (i >= 1 && i + kDepth - 1 < nst && !bar_wait(&ctl->bar[(i - 1) % kDepth], ((i - 1) / kDepth) & 1))
      ok = false;
    issue_loads(i + kDepth - 1);
    convert(i + 1);
  }
  if (tid == 0) {
    ctl->inited[0] = ini_hi;
    ctl->inited[1] = ini_lo;
  }
  if (ok && nst > 0 && !bar_wait(&ctl->bar[(nst - 1) % kDepth], ((nst - 1) / kDepth) & 1)) ok = false;
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicOr(a.status, 8);
  } else if (ctl->inited[0]) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: TMEM lane = tile row, column = right-hand side; warps 4-7 take
    // the upper half of the columns
    const int w = tid >> 5, lane = tid & 31;
    const int row = 32 * (w & 3) + lane;
    const bool has_lo = ctl->inited[1] != 0;
    const uint32_t tbase = ctl->tmem + (static_cast<uint32_t>(32 * (w & 3)) << 16);
    for (int cb = 4 * (w >> 2); cb < 4 * (w >> 2) + 4 && 16 * cb < rp; ++cb) {
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
  tc_end(ctl);
}

// ------------------------------------------------------------------ fp32 blocks
// fp32 factors and inputs as three exact bf16 slices, six products (slice
// indices summing to at most 2).  Every pair of stages (32 terms of the
// contraction) starts a fresh pair of accumulators (main product,
// corrections) in one of two tensor-memory banks, and the drain warps add the
// finished bank into fp32 registers (round to nearest) while the next pair's
// MMAs fill the other bank: the tensor core's truncating accumulation acts on
// 32-term partial sums instead of growing with the length of the
// contraction, which keeps fp32 accuracy.
//
// Warp roles, no CTA-wide barrier inside the loop (each hand-off is an
// mbarrier with a bounded wait that also gives up when another role aborted):
//   warp 0     producer: copies of the stage's operand bytes into a
//              kWsDepth-deep ring (bulk copies for the contiguous input and T
//              slices and U rows, per-lane 16-byte cp.async for the 64-byte V
//              rows), completion counted on full[s]
//   warp 1     one thread issues the MMAs of a stage once it is converted
//              (conv[s]) and, for a pair's first stage, its bank is drained
//              (bempty[b]); tcgen05.commit frees the stage (empty[s]) and,
//              after a pair's second stage, hands the bank over (bfull[b])
//   warps 2-3  convert raw fp32 bytes into bf16 slices in the operand layout
//   warps 4-7  drain the banks (one tensor-memory lane quarter each) into
//              fp32 registers, then write the results
// ~195 KB of shared memory and 512 tensor-memory columns: one CTA per SM.
constexpr int kWsDepth = 6;
constexpr int kF1XOp = 3 * 4096;                   // X slices [3][128 rows x 32 B]
constexpr int kF1VOp = 3 * kTcGroupRanks * 32;     // V slices [3][nk rows x 32 B]
constexpr int kF1Raw = kTcGroupRanks * 64;         // raw fp32 V [4 chunks of 4 positions][nk ranks] x 16 B
constexpr int kF1Stage = kF1XOp + kF1VOp + kF1Raw;
constexpr int kF2Raw = 16 * kTcRows * 4;           // raw fp32 U [16 ranks][128 rows]
constexpr int kF2UOp = 3 * kTcRows * 32;           // U slices [3][128 rows x 32 B]
constexpr int kF2TOp = 3 * 128 * 32;               // T slices [3][rp rows x 32 B]
constexpr int kF2Stage = kF2Raw + kF2UOp + kF2TOp;
constexpr uint32_t kFTmemCols = 512;               // bank b: main at 256 b, corrections at 256 b + 128
// products: factor slice fpf(p) times input slice fpx(p): (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
__device__ __forceinline__ int fpf(int p) { return (0x210100 >> (4 * p)) & 0xf; }
__device__ __forceinline__ int fpx(int p) { return (0x012010 >> (4 * p)) & 0xf; }

struct WsCtl {
  uint64_t full[kWsDepth], conv[kWsDepth], empty[kWsDepth];
  uint64_t bfull[2], bempty[2];
  uint32_t tmem;
  int abort;
  int last;
};

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
__device__ __forceinline__ void bulk_copy_once(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                               uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar)), "l"(policy)
      : "memory");
}
// the mbarrier counts the completion of this thread's earlier cp.async copies
// (it raises the pending count first, so no arrival needs to be pre-counted)
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ uint64_t evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

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

__device__ __forceinline__ void ws_setup(WsCtl* c) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kWsDepth; ++s) {
      mbar_init(&c->full[s], 1);
      mbar_init(&c->conv[s], 2);
      mbar_init(&c->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&c->bfull[b], 1);
      mbar_init(&c->bempty[b], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    c->abort = 0;
    c->last = 0;
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&c->tmem)),
                 "r"(kFTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// after the role loops: on an abort the producer waits for the copies it
// issued and the MMA thread for its last MMAs, then tensor memory is freed
__device__ __forceinline__ void ws_teardown(WsCtl* c, int produced, int mmas, int* status) {
  asm volatile("cp.async.wait_all;" ::: "memory");  // the producer's per-lane copies (not in commit groups)
  __syncthreads();
  if (c->abort) {
    volatile int no = 0;
    if (threadIdx.x == 0)
      for (int i = produced > kWsDepth ? produced - kWsDepth : 0; i < produced; ++i)
        ws_wait(&c->full[i % kWsDepth], (i / kWsDepth) & 1, &no);
    if (threadIdx.x == 32 && mmas > 0) ws_wait(&c->empty[(mmas - 1) % kWsDepth], ((mmas - 1) / kWsDepth) & 1, &no);
    if (threadIdx.x == 0) atomicOr(status, 8);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c->tmem), "r"(kFTmemCols));
}

// drain warps: add bank b (this lane, columns 0 .. ncols) into acc, 32
// columns (main and corrections) per tcgen05.wait::ld
__device__ __forceinline__ void ws_drain(const WsCtl* c, int bank, int ncols, float* acc) {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int w = threadIdx.x >> 5;
  const uint32_t t = c->tmem + (static_cast<uint32_t>(32 * (w & 3)) << 16) + 256 * bank;
#pragma unroll
  for (int cb = 0; cb < 4; ++cb) {
    if (32 * cb < ncols) {
      uint32_t h0[16], h1[16], l0[16], l1[16];
      tmem_ld16_nowait(t + 32 * cb, h0);
      tmem_ld16_nowait(t + 32 * cb + 16, h1);
      tmem_ld16_nowait(t + 128 + 32 * cb, l0);
      tmem_ld16_nowait(t + 128 + 32 * cb + 16, l1);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        acc[32 * cb + j] += __uint_as_float(h0[j]) + __uint_as_float(l0[j]);
        acc[32 * cb + 16 + j] += __uint_as_float(h1[j]) + __uint_as_float(l1[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1) tc_phase1_f32(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align128(smem_raw);
  WsCtl* c = reinterpret_cast<WsCtl*>(base + kWsDepth * kF1Stage);
  const uint8_t** colp = reinterpret_cast<const uint8_t**>(c + 1);
  int* rowpiece = reinterpret_cast<int*>(colp + kTcGroupRanks);
  const TcGroup g = a.groups[blockIdx.x];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  if (tid < g.count) {
    const TcPiece& q = a.pieces[g.first + tid];
    for (int j = 0; j < q.kp; ++j) {
      rowpiece[q.col + j] = g.first + tid;
      colp[q.col + j] = j < q.k ? q.f1 + static_cast<int64_t>(j) * q.ld1 * 4 : nullptr;
    }
  }
  ws_setup(c);  // its barrier also publishes colp / rowpiece
  const int nk = g.nk;
  const int nst = (g.p1 - g.p0 + 15) >> 4;
  volatile int* abort = &c->abort;
  int produced = 0, mmas = 0;
  float acc[128];
#pragma unroll
  for (int j = 0; j < 128; ++j) acc[j] = 0.f;

  if (w == 0) {  // producer: V rows by cp.async (16 bytes per lane copy), X slices by bulk copy
    for (int i = 0; i < nst; ++i) {
      const int s = i % kWsDepth;
      if (i >= kWsDepth && !ws_wait(&c->empty[s], ((i / kWsDepth) - 1) & 1, abort)) break;
      uint8_t* st = base + s * kF1Stage;
      const int p = g.p0 + 16 * i;
      const int64_t blk = (static_cast<int64_t>(g.in_off) + p) >> 4;
      for (int j = lane; j < nk; j += 32)
        if (colp[j]) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (p + 4 * q < g.p1)
              cp16(st + kF1XOp + kF1VOp + (q * nk + j) * 16, colp[j] + 4 * static_cast<int64_t>(p + 4 * q));
        }
      cp_async_arrive(&c->full[s]);
      __syncwarp();
      if (lane == 0) {
        mbar_expect_tx(&c->full[s], 3u * 4096u);
        for (int sl = 0; sl < 3; ++sl)
          bulk_copy(st + sl * 4096, a.ximg + ((static_cast<int64_t>(sl) * a.nblk + blk) << 12), 4096, &c->full[s]);
      }
      produced = i + 1;
    }
  } else if (w == 1) {  // MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(nk);
      for (int i = 0; i < nst; ++i) {
        // banks alternate per pair of stages: the pair's first stage starts
        // fresh accumulators, the second adds to them, then the bank is drained
        const int s = i % kWsDepth, q = i >> 1, b = q & 1, second = i & 1;
        // the stage's bulk copies (operands the converters do not touch) and its conversion
        if (!ws_wait(&c->full[s], (i / kWsDepth) & 1, abort)) break;
        if (!ws_wait(&c->conv[s], (i / kWsDepth) & 1, abort)) break;
        if (!second && q >= 2 && !ws_wait(&c->bempty[b], ((q >> 1) - 1) & 1, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint8_t* st = base + s * kF1Stage;
        const uint32_t tb = c->tmem + 256 * b;
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const uint64_t da = op_desc(st + fpx(p) * 4096);
          const uint64_t db = op_desc(st + kF1XOp + fpf(p) * (nk * 32));
          mma(tb + (p ? 128 : 0), da, db, idesc, (p >= 2 || second) ? 1u : 0u);
        }
        mma_commit(&c->empty[s]);
        if (second || i == nst - 1) mma_commit(&c->bfull[b]);
        mmas = i + 1;
      }
    }
  } else if (w < 4) {  // converters
    const int ct = tid - 64;
    for (int i = 0; i < nst; ++i) {
      const int s = i % kWsDepth;
      if (!ws_wait(&c->full[s], (i / kWsDepth) & 1, abort)) break;
      uint8_t* st = base + s * kF1Stage;
      const int p = g.p0 + 16 * i;
      for (int u = ct; u < 2 * nk; u += 64) {
        const int j = u < nk ? u : u - nk, half = u < nk ? 0 : 1, pos = p + 8 * half;
        // chunks 2 half and 2 half + 1 of rank j (a quarter warp reads 128 contiguous bytes)
        const float4 r0 = *reinterpret_cast<const float4*>(st + kF1XOp + kF1VOp + ((2 * half) * nk + j) * 16);
        const float4 r1 = *reinterpret_cast<const float4*>(st + kF1XOp + kF1VOp + ((2 * half + 1) * nk + j) * 16);
        const float raw[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        const bool live = colp[j] != nullptr;
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = (live && pos + t < g.p1) ? raw[t] : 0.f;
        store_slices3(v, st + kF1XOp + core_off(j, half), nk * 32);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&c->conv[s]);
    }
  } else {  // drain warps
    for (int q = 0; 2 * q < nst; ++q) {
      const int b = q & 1;
      if (!ws_wait(&c->bfull[b], (q >> 1) & 1, abort)) break;
      ws_drain(c, b, nk, acc);
      __syncwarp();
      if (lane == 0) mbar_arrive(&c->bempty[b]);
    }
  }
  if (__syncthreads_or(c->abort)) {
    ws_teardown(c, produced, mmas, a.status);
    return;
  }
  // epilogue (drain warps): right-hand side r, ranks 0 .. nk of the group
  const int r = 32 * (w & 3) + lane;
  const int64_t pstride = static_cast<int64_t>(128) * nk;
  if (w >= 4) {
#pragma unroll
    for (int cb = 0; cb < 8; ++cb) {
      const int c16 = 16 * cb;
      if (c16 >= nk) break;
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = acc[c16 + j];
      if (g.nsplit == 1) {
        write_t(a, a.pieces[rowpiece[c16]], c16, r, v);
      } else {
        float4* dst = reinterpret_cast<float4*>(a.part + g.poff + static_cast<int64_t>(r) * nk + c16);
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      }
    }
  }
  if (g.nsplit > 1) {
    __threadfence();
    __syncthreads();
    if (tid == 0) c->last = atomicAdd(a.cnt + g.gid, 1) == g.nsplit - 1;
    __syncthreads();
    if (c->last && w >= 4) {
      __threadfence();
      const float* p0 = a.part + g.poff - static_cast<int64_t>(g.split) * pstride;
      for (int cb = 0; cb < 8; ++cb) {
        const int c16 = 16 * cb;
        if (c16 >= nk) break;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
        for (int sp = 0; sp < g.nsplit; ++sp) {
          const float4* src = reinterpret_cast<const float4*>(p0 + sp * pstride + static_cast<int64_t>(r) * nk + c16);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 f = __ldcg(src + j);
            v[4 * j] += f.x;
            v[4 * j + 1] += f.y;
            v[4 * j + 2] += f.z;
            v[4 * j + 3] += f.w;
          }
        }
        write_t(a, a.pieces[rowpiece[c16]], c16, r, v);
      }
    }
    if (c->last && tid == 0) a.cnt[g.gid] = 0;
  }
  ws_teardown(c, produced, mmas, a.status);
}

__global__ void __launch_bounds__(kThreads, 1) tc_phase2_f32(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align128(smem_raw);
  WsCtl* c = reinterpret_cast<WsCtl*>(base + kWsDepth * kF2Stage);
  const TcTile tl = a.tiles[blockIdx.x];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, rp = a.rp;
  ws_setup(c);
  int nst = 0;
  for (int e = 0; e < tl.count; ++e) nst += a.pieces[a.entries[tl.first + e].piece].kp >> 4;
  volatile int* abort = &c->abort;
  int produced = 0, mmas = 0;
  float acc[128];
#pragma unroll
  for (int j = 0; j < 128; ++j) acc[j] = 0.f;

  if (w == 0) {  // producer: T slices (rp rows each) and the raw fp32 U rows of 16 ranks
    Cursor ld{};
    cursor_load(ld, a, tl);
    const uint64_t pol = evict_first();
    for (int i = 0; i < nst; ++i) {
      const int s = i % kWsDepth;
      if (i >= kWsDepth && !ws_wait(&c->empty[s], ((i / kWsDepth) - 1) & 1, abort)) break;
      uint8_t* st = base + s * kF2Stage;
      const TcEntry& en = ld.en;
      const int nj = min(16, ld.k - 16 * ld.step);
      const uint32_t segb = 16u * static_cast<uint32_t>((en.nrows + 3) >> 2);
      if (lane == 0) mbar_expect_tx(&c->full[s], 3u * static_cast<uint32_t>(rp) * 32u + static_cast<uint32_t>(nj) * segb);
      __syncwarp();
      if (lane < 3)
        bulk_copy(st + kF2Raw + kF2UOp + lane * 4096,
                  a.timg + ld.toff + (static_cast<int64_t>(lane) * ld.steps + ld.step) * 4096,
                  static_cast<uint32_t>(rp) * 32u, &c->full[s]);
      if (lane < nj)
        bulk_copy_once(st + (lane * kTcRows + en.dst) * 4,
                       ld.f2 + (static_cast<int64_t>(16 * ld.step + lane) * ld.ld2 + en.src) * 4, segb, &c->full[s],
                       pol);
      cursor_advance(ld, a, tl);
      produced = i + 1;
    }
  } else if (w == 1) {  // MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(rp);
      for (int i = 0; i < nst; ++i) {
        // banks alternate per pair of stages: the pair's first stage starts
        // fresh accumulators, the second adds to them, then the bank is drained
        const int s = i % kWsDepth, q = i >> 1, b = q & 1, second = i & 1;
        // the stage's bulk copies (operands the converters do not touch) and its conversion
        if (!ws_wait(&c->full[s], (i / kWsDepth) & 1, abort)) break;
        if (!ws_wait(&c->conv[s], (i / kWsDepth) & 1, abort)) break;
        if (!second && q >= 2 && !ws_wait(&c->bempty[b], ((q >> 1) - 1) & 1, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint8_t* st = base + s * kF2Stage;
        const uint32_t tb = c->tmem + 256 * b;
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const uint64_t da = op_desc(st + kF2Raw + fpf(p) * (kTcRows * 32));
          const uint64_t db = op_desc(st + kF2Raw + kF2UOp + fpx(p) * 4096);
          mma(tb + (p ? 128 : 0), da, db, idesc, (p >= 2 || second) ? 1u : 0u);
        }
        mma_commit(&c->empty[s]);
        if (second || i == nst - 1) mma_commit(&c->bfull[b]);
        mmas = i + 1;
      }
    }
  } else if (w < 4) {  // converters: U rows from [rank][row] to K-major slices
    const int ct = tid - 64;
    Cursor cv{};
    cursor_load(cv, a, tl);
    for (int i = 0; i < nst; ++i) {
      const int s = i % kWsDepth;
      if (!ws_wait(&c->full[s], (i / kWsDepth) & 1, abort)) break;
      uint8_t* st = base + s * kF2Stage;
      const TcEntry& en = cv.en;
      const float* raw = reinterpret_cast<const float*>(st);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int u = ct + 64 * k, m = u & 127, uo = u >> 7;
        const bool in = m >= en.dst && m < en.dst + en.nrows;
        const int j0 = 16 * cv.step + 8 * uo;
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = (in && j0 + t < cv.k) ? raw[(8 * uo + t) * kTcRows + m] : 0.f;
        store_slices3(v, st + kF2Raw + core_off(m, uo), kTcRows * 32);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&c->conv[s]);
      cursor_advance(cv, a, tl);
    }
  } else {  // drain warps
    for (int q = 0; 2 * q < nst; ++q) {
      const int b = q & 1;
      if (!ws_wait(&c->bfull[b], (q >> 1) & 1, abort)) break;
      ws_drain(c, b, rp, acc);
      __syncwarp();
      if (lane == 0) mbar_arrive(&c->bempty[b]);
    }
  }
  if (__syncthreads_or(c->abort)) {
    ws_teardown(c, produced, mmas, a.status);
    return;
  }
  // epilogue (drain warps): tile row of this lane, right-hand sides 0 .. rp
  if (w >= 4 && nst > 0) {
    const int row = 32 * (w & 3) + lane;
    if (row < tl.rows) {
#pragma unroll
      for (int j = 0; j < 128; ++j)
        if (j < a.nr) a.acc[static_cast<int64_t>(j) * a.npad + tl.row0 + row] += static_cast<double>(acc[j]);
    }
  }
  ws_teardown(c, produced, mmas, a.status);
}

// X (caller's order, column-major, ld) -> tree order, fp32, three bf16 slices in
// the phase-1 operand image [slice][16-position block][128 rows x 32 B]; rows
// r >= nr and positions >= n are zero.  Also clears the output accumulator
// and the arrival counters of the split groups.
__global__ void tc_prep_kernel(const double* __restrict__ x, int64_t ld, int nr, const int32_t* __restrict__ perm,
                               int64_t n, int64_t nblk, uint8_t* __restrict__ ximg, double* __restrict__ acc,
                               int64_t npad, int* __restrict__ cnt, int n_cnt) {
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
      v[t] = (r < nr && p < n) ? __double2float_rn(x[static_cast<int64_t>(perm[p]) + r * ld]) : 0.f;
    }
    store_slices3(v, ximg + (blk << 12) + core_off(r, c), nblk << 12);
  }
  const int64_t ntot = static_cast<int64_t>(nr) * npad;
  for (int64_t q = t0; q < ntot; q += stride) acc[q] = 0.0;
  for (int64_t q = t0; q < n_cnt; q += stride) cnt[q] = 0;
}

}  // namespace

size_t tc_smem_bytes(int phase) {
  return (phase == 1 ? kDepth * kP1Stage : kDepth * kP2Stage) + 128 + sizeof(Ctl) + kTcGroupRanks * 12;
}

cudaError_t launch_tc_prep(const double* x, int64_t ld, int nr, const int32_t* perm, int64_t n, int64_t nblk,
                           uint8_t* ximg, double* acc, int64_t npad, int* cnt, int n_cnt, cudaStream_t st) {
  int64_t blocks = (nblk * 256 + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  tc_prep_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(x, ld, nr, perm, n, nblk, ximg, acc, npad, cnt, n_cnt);
  return cudaGetLastError();
}

cudaError_t launch_tc(int phase, const TcArgs& a, cudaStream_t st, bool f32) {
  if (a.rp < 16 || a.rp > 128 || (a.rp & 15)) return cudaErrorInvalidValue;
  if (f32) {
    const size_t smem =
        (phase == 1 ? kWsDepth * kF1Stage : kWsDepth * kF2Stage) + 128 + sizeof(WsCtl) + kTcGroupRanks * 12;
    if (phase == 1) {
      if (a.n_groups <= 0) return cudaSuccess;
      cudaError_t e = cudaFuncSetAttribute(tc_phase1_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      tc_phase1_f32<<<a.n_groups, kThreads, smem, st>>>(a);
    } else {
      if (a.n_tiles <= 0) return cudaSuccess;
      cudaError_t e = cudaFuncSetAttribute(tc_phase2_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      tc_phase2_f32<<<a.n_tiles, kThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
  }
  const size_t smem = tc_smem_bytes(phase);
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
