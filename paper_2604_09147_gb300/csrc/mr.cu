// CUDA-core products for many right-hand sides (32 to 128 per launch): the
// blocks the tensor-core path leaves to the CUDA cores, computed with every
// right-hand side in one pass over their bytes.
//
//   mr_phase1  T_b = 2^(e_u+e_v) V_b^T X_J for the 32-, 16- and 8-bit blocks
//              outside the tensor-core path (fp32 blocks, and 16/8-bit blocks
//              on clusters that do not start at multiples of 16): one CTA per
//              (group of at most 64 ranks sharing the input cluster, range of
//              at most 1,024 positions); a thread holds 8 ranks x RPT
//              right-hand sides.  Factors are upcast to fp32, the input is
//              fp32 (relative 2^-24), products and sums are fp32 with round
//              to nearest; split ranges add into T with atomics.
//   mr_phase2  Y_I += U_b T_b for the same blocks: one CTA per 128-row output
//              tile over every such block covering it; a thread holds 8 rows
//              x RPT right-hand sides.
// The tiles of phase 2 add into the fp64 output
// accumulator with plain read-modify-writes: within one launch every output
// row belongs to one CTA, and launches are ordered on the stream.  Operands
// are staged through shared memory with register double buffering (the loads
// of stage i + 1 are in flight while stage i is computed), which needs no
// alignment of the clusters.
#include "hh_device.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

namespace hh {
namespace dev {

namespace {

constexpr int kThreads = 256;
constexpr int kK1 = 32;       // positions per phase-1 stage
constexpr int kK2 = 16;       // ranks (dense: K columns) per phase-2 stage

constexpr int kF32 = 1, kBF16 = 3, kE4M3 = 4;

__device__ __forceinline__ int fsize(int f) { return f == kF32 ? 4 : (f == kE4M3 ? 1 : 2); }

__device__ __forceinline__ float load_elem(const uint8_t* base, int64_t i, int fmt) {
  if (fmt == kF32) return __ldg(reinterpret_cast<const float*>(base) + i);
  if (fmt == kE4M3) {
    __half_raw h = __nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(__ldg(base + i)), __NV_E4M3);
    return __half2float(__half(h));
  }
  const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(base) + i);
  if (fmt == kBF16) return __uint_as_float(static_cast<uint32_t>(b) << 16);
  __half_raw h;
  h.x = b;
  return __half2float(__half(h));
}

// right-hand side of element e of thread column tc (RPT = 8: two float4 64
// columns apart, so a quarter warp reads 128 consecutive bytes)
template <int RPT>
__device__ __forceinline__ int rhs_col(int tc, int e) {
  if (RPT == 8) return (e >> 2) * 64 + 4 * tc + (e & 3);
  return RPT * tc + e;
}

template <int RPT>
__device__ __forceinline__ void load_x(const float* row, int tc, float* x) {
  if (RPT == 8) {
    const float4 a = *reinterpret_cast<const float4*>(row + 4 * tc);
    const float4 b = *reinterpret_cast<const float4*>(row + 64 + 4 * tc);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
  } else if (RPT == 4) {
    const float4 a = *reinterpret_cast<const float4*>(row + 4 * tc);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
  } else {
    const float2 a = *reinterpret_cast<const float2*>(row + 2 * tc);
    x[0] = a.x; x[1] = a.y;
  }
}

// ------------------------------------------------------------------ phase 1
constexpr int kP1Threads = 128;
constexpr int kVRow = kMrRanks + 4;  // floats per position row of the V stage

template <int RPT>
__global__ void __launch_bounds__(kP1Threads) mr_phase1(MrArgs a) {
  constexpr int RP = 16 * RPT;
  extern __shared__ __align__(16) float sm1[];
  float* sV = sm1;                        // [2][kK1][kVRow]: V transposed, position-major
  float* sX = sm1 + 2 * kK1 * kVRow;      // [2][kK1][RP]
  __shared__ const uint8_t* colp[kMrRanks];
  __shared__ int rowpiece[kMrRanks];
  const TcGroup g = a.groups[blockIdx.x];
  const int tid = threadIdx.x;
  if (tid < kMrRanks) {
    colp[tid] = nullptr;
    rowpiece[tid] = -1;
  }
  __syncthreads();
  if (tid < g.count) {
    const TcPiece& q = a.pieces[g.first + tid];
    const int sz = fsize(q.fmt);
    for (int j = 0; j < q.kp; ++j) {
      rowpiece[q.col + j] = g.first + tid;
      colp[q.col + j] = j < q.k ? q.f1 + static_cast<int64_t>(j) * q.ld1 * sz : nullptr;
    }
  }
  __syncthreads();
  const int fmt = g.fmt, nst = (g.p1 - g.p0 + kK1 - 1) / kK1;
  // loader roles: V rank vj, positions 16 vh .. 16 vh + 15 of the stage (a warp
  // covers 32 consecutive ranks, so the transposed stores are conflict-free)
  const int vj = tid & 63, vh = tid >> 6;
  const uint8_t* vcol = colp[vj];
  constexpr int XU = kK1 * RP / 4 / kP1Threads;  // float4 units of X per thread
  float vr[16];
  float4 xr[XU];
  auto load = [&](int i) {
    const int pos = g.p0 + kK1 * i + 16 * vh;
    if (fmt == 1 && vcol && pos + 16 <= g.p1) {
      const float4* src = reinterpret_cast<const float4*>(vcol) + (pos >> 2);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float4 f = __ldg(src + t);
        vr[4 * t] = f.x;
        vr[4 * t + 1] = f.y;
        vr[4 * t + 2] = f.z;
        vr[4 * t + 3] = f.w;
      }
    } else {
#pragma unroll
      for (int t = 0; t < 16; ++t) vr[t] = (vcol && pos + t < g.p1) ? load_elem(vcol, pos + t, fmt) : 0.f;
    }
    const int P = g.p0 + kK1 * i;
#pragma unroll
    for (int h = 0; h < XU; ++h) {
      const int u = tid + h * kP1Threads, p = u / (RP / 4), c4 = u - p * (RP / 4);
      xr[h] = *reinterpret_cast<const float4*>(a.xh + (static_cast<int64_t>(g.in_off) + P + p) * 128 + 4 * c4);
    }
  };
  auto store = [&](int buf) {
    float* v = sV + (buf * kK1 + 16 * vh) * kVRow + vj;
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t * kVRow] = vr[t];
#pragma unroll
    for (int h = 0; h < XU; ++h) {
      const int u = tid + h * kP1Threads, p = u / (RP / 4), c4 = u - p * (RP / 4);
      *reinterpret_cast<float4*>(sX + (buf * kK1 + p) * RP + 4 * c4) = xr[h];
    }
  };
  // thread tile: ranks 8 tr .. 8 tr + 7 (two float4 32 ranks apart), columns of tc
  const int tr = tid >> 4, tc = tid & 15;
  float acc[8][RPT];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int e = 0; e < RPT; ++e) acc[i][e] = 0.f;
  load(0);
  store(0);
  __syncthreads();
  for (int i = 0; i < nst; ++i) {
    const int buf = i & 1;
    if (i + 1 < nst) load(i + 1);
    const float* V = sV + buf * kK1 * kVRow + 4 * tr;
    const float* X = sX + buf * kK1 * RP;
#pragma unroll 4
    for (int p = 0; p < kK1; ++p) {
      float x[RPT];
      load_x<RPT>(X + p * RP, tc, x);
      const float4 va = *reinterpret_cast<const float4*>(V + p * kVRow);
      const float4 vb = *reinterpret_cast<const float4*>(V + p * kVRow + 32);
      const float v[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int e = 0; e < RPT; ++e) acc[r][e] = fmaf(v[r], x[e], acc[r][e]);
    }
    if (i + 1 < nst) store(buf ^ 1);
    __syncthreads();
  }
  // T = 2^e D, rank-major [rank][128] per piece
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int rank = (r < 4 ? 4 * tr + r : 32 + 4 * tr + r - 4);
    const int pi = rowpiece[rank];
    if (pi < 0) continue;
    const TcPiece& q = a.pieces[pi];
    const int rl = rank - q.col;
    if (rl >= q.k) continue;
    float* t = a.t32 + q.toff + static_cast<int64_t>(rl) * 128;
#pragma unroll
    for (int e = 0; e < RPT; ++e) {
      const float v = ldexpf(acc[r][e], q.e);
      if (g.nsplit > 1)
        atomicAdd(t + rhs_col<RPT>(tc, e), v);
      else
        t[rhs_col<RPT>(tc, e)] = v;
    }
  }
}

// ------------------------------------------------------------------ phase 2
// epilogue of a 128 x RP (or 64 x RP) tile: through shared memory so that the
// fp64 read-modify-writes of the output run along rows
template <int RPT, int ROWS, int RPTHR>
__device__ __forceinline__ void add_tile(const MrArgs& a, const TcTile& tl, float* sAcc, const float (*acc)[RPT],
                                         int tr, int tc) {
  constexpr int RP = 16 * RPT;
  constexpr int HALF = RP > 64 ? 64 : RP;
  for (int h = 0; h < RP / HALF; ++h) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RPTHR; ++i)
#pragma unroll
      for (int e = 0; e < RPT; ++e) {
        const int c = rhs_col<RPT>(tc, e) - h * HALF;
        if (c >= 0 && c < HALF) sAcc[(RPTHR * tr + i) * (HALF + 1) + c] = acc[i][e];
      }
    __syncthreads();
    for (int u = threadIdx.x; u < ROWS * HALF; u += kThreads) {
      const int row = u % ROWS, c = u / ROWS, rr = h * HALF + c;
      if (row < tl.rows && rr < a.nr)
        a.acc[static_cast<int64_t>(rr) * a.npad + tl.row0 + row] += static_cast<double>(sAcc[row * (HALF + 1) + c]);
    }
  }
}

struct Cur {
  int e, chunk;
};

template <int RPT>
__global__ void __launch_bounds__(kThreads, 2) mr_phase2(MrArgs a) {
  constexpr int RP = 16 * RPT;
  extern __shared__ __align__(16) float sm2[];
  float* sU = sm2;                      // [2][kK2][128]
  float* sT = sm2 + 2 * kK2 * kMrRows;  // [2][kK2][RP]
  const TcTile tl = a.tiles[blockIdx.x];
  const int tid = threadIdx.x;
  int nst = 0;
  for (int e = 0; e < tl.count; ++e) nst += (a.pieces[a.entries[tl.first + e].piece].kp + kK2 - 1) / kK2;
  // loader roles: U rank uj, tile rows 8 um .. 8 um + 7; T units
  const int uj = tid >> 4, um = tid & 15;
  constexpr int TU = kK2 * RP / 4 / kThreads > 0 ? kK2 * RP / 4 / kThreads : 1;
  float ur[8];
  float4 trg[TU];
  Cur lc{0, 0};
  auto load = [&]() {
    const TcEntry en = a.entries[tl.first + lc.e];
    const TcPiece& q = a.pieces[en.piece];
    const int j = kK2 * lc.chunk + uj;
    const bool jin = j < q.k;
    const int sz = fsize(q.fmt);
    const uint8_t* col = q.f2 + static_cast<int64_t>(j) * q.ld2 * sz;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int m = 8 * um + t;
      ur[t] = (jin && m >= en.dst && m < en.dst + en.nrows) ? load_elem(col, en.src + (m - en.dst), q.fmt) : 0.f;
    }
#pragma unroll
    for (int h = 0; h < TU; ++h) {
      const int u = tid + h * kThreads;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (u < kK2 * RP / 4) {
        const int r = u / (RP / 4), c4 = u - r * (RP / 4), jj = kK2 * lc.chunk + r;
        if (jj < q.k) v = *reinterpret_cast<const float4*>(a.t32 + q.toff + static_cast<int64_t>(jj) * 128 + 4 * c4);
      }
      trg[h] = v;
    }
    if (++lc.chunk == (q.kp + kK2 - 1) / kK2) {
      lc.chunk = 0;
      ++lc.e;
    }
  };
  auto store = [&](int buf) {
    float* u = sU + (buf * kK2 + uj) * kMrRows + 8 * um;
    *reinterpret_cast<float4*>(u) = make_float4(ur[0], ur[1], ur[2], ur[3]);
    *reinterpret_cast<float4*>(u + 4) = make_float4(ur[4], ur[5], ur[6], ur[7]);
#pragma unroll
    for (int h = 0; h < TU; ++h) {
      const int u2 = tid + h * kThreads;
      if (u2 < kK2 * RP / 4) {
        const int r = u2 / (RP / 4), c4 = u2 - r * (RP / 4);
        *reinterpret_cast<float4*>(sT + (buf * kK2 + r) * RP + 4 * c4) = trg[h];
      }
    }
  };
  const int tr = tid >> 4, tc = tid & 15;
  float acc[8][RPT];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int e = 0; e < RPT; ++e) acc[i][e] = 0.f;
  if (nst > 0) {
    load();
    store(0);
  }
  __syncthreads();
  for (int i = 0; i < nst; ++i) {
    const int buf = i & 1;
    if (i + 1 < nst) load();
    const float* U = sU + buf * kK2 * kMrRows + 8 * tr;
    const float* T = sT + buf * kK2 * RP;
#pragma unroll 4
    for (int j = 0; j < kK2; ++j) {
      const float4 u0 = *reinterpret_cast<const float4*>(U + j * kMrRows);
      const float4 u1 = *reinterpret_cast<const float4*>(U + j * kMrRows + 4);
      float x[RPT];
      load_x<RPT>(T + j * RP, tc, x);
      const float uu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int e = 0; e < RPT; ++e) acc[r][e] = fmaf(uu[r], x[e], acc[r][e]);
    }
    if (i + 1 < nst) store(buf ^ 1);
    __syncthreads();
  }
  add_tile<RPT, kMrRows, 8>(a, tl, sm2, acc, tr, tc);
}

template <int RPT>
cudaError_t launch_rpt(int kind, const MrArgs& a, cudaStream_t st) {
  constexpr int RP = 16 * RPT;
  if (kind == 1) {
    const size_t smem = sizeof(float) * (2 * kK1 * kVRow + 2 * kK1 * RP);
    cudaError_t e = cudaFuncSetAttribute(mr_phase1<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) mr_phase1<RPT><<<a.n_groups, kP1Threads, smem, st>>>(a);
  } else {
    const size_t smem = sizeof(float) * std::max(2 * kK2 * (kMrRows + RP), kMrRows * (std::min(RP, 64) + 1));
    cudaError_t e = cudaFuncSetAttribute(mr_phase2<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) mr_phase2<RPT><<<a.n_tiles, kThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace


cudaError_t launch_mr(int kind, const MrArgs& a, cudaStream_t st) {
  if ((kind == 1 && a.n_groups <= 0) || (kind != 1 && a.n_tiles <= 0)) return cudaSuccess;
  if (a.rp <= 32) return launch_rpt<2>(kind, a, st);
  if (a.rp <= 64) return launch_rpt<4>(kind, a, st);
  return launch_rpt<8>(kind, a, st);
}

}  // namespace dev
}  // namespace hh
