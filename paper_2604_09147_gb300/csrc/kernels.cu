// sm_103a kernels of the H_h matrix-vector product (Algorithm 4).
//
// One product is four launches on the caller's stream:
//   prep    : input vector -> tree order, fp32 and fp64 copies shifted by
//             0..3 (resp. 0..1) positions so that every 16-byte vector of a
//             factor column meets an aligned 16-byte vector of the input,
//             and the fp64 output accumulator is cleared;
//   phase 1 : t_b = f1_b^T in_J for every low-rank block (warp per column,
//             16-byte streaming loads, upcast in registers, fp32 accumulation
//             -- fp64 for fp64-stored blocks -- and a warp-shuffle tree);
//   phase 2 : out_I += 2^e f2_b t_b for every low-rank block (lanes along
//             rows, loop over the k columns, fp32 accumulation in chunks of
//             eight columns, fp64 scatter-add), and out += D in for the
//             dense fp64 blocks;
//   finish  : output accumulator -> the caller's point order.
// Work is a list of warp-sized items sorted by size; the pass kernels are
// persistent grids whose warps stride through the list.  No kernel waits on
// another block.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "hh_device.h"

namespace hh {
namespace dev {

namespace {

template <int FMT>
struct FmtTraits;
template <>
struct FmtTraits<0> {
  static constexpr int SZ = 8;
};
template <>
struct FmtTraits<1> {
  static constexpr int SZ = 4;
};
template <>
struct FmtTraits<2> {
  static constexpr int SZ = 2;
};
template <>
struct FmtTraits<3> {
  static constexpr int SZ = 2;
};
template <>
struct FmtTraits<4> {
  static constexpr int SZ = 1;
};

// 16-byte streaming load: factor data is read once per product.
__device__ __forceinline__ uint4 ld_stream16(const uint8_t* p) {
  return __ldcs(reinterpret_cast<const uint4*>(p));
}
__device__ __forceinline__ uint2 ld_stream8(const uint8_t* p) {
  return __ldcs(reinterpret_cast<const uint2*>(p));
}

__device__ __forceinline__ float2 h2f(uint32_t w) {
  __half2_raw r;
  r.x = static_cast<unsigned short>(w & 0xffffu);
  r.y = static_cast<unsigned short>(w >> 16);
  return __half22float2(__half2(r));
}
__device__ __forceinline__ float2 bf2f(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
__device__ __forceinline__ void e4m3x4_to_f(uint32_t w, float* v) {
  __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w & 0xffffu), __NV_E4M3);
  __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w >> 16), __NV_E4M3);
  float2 a = __half22float2(__half2(lo));
  float2 b = __half22float2(__half2(hi));
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// decode one 32-bit word holding 32/8/SZ elements of format FMT (FMT != 0)
template <int FMT>
__device__ __forceinline__ void decode_word(uint32_t w, float* v) {
  if constexpr (FMT == 1) {
    v[0] = __uint_as_float(w);
  } else if constexpr (FMT == 2) {
    float2 f = h2f(w);
    v[0] = f.x;
    v[1] = f.y;
  } else if constexpr (FMT == 3) {
    float2 f = bf2f(w);
    v[0] = f.x;
    v[1] = f.y;
  } else {
    e4m3x4_to_f(w, v);
  }
}

template <int FMT>
__device__ __forceinline__ void decode16(const uint4& r, float* v) {
  constexpr int PW = 4 / FmtTraits<FMT>::SZ;  // elements per 32-bit word
  decode_word<FMT>(r.x, v);
  decode_word<FMT>(r.y, v + PW);
  decode_word<FMT>(r.z, v + 2 * PW);
  decode_word<FMT>(r.w, v + 3 * PW);
}
template <int FMT>
__device__ __forceinline__ void decode8(const uint2& r, float* v) {
  constexpr int PW = 4 / FmtTraits<FMT>::SZ;
  decode_word<FMT>(r.x, v);
  decode_word<FMT>(r.y, v + PW);
}

// vectors in flight per lane: 64 bytes for narrow formats, fewer for the
// wide decodes so that every format path fits the register budget
template <int FMT>
struct Unroll {
  static constexpr int P1 = FmtTraits<FMT>::SZ >= 4 ? 4 : 2;
  static constexpr int P2 = FmtTraits<FMT>::SZ >= 4 ? 8 : 4;
};

__device__ __forceinline__ int lanes_for(int nvec) {
  int g = 1;
  while (g < nvec && g < 32) g <<= 1;
  return g;
}

// ------------------------------------------------------------------ phase 1
// t_j = sum_i f1[i, j] in[c1 + i] for columns [lo, hi) of one block.
template <int FMT, int NR>
__device__ __forceinline__ void p1_lowrank(const BlkDesc& d, int lo, int hi, const PassArgs& a,
                                           int lane) {
  constexpr int SZ = FmtTraits<FMT>::SZ;
  constexpr int VW = 16 / SZ;
  constexpr int UN = Unroll<FMT>::P1;
  const int nvec = (d.n1 + VW - 1) / VW;
  const int G = lanes_for(nvec);
  const int C = 32 / G, g = lane / G, li = lane % G;
  for (int j0 = lo; j0 < hi; j0 += C) {
    const int j = j0 + g;
    const bool act = j < hi;
    if constexpr (FMT == 0) {
      double acc[NR][2];
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[r][0] = acc[r][1] = 0.0;
      if (act) {
        const uint8_t* col = d.f1 + static_cast<size_t>(j) * d.ld1 * SZ;
        for (int v0 = li; v0 < nvec; v0 += UN * G) {
          uint4 raw[UN];
#pragma unroll
          for (int u = 0; u < UN; ++u) {
            const int v = v0 + u * G;
            if (v < nvec) raw[u] = ld_stream16(col + static_cast<size_t>(v) * 16);
          }
#pragma unroll
          for (int u = 0; u < UN; ++u) {
            const int v = v0 + u * G;
            if (v < nvec) {
              const double f0 = __hiloint2double(raw[u].y, raw[u].x);
              const double f1 = __hiloint2double(raw[u].w, raw[u].z);
              const int q = d.c1 + v * VW, s = q & 1;
#pragma unroll
              for (int r = 0; r < NR; ++r) {
                const double2 xv =
                    __ldg(reinterpret_cast<const double2*>(a.xs64 + (static_cast<size_t>(s * NR + r)) * a.npad + (q - s)));
                acc[r][0] = fma(f0, xv.x, acc[r][0]);
                acc[r][1] = fma(f1, xv.y, acc[r][1]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        double s = acc[r][0] + acc[r][1];
        for (int off = G >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (act && li == 0) a.t64[d.toff + static_cast<int64_t>(j) * NR + r] = s;
      }
    } else {
      // four partial sums per lane and RHS: element e goes to e % 4
      float acc[NR][4];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[r][e] = 0.f;
      if (act) {
        const uint8_t* col = d.f1 + static_cast<size_t>(j) * d.ld1 * SZ;
        for (int v0 = li; v0 < nvec; v0 += UN * G) {
          uint4 raw[UN];
#pragma unroll
          for (int u = 0; u < UN; ++u) {
            const int v = v0 + u * G;
            if (v < nvec) raw[u] = ld_stream16(col + static_cast<size_t>(v) * 16);
          }
#pragma unroll
          for (int u = 0; u < UN; ++u) {
            const int v = v0 + u * G;
            if (v < nvec) {
              float f[VW];
              decode16<FMT>(raw[u], f);
              const int q = d.c1 + v * VW, s = q & 3;
#pragma unroll
              for (int r = 0; r < NR; ++r) {
                const float* xp = a.xs + static_cast<size_t>(s * NR + r) * a.npad + (q - s);
#pragma unroll
                for (int e4 = 0; e4 < VW; e4 += 4) {
                  const float4 xv = __ldg(reinterpret_cast<const float4*>(xp + e4));
                  acc[r][0] = fmaf(f[e4 + 0], xv.x, acc[r][0]);
                  acc[r][1] = fmaf(f[e4 + 1], xv.y, acc[r][1]);
                  acc[r][2] = fmaf(f[e4 + 2], xv.z, acc[r][2]);
                  acc[r][3] = fmaf(f[e4 + 3], xv.w, acc[r][3]);
                }
              }
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        float s = (acc[r][0] + acc[r][1]) + (acc[r][2] + acc[r][3]);
        for (int off = G >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (act && li == 0) a.t32[d.toff + static_cast<int64_t>(j) * NR + r] = s;
      }
    }
  }
}

// ------------------------------------------------------------------ phase 2
// out[c2 + i] += 2^e sum_j f2[i, j] t_j for rows [lo, hi) of one block.
template <int FMT, int NR>
__device__ __forceinline__ void p2_lowrank(const BlkDesc& d, int lo, int hi, const PassArgs& a,
                                           int lane) {
  constexpr int SZ = FmtTraits<FMT>::SZ;
  // e4m3 uses 8-byte loads here to keep the accumulator count at 8 per RHS
  constexpr int LB = (FMT == 4) ? 8 : 16;
  constexpr int VW = LB / SZ;
  constexpr int CH = Unroll<FMT>::P2;  // columns per fp32 chunk
  const int nvec = (hi - lo + VW - 1) / VW;
  const int G = lanes_for(nvec);
  const int C = 32 / G, g = lane / G, li = lane % G;
  const int row0 = lo + li * VW;
  const bool act = li < nvec;
  const uint8_t* base = d.f2 + static_cast<size_t>(row0) * SZ;
  if constexpr (FMT == 0) {
    double acc[VW][NR];
#pragma unroll
    for (int e = 0; e < VW; ++e)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[e][r] = 0.0;
    for (int jc = g; jc < d.k; jc += CH * C) {
      uint4 raw[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int j = jc + u * C;
        if (act && j < d.k) raw[u] = ld_stream16(base + static_cast<size_t>(j) * d.ld2 * SZ);
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int j = jc + u * C;
        if (j < d.k) {
          double tj[NR];
#pragma unroll
          for (int r = 0; r < NR; ++r) tj[r] = __ldg(a.t64 + d.toff + static_cast<int64_t>(j) * NR + r);
          if (act) {
            const double f0 = __hiloint2double(raw[u].y, raw[u].x);
            const double f1 = __hiloint2double(raw[u].w, raw[u].z);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              acc[0][r] = fma(f0, tj[r], acc[0][r]);
              acc[1][r] = fma(f1, tj[r], acc[1][r]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int e = 0; e < VW; ++e)
#pragma unroll
      for (int r = 0; r < NR; ++r)
        for (int off = G; off < 32; off <<= 1) acc[e][r] += __shfl_xor_sync(0xffffffffu, acc[e][r], off);
    if (act && g == 0) {
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const int row = row0 + e;
        if (row < hi)
#pragma unroll
          for (int r = 0; r < NR; ++r)
            atomicAdd(a.acc + static_cast<size_t>(r) * a.npad + d.c2 + row, ldexp(acc[e][r], d.e));
      }
    }
  } else {
    float acc[VW][NR];
#pragma unroll
    for (int e = 0; e < VW; ++e)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[e][r] = 0.f;
    // fp32-stored blocks sum each chunk of CH columns separately before
    // adding it to the running total (shorter fp32 sums); 16- and 8-bit
    // blocks, whose storage error dominates, accumulate directly
    constexpr bool kChunk = (FMT == 1);
    for (int jc = g; jc < d.k; jc += CH * C) {
      float part_store[kChunk ? VW : 1][kChunk ? NR : 1];
      auto part = [&](int e, int r) -> float& { return kChunk ? part_store[e][r] : acc[e][r]; };
      if constexpr (kChunk) {
#pragma unroll
        for (int e = 0; e < VW; ++e)
#pragma unroll
          for (int r = 0; r < NR; ++r) part_store[e][r] = 0.f;
      }
      if constexpr (LB == 16) {
        uint4 raw[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = jc + u * C;
          if (act && j < d.k) raw[u] = ld_stream16(base + static_cast<size_t>(j) * d.ld2 * SZ);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = jc + u * C;
          if (j < d.k) {
            float tj[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) tj[r] = __ldg(a.t32 + d.toff + static_cast<int64_t>(j) * NR + r);
            if (act) {
              float f[VW];
              decode16<FMT>(raw[u], f);
#pragma unroll
              for (int e = 0; e < VW; ++e)
#pragma unroll
                for (int r = 0; r < NR; ++r) part(e, r) = fmaf(f[e], tj[r], part(e, r));
            }
          }
        }
      } else {
        uint2 raw[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = jc + u * C;
          if (act && j < d.k) raw[u] = ld_stream8(base + static_cast<size_t>(j) * d.ld2 * SZ);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = jc + u * C;
          if (j < d.k) {
            float tj[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) tj[r] = __ldg(a.t32 + d.toff + static_cast<int64_t>(j) * NR + r);
            if (act) {
              float f[VW];
              decode8<FMT>(raw[u], f);
#pragma unroll
              for (int e = 0; e < VW; ++e)
#pragma unroll
                for (int r = 0; r < NR; ++r) part(e, r) = fmaf(f[e], tj[r], part(e, r));
            }
          }
        }
      }
      if constexpr (kChunk) {
#pragma unroll
        for (int e = 0; e < VW; ++e)
#pragma unroll
          for (int r = 0; r < NR; ++r) acc[e][r] += part_store[e][r];
      }
    }
#pragma unroll
    for (int e = 0; e < VW; ++e)
#pragma unroll
      for (int r = 0; r < NR; ++r)
        for (int off = G; off < 32; off <<= 1) acc[e][r] += __shfl_xor_sync(0xffffffffu, acc[e][r], off);
    if (act && g == 0) {
#pragma unroll
      for (int e = 0; e < VW; ++e) {
        const int row = row0 + e;
        if (row < hi)
#pragma unroll
          for (int r = 0; r < NR; ++r)
            atomicAdd(a.acc + static_cast<size_t>(r) * a.npad + d.c2 + row,
                      ldexp(static_cast<double>(acc[e][r]), d.e));
      }
    }
  }
}

// dense forward: out[r0 + i] += sum_j D[i, j] in[c0 + j] for rows [lo, hi)
template <int NR>
__device__ __forceinline__ void dense_fwd(const DenseDesc& D, int lo, int hi, const PassArgs& a, int lane) {
  const int row = lo + lane;
  const bool act = row < hi;
  double acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = 0.0;
  const double* col = D.d + row;
  int c = 0;
  for (; c + 8 <= D.n; c += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = act ? __ldcs(col + static_cast<int64_t>(c + u) * D.ld) : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int r = 0; r < NR; ++r)
        acc[r] = fma(v[u], __ldg(a.xs64 + static_cast<size_t>(r) * a.npad + D.c0 + c + u), acc[r]);
  }
  for (; c < D.n; ++c) {
    const double v = act ? __ldcs(col + static_cast<int64_t>(c) * D.ld) : 0.0;
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = fma(v, __ldg(a.xs64 + static_cast<size_t>(r) * a.npad + D.c0 + c), acc[r]);
  }
  if (act)
#pragma unroll
    for (int r = 0; r < NR; ++r) atomicAdd(a.acc + static_cast<size_t>(r) * a.npad + D.r0 + row, acc[r]);
}

// dense transposed: out[c0 + j] += sum_i D[i, j] in[r0 + i] for columns [lo, hi)
template <int NR>
__device__ __forceinline__ void dense_T(const DenseDesc& D, int lo, int hi, const PassArgs& a, int lane) {
  const int G = lanes_for(D.m);
  const int C = 32 / G, g = lane / G, li = lane % G;
  for (int j0 = lo; j0 < hi; j0 += C) {
    const int j = j0 + g;
    const bool act = j < hi;
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0;
    if (act) {
      const double* col = D.d + static_cast<int64_t>(j) * D.ld;
      for (int i = li; i < D.m; i += G) {
        const double v = __ldcs(col + i);
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = fma(v, __ldg(a.xs64 + static_cast<size_t>(r) * a.npad + D.r0 + i), acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      double s = acc[r];
      for (int off = G >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (act && li == 0) atomicAdd(a.acc + static_cast<size_t>(r) * a.npad + D.c0 + j, s);
    }
  }
}

// FSET: bit f set = this variant contains the code path of format f.  The
// host launches the narrowest variant that covers the matrix, so the paths a
// matrix does not use do not raise the register count of the ones it does.
template <int PHASE, int NR, unsigned FSET>
__global__ void __launch_bounds__(kThreads, kMinBlocks) pass_kernel(PassArgs a) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (kThreads / 32);
  for (int it = gw; it < a.n_items; it += nw) {
    const Item w = a.items[it];
    if (w.kind == 0 || w.kind == 1) {
      const BlkDesc d = a.blk[w.idx];
      if (PHASE == 1 && w.kind == 0) {
        switch (d.fmt) {
          case 0:
            if constexpr ((FSET >> 0) & 1u) {
              p1_lowrank<0, NR>(d, w.lo, w.hi, a, lane);
              break;
            }
            [[fallthrough]];
          case 1:
            if constexpr ((FSET >> 1) & 1u) {
              p1_lowrank<1, NR>(d, w.lo, w.hi, a, lane);
              break;
            }
            [[fallthrough]];
          case 2:
            if constexpr ((FSET >> 2) & 1u) {
              p1_lowrank<2, NR>(d, w.lo, w.hi, a, lane);
              break;
            }
            [[fallthrough]];
          case 3:
            if constexpr ((FSET >> 3) & 1u) {
              p1_lowrank<3, NR>(d, w.lo, w.hi, a, lane);
              break;
            }
            [[fallthrough]];
          case 4:
            if constexpr ((FSET >> 4) & 1u) {
              p1_lowrank<4, NR>(d, w.lo, w.hi, a, lane);
              break;
            }
            [[fallthrough]];
          default:
            if (lane == 0) atomicOr(a.status, 1);
        }
      } else if (PHASE == 2 && w.kind == 1) {
        switch (d.fmt) {
          case 0:
            if constexpr ((FSET >> 0) & 1u) {
              p2_lowrank<0, NR>(d, w.lo, w.hi, a, lane);
              break;
            }
            [[fallthrough]];
          case 1:
            if constexpr ((FSET >> 1) & 1u) {
              p2_lowrank<1, NR>(d, w.lo, w.hi, a, lane);
              break;
            }
            [[fallthrough]];
          case 2:
            if constexpr ((FSET >> 2) & 1u) {
              p2_lowrank<2, NR>(d, w.lo, w.hi, a, lane);
              break;
            }
            [[fallthrough]];
          case 3:
            if constexpr ((FSET >> 3) & 1u) {
              p2_lowrank<3, NR>(d, w.lo, w.hi, a, lane);
              break;
            }
            [[fallthrough]];
          case 4:
            if constexpr ((FSET >> 4) & 1u) {
              p2_lowrank<4, NR>(d, w.lo, w.hi, a, lane);
              break;
            }
            [[fallthrough]];
          default:
            if (lane == 0) atomicOr(a.status, 1);
        }
      } else if (lane == 0) {
        atomicOr(a.status, 2);
      }
    } else if (PHASE == 2 && w.kind == 2) {
      dense_fwd<NR>(a.dns[w.idx], w.lo, w.hi, a, lane);
    } else if (PHASE == 2 && w.kind == 3) {
      dense_T<NR>(a.dns[w.idx], w.lo, w.hi, a, lane);
    } else if (lane == 0) {
      atomicOr(a.status, 2);
    }
  }
}

// input (user order, column-major) -> tree-ordered shifted copies; clears acc
__global__ void prep_kernel(const double* __restrict__ in, int64_t ld, int nr,
                            const int32_t* __restrict__ perm, int64_t n, int64_t npad,
                            float* __restrict__ xs, double* __restrict__ xs64, double* __restrict__ acc) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < npad;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    for (int r = 0; r < nr; ++r) {
      double v[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int64_t q = p + s;
        v[s] = q < n ? in[static_cast<int64_t>(perm[q]) + r * ld] : 0.0;
        xs[(static_cast<int64_t>(s) * nr + r) * npad + p] = static_cast<float>(v[s]);
      }
      xs64[(static_cast<int64_t>(0) * nr + r) * npad + p] = v[0];
      xs64[(static_cast<int64_t>(1) * nr + r) * npad + p] = v[1];
      acc[static_cast<int64_t>(r) * npad + p] = 0.0;
    }
  }
}

__global__ void finish_kernel(const double* __restrict__ acc, int nr, const int32_t* __restrict__ perm,
                              int64_t n, int64_t npad, double* __restrict__ out, int64_t ld) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t u = perm[p];
    for (int r = 0; r < nr; ++r) out[u + r * ld] = acc[static_cast<int64_t>(r) * npad + p];
  }
}

template <int PHASE, unsigned FSET>
cudaError_t launch_phase(const PassArgs& a, int grid, cudaStream_t st) {
  switch (a.nr) {
    case 1: pass_kernel<PHASE, 1, FSET><<<grid, kThreads, 0, st>>>(a); break;
    case 2: pass_kernel<PHASE, 2, FSET><<<grid, kThreads, 0, st>>>(a); break;
    case 4: pass_kernel<PHASE, 4, FSET><<<grid, kThreads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int PHASE, unsigned FSET>
int occupancy(int nr) {
  int b = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (nr == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pass_kernel<PHASE, 1, FSET>, kThreads, 0);
  if (nr == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pass_kernel<PHASE, 2, FSET>, kThreads, 0);
  if (nr == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pass_kernel<PHASE, 4, FSET>, kThreads, 0);
  return (e != cudaSuccess || b < 1) ? 1 : b;
}

}  // namespace

cudaError_t launch_prep(const double* in, int64_t ld, int nr, const int32_t* perm, int64_t n,
                        int64_t npad, float* xs, double* xs64, double* acc, cudaStream_t st) {
  int64_t blocks = (npad + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  prep_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(in, ld, nr, perm, n, npad, xs, xs64, acc);
  return cudaGetLastError();
}

cudaError_t launch_pass(int phase, unsigned fset, const PassArgs& a, int grid, cudaStream_t st) {
  if (a.n_items == 0) return cudaSuccess;
  if (fset == kSetF64) return phase == 1 ? launch_phase<1, kSetF64>(a, grid, st) : launch_phase<2, kSetF64>(a, grid, st);
  if (fset == kSetF32) return phase == 1 ? launch_phase<1, kSetF32>(a, grid, st) : launch_phase<2, kSetF32>(a, grid, st);
  return phase == 1 ? launch_phase<1, kSetAll>(a, grid, st) : launch_phase<2, kSetAll>(a, grid, st);
}

cudaError_t launch_finish(const double* acc, int nr, const int32_t* perm, int64_t n, int64_t npad,
                          double* out, int64_t ld, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  finish_kernel<<<static_cast<int>(blocks), 256, 0, st>>>(acc, nr, perm, n, npad, out, ld);
  return cudaGetLastError();
}

int pass_blocks_per_sm(int phase, unsigned fset, int nr) {
  if (fset == kSetF64) return phase == 1 ? occupancy<1, kSetF64>(nr) : occupancy<2, kSetF64>(nr);
  if (fset == kSetF32) return phase == 1 ? occupancy<1, kSetF32>(nr) : occupancy<2, kSetF32>(nr);
  return phase == 1 ? occupancy<1, kSetAll>(nr) : occupancy<2, kSetAll>(nr);
}

unsigned pass_set_for(unsigned fmts_present) {
  if ((fmts_present & ~kSetF64) == 0) return kSetF64;
  if ((fmts_present & ~kSetF32) == 0) return kSetF32;
  return kSetAll;
}

}  // namespace dev
}  // namespace hh
