// Pipelined streaming passes of the H_h product (Algorithm 4) for sm_103a.
//
// Both passes stream factor columns from HBM into a ring of shared-memory
// stages with bulk asynchronous copies (cp.async.bulk, completion counted on
// an mbarrier), so the bytes in flight do not depend on registers.  Each
// persistent CTA has one producer warp and kConsumers consumer warps.
//
//   phase 1 item: columns [lo, hi) (at most kP1Cols) of a factor f with
//     `rows` rows; stage s holds rows [s*RC, (s+1)*RC) of those columns,
//     RC * sizeof(fmt) = 2 KB per column.  Consumers compute
//     sum_i f[i, j] in[in_off + i]; mode 0 stores it to t (low-rank phase 1),
//     mode 1 adds it to out[out_off + j] (dense block, transposed product).
// fp64 factors and dense blocks (held as fp32 pairs) are computed in
// double-float arithmetic on the fp32 pipe (dd_acc below).
//
//   phase 2 item: rows [lo, hi) (at most RT, RT * sizeof(fmt) = 1 KB) of a
//     factor f with `cols` columns; stage s holds columns [s*16, s*16+16) of
//     those rows.  Consumers compute 2^e sum_j f[i, j] t_j and add it to
//     out[out_off + i]; t is the block's t arena (mode 0) or the fp64 input
//     itself (mode 1, dense block, forward product).
//
// Items come from a global counter (dynamic schedule, zeroed by the prep
// launch).  Every wait on an mbarrier has a clock-based limit; on expiry the
// kernel sets bit 2 of the status word, lets the copies it issued complete
// (again bounded) and returns.
//
// Programmatic dependent launch: every CTA lets the next kernel of the stream
// start early (griddepcontrol.launch_dependents).  Phase 2 may be launched
// that way after phase 1: its producer streams U factors (which phase 1 does
// not write) while phase 1 drains, and its consumers wait for phase 1 to
// complete (griddepcontrol.wait, a no-op for a normal launch) before they
// read t.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "hh_device.h"

namespace hh {
namespace dev {

namespace {

constexpr int kConsumers = 4;                       // consumer warps per CTA
constexpr int kStreamThreads = 32 * (kConsumers + 1);
constexpr int kStages = 4;                          // default pipeline depth (stages per CTA)
constexpr int kStageBytes = 16384;
constexpr int kP1Cols = 8;                          // columns per phase-1 item
constexpr int kP1ColBytes = kStageBytes / kP1Cols;  // 2 KB per column and stage
constexpr int kP2Cols = 16;                         // columns per phase-2 stage
constexpr int kP2RowBytes = kStageBytes / kP2Cols;  // 1 KB of rows per column
constexpr long long kWaitCycles = 4000000000LL;     // about 2 s at 2 GHz

// What consumers need about a stage, written by the producer next to the
// data so that consumers read no descriptor from global memory.
struct Meta {
  int32_t item;    // item index, or -1: no more work
  int32_t part;    // stage number within the item
  int32_t count;   // rows (phase 1) or columns (phase 2) in this stage
  int32_t last;    // 1 if this is the item's last stage
  int32_t fmt, mode, e, lo, hi, in_off, out_off, xs;  // xs: 1 if the input segment is staged
  int64_t toff;
};

// Staged fp32 input of a phase-1 stage: RC rows of 4 bytes, RC = 2 KB / size
// of the format (fp32: 512 rows, 16-bit: 1024, fp8: 2048); fp64 stages hold
// the 256-row leading halves at offset 0 and the trailing halves at XBytes/2.
template <unsigned FSET>
struct XArea {
  static constexpr int bytes = (FSET & 28u) ? 8192 : 2048;
};

template <int PHASE, unsigned FSET, int NST>
struct __align__(128) Smem {
  static constexpr int kX = XArea<FSET>::bytes;
  uint8_t data[NST][kStageBytes];
  uint8_t x[PHASE == 1 ? NST : 1][PHASE == 1 ? kX : 16];
  Meta meta[NST];
  unsigned long long full[NST];
  unsigned long long empty[NST];
};

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false (and status bit 2) when the limit expires
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, uint32_t parity, int* status) {
  if (mbar_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(b, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      atomicOr(status, 4);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s_plain(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar,
                                         uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <int FMT>
struct Sz;
template <> struct Sz<0> { static constexpr int v = 8; };
template <> struct Sz<1> { static constexpr int v = 4; };
template <> struct Sz<2> { static constexpr int v = 2; };
template <> struct Sz<3> { static constexpr int v = 2; };
template <> struct Sz<4> { static constexpr int v = 1; };

__device__ __forceinline__ int fmt_size(int fmt) { return fmt == 0 ? 8 : (fmt == 1 ? 4 : (fmt == 4 ? 1 : 2)); }

// decode 8 bytes of format FMT (FMT != 0) into 8 / Sz floats
template <int FMT>
__device__ __forceinline__ void dec8(uint2 w, float* v) {
  if constexpr (FMT == 1) {
    v[0] = __uint_as_float(w.x);
    v[1] = __uint_as_float(w.y);
  } else if constexpr (FMT == 2) {
    __half2_raw a, b;
    a.x = (unsigned short)(w.x & 0xffffu); a.y = (unsigned short)(w.x >> 16);
    b.x = (unsigned short)(w.y & 0xffffu); b.y = (unsigned short)(w.y >> 16);
    float2 fa = __half22float2(__half2(a)), fb = __half22float2(__half2(b));
    v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
  } else if constexpr (FMT == 3) {
    v[0] = __uint_as_float(w.x << 16); v[1] = __uint_as_float(w.x & 0xffff0000u);
    v[2] = __uint_as_float(w.y << 16); v[3] = __uint_as_float(w.y & 0xffff0000u);
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t x = h ? w.y : w.x;
      __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(x & 0xffffu), __NV_E4M3);
      __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(x >> 16), __NV_E4M3);
      float2 a = __half22float2(__half2(lo)), b = __half22float2(__half2(hi));
      v[4 * h + 0] = a.x; v[4 * h + 1] = a.y; v[4 * h + 2] = b.x; v[4 * h + 3] = b.y;
    }
  }
}

// ------------------------------------------------- fp64 on the fp32 pipe
// fp64 factors and dense blocks are held on the device as pairs of fp32
// values in the same 8 bytes (v ~= hi + lo, hi = fl32(v), lo = fl32(v - hi),
// written once when the matrix is uploaded; about 2^-48 relative, values
// below 2^-126 of the block's largest entry flushed).  Products of such
// pairs with the fp32 halves of the input are summed as unevaluated pairs
// S + C (two-sum of the leading products, the small cross terms gathered in
// C): about 2^-46 relative per product, without the device's low-rate fp64
// units.  Reductions of pairs and the conversion of the result to fp64 stay
// off those units too (dd_add, f2d_scaled): on this device a single fp64
// instruction per output costs as much issue time as the whole fp32 pipeline
// of a stage.

// (S, C) += (vh + vl) * (xh + xl), dropping vl * xl
__device__ __forceinline__ void dd_acc(float& S, float& C, float vh, float vl, float xh, float xl) {
  const float p = vh * xh;
  const float pe = fmaf(vh, xh, -p);
  const float cr = fmaf(vh, xl, fmaf(vl, xh, pe));
  const float t = S + p;
  const float bp = t - S;
  const float err = (S - (t - bp)) + (p - bp);
  S = t;
  C += err + cr;
}

// (S, C) += (s2, c2): leading parts by two-sum, trailing parts in fp32
__device__ __forceinline__ void dd_add(float& S, float& C, float s2, float c2) {
  const float t = S + s2;
  const float bp = t - S;
  const float err = (S - (t - bp)) + (s2 - bp);
  S = t;
  C += err + c2;
}

// v * 2^e as an fp64 value, built from v's bits with integer operations
// (exact); zero, subnormal, non-finite or out-of-range results take the
// fp64 units (rare)
__device__ __forceinline__ double f2d_scaled(float v, int e) {
  const uint32_t b = __float_as_uint(v);
  const int ex = static_cast<int>((b >> 23) & 0xffu);
  if ((b & 0x7fffffffu) == 0u) return 0.0;
  const int de = ex - 127 + 1023 + e;
  if (ex == 0 || ex == 255 || de < 1 || de > 2046) return ldexp(static_cast<double>(v), e);
  const unsigned long long bits = (static_cast<unsigned long long>(b & 0x80000000u) << 32) |
                                  (static_cast<unsigned long long>(de) << 52) |
                                  (static_cast<unsigned long long>(b & 0x7fffffu) << 29);
  return __longlong_as_double(static_cast<long long>(bits));
}

// ---------------------------------------------------------------- producer
// Walks the item list (dynamic schedule) and fills stages.  Phase 1 stages
// carry up to kP1Cols column segments of RC rows; phase 2 stages up to
// kP2Cols column segments of the item's rows.
template <int PHASE, unsigned FSET, int NST>
__device__ void produce(Smem<PHASE, FSET, NST>& sm, const StreamArgs& a) {
  constexpr int kXBytes = XArea<FSET>::bytes;
  const int lane = threadIdx.x & 31;
  const uint64_t pol = evict_first_policy();
  int stage = 0;
  uint32_t par = 1;  // empty barriers: the first round passes immediately
  bool ok = true;
  int issued_mask = 0;  // stages whose copies may be in flight after a timeout
  uint32_t issued_par[NST] = {};  // full-barrier phase parity of the last issue per stage
  // the next item's number is taken from the counter while the current
  // item's stages are issued, so that the atomic's round trip overlaps them
  int next = 0;
  if (lane == 0) next = atomicAdd(a.counter, 1);
  while (ok) {
    const int item = __shfl_sync(0xffffffffu, next, 0);
    if (item >= a.n_items) break;
    if (lane == 0) next = atomicAdd(a.counter, 1);
    const Item it = a.items[item];
    const StreamDesc d = a.desc[it.idx];
    const int sz = fmt_size(d.fmt);
    int nparts, per;  // stages in this item, rows (phase 1) or columns (phase 2) per stage
    if (PHASE == 1) {
      per = kP1ColBytes / sz;
      nparts = (d.rows + per - 1) / per;
      if (nparts == 0) nparts = 1;
    } else {
      per = kP2Cols;
      nparts = (d.cols + per - 1) / per;
      if (nparts == 0) nparts = 1;
    }
    // phase 1: an item of short columns spans several groups of kP1Cols
    // columns, streamed group after group (each group is a run of stages the
    // consumers reduce and flush on its own)
    const int ngroups = PHASE == 1 ? (it.hi - it.lo + kP1Cols - 1) / kP1Cols : 1;
    for (int q = 0; q < ngroups * nparts; ++q) {
      const int p = q % nparts;
      const int glo = PHASE == 1 ? it.lo + (q / nparts) * kP1Cols : it.lo;
      const int ghi = PHASE == 1 ? min(glo + kP1Cols, it.hi) : it.hi;
      if (!mbar_wait(&sm.empty[stage], par, a.status)) {
        ok = false;
        break;
      }
      int count, bytes_each, nseg;
      const uint8_t* src0;
      size_t seg_stride;  // bytes between consecutive segments in global memory
      if (PHASE == 1) {
        count = min(per, d.rows - p * per);
        if (count < 0) count = 0;
        bytes_each = ((count * sz) + 15) & ~15;
        nseg = ghi - glo;
        src0 = d.f + (static_cast<size_t>(glo) * d.ld + static_cast<size_t>(p) * per) * sz;
        seg_stride = static_cast<size_t>(d.ld) * sz;
      } else {
        count = min(per, d.cols - p * per);
        if (count < 0) count = 0;
        bytes_each = (((it.hi - it.lo) * sz) + 15) & ~15;
        nseg = count;
        src0 = d.f + (static_cast<size_t>(p) * per * d.ld + static_cast<size_t>(it.lo)) * sz;
        seg_stride = static_cast<size_t>(d.ld) * sz;
      }
      // phase 1, one right-hand side, non-fp64 factor: stage the fp32 input
      // segment of these rows (from the copy shifted so that row 0 is aligned)
      int xbytes = 0;
      const float* xsrc = nullptr;
      const float* xsrc_lo = nullptr;
      if (PHASE == 1 && a.nr == 1 && count > 0) {
        const int q0 = d.in_off + p * per, sh = q0 & 3;
        xsrc = a.xs + static_cast<size_t>(sh) * a.npad + (q0 - sh);
        xsrc_lo = a.xs_lo + static_cast<size_t>(sh) * a.npad + (q0 - sh);
        // whole 16-element groups: a lane reads up to 16 inputs per vector,
        // and rows past `count` meet zero factor padding, which must not
        // meet stale shared memory
        xbytes = ((count + 15) & ~15) * 4;
      }
      const int xtotal = (d.fmt == 0) ? 2 * xbytes : xbytes;  // fp64 factors also need the low halves
      if (lane == 0) {
        Meta m;
        m.item = item;
        m.part = p;
        m.count = count;
        m.last = (p == nparts - 1);
        m.fmt = d.fmt;
        m.mode = d.mode;
        m.e = d.e;
        m.lo = glo;
        m.hi = ghi;
        m.in_off = d.in_off;
        m.out_off = d.out_off;
        m.xs = xbytes > 0;
        m.toff = d.toff;
        sm.meta[stage] = m;
        mbar_expect_tx(&sm.full[stage], static_cast<uint32_t>(bytes_each * nseg + xtotal));
      }
      __syncwarp();
      const int slot = PHASE == 1 ? kP1ColBytes : kP2RowBytes;
      if (bytes_each > 0)
        for (int q = lane; q < nseg; q += 32)
          bulk_g2s(sm.data[stage] + q * slot, src0 + q * seg_stride, static_cast<uint32_t>(bytes_each),
                   &sm.full[stage], pol);
      if constexpr (PHASE == 1) {
        if (xbytes > 0 && lane == 31)
          bulk_g2s_plain(sm.x[stage], xsrc, static_cast<uint32_t>(xbytes), &sm.full[stage]);
        if (xbytes > 0 && d.fmt == 0 && lane == 30)
          bulk_g2s_plain(sm.x[stage] + kXBytes / 2, xsrc_lo, static_cast<uint32_t>(xbytes), &sm.full[stage]);
      }
      issued_mask |= 1 << stage;
      issued_par[stage] = par ^ 1u;
      if (++stage == NST) {
        stage = 0;
        par ^= 1u;
      }
    }
  }
  if (ok) {
    // sentinel: no more items
    if (mbar_wait(&sm.empty[stage], par, a.status)) {
      if (lane == 0) {
        Meta m;
        m.item = -1;
        sm.meta[stage] = m;
        mbar_arrive(&sm.full[stage]);
      }
    } else {
      ok = false;
    }
  }
  if (!ok) {
    // consumers may be gone: let the copies issued into this CTA's shared
    // memory finish (bounded) before the CTA can exit
    const long long t0 = clock64();
    for (int s = 0; s < NST; ++s) {
      if (!(issued_mask & (1 << s))) continue;
      while (!mbar_try(&sm.full[s], issued_par[s])) {
        if (clock64() - t0 > kWaitCycles) break;
      }
    }
  }
}

// ---------------------------------------------------------------- phase 1
// Consumer warp w takes columns w and w + kConsumers of the item; lane l
// takes the 16-byte vector l of every 512-byte group of a column segment
// (contiguous across lanes: conflict-free shared-memory reads).  Partial
// sums stay in registers across the item's stages.
template <int FMT, int NR, int XB>
__device__ __forceinline__ void p1_consume_stage(const uint8_t* data, const float* xsm, const Meta& m,
                                                 const StreamArgs& a, int wc, int lane, float (&acc)[2][NR][4],
                                                 float (&acd)[2][NR][16]) {
  constexpr int SZ = Sz<FMT>::v;
  constexpr int RC = kP1ColBytes / SZ;  // rows per stage
  const int ncols = m.hi - m.lo;
  const int row_base = m.part * RC;
  const bool c0 = wc < ncols, c1 = wc + kConsumers < ncols;
  if constexpr (FMT == 0) {
    // 2 doubles per 16 bytes; lane covers rows 2l, 2l+1 of every 64-row
    // group g.  acd[c][rr][2*q], acd[c][rr][2*q+1] is the double-float sum of
    // chain q = 2 * (g % G) + (row parity): independent chains for the
    // latency of the double-float updates (G = 4 groups for one right-hand
    // side, 2 otherwise).
    constexpr int G = NR == 1 ? 4 : 2;
#pragma unroll
    for (int g = 0; g < RC / 64; ++g) {
      const int r = g * 64 + 2 * lane;
      if (r >= m.count) break;
      float xh[NR][2], xl[NR][2];
      if (NR == 1 && m.xs) {
        const float2 h2 = *reinterpret_cast<const float2*>(xsm + r);
        const float2 l2 = *reinterpret_cast<const float2*>(xsm + XB / 8 + r);
        xh[0][0] = h2.x; xh[0][1] = h2.y; xl[0][0] = l2.x; xl[0][1] = l2.y;
      } else {
        const int q = m.in_off + row_base + r, s = q & 1;
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
          const size_t o = static_cast<size_t>(s * NR + rr) * a.npad + (q - s);
          const float2 h2 = __ldg(reinterpret_cast<const float2*>(a.xs + o));
          const float2 l2 = __ldg(reinterpret_cast<const float2*>(a.xs_lo + o));
          xh[rr][0] = h2.x; xh[rr][1] = h2.y; xl[rr][0] = l2.x; xl[rr][1] = l2.y;
        }
      }
      const int q0 = 4 * (g % G);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!(c ? c1 : c0)) continue;
        const float4 f = *reinterpret_cast<const float4*>(data + (wc + c * kConsumers) * kP1ColBytes + r * 8);
        const float h0 = f.x, l0 = f.y, h1 = f.z, l1 = f.w;
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
          dd_acc(acd[c][rr][q0 + 0], acd[c][rr][q0 + 1], h0, l0, xh[rr][0], xl[rr][0]);
          dd_acc(acd[c][rr][q0 + 2], acd[c][rr][q0 + 3], h1, l1, xh[rr][1], xl[rr][1]);
        }
      }
    }
  } else {
    constexpr int EPV = 16 / SZ;  // elements per 16-byte vector
    constexpr int NCH = EPV / 4;  // float4 chunks of input per vector (1, 2 or 4)
    // A lane's input rows are EPV * 4 bytes apart from its neighbour's: with
    // 16- and 8-bit factors the warp's 16-byte input reads would fall on 2 or 4
    // times fewer shared-memory bank groups than lanes need.  Each lane
    // therefore visits its chunks in an order rotated by rot (and rotates the
    // factor words alike), which spreads every read over all bank groups.
    const int rot = NCH == 4 ? ((lane >> 1) & 3) : (NCH == 2 ? ((lane >> 2) & 1) : 0);
#pragma unroll
    for (int g = 0; g < RC / (32 * EPV); ++g) {
      const int r = g * 32 * EPV + lane * EPV;
      if (r >= m.count) break;
      // the input of these EPV rows, NR right-hand sides
      // chunk j of the lane's registers holds input chunk (j + rot) mod NCH
      float xv[NR][EPV];
      if (NR == 1 && m.xs) {
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
          const int e4 = 4 * ((j + rot) & (NCH - 1));
          const float4 v = *reinterpret_cast<const float4*>(xsm + r + e4);
          xv[0][4 * j] = v.x; xv[0][4 * j + 1] = v.y; xv[0][4 * j + 2] = v.z; xv[0][4 * j + 3] = v.w;
        }
      } else {
        const int q = m.in_off + row_base + r, s = q & 3;
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
          const float* xp = a.xs + static_cast<size_t>(s * NR + rr) * a.npad + (q - s);
#pragma unroll
          for (int j = 0; j < NCH; ++j) {
            const int e4 = 4 * ((j + rot) & (NCH - 1));
            const float4 v = __ldg(reinterpret_cast<const float4*>(xp + e4));
            xv[rr][4 * j] = v.x; xv[rr][4 * j + 1] = v.y; xv[rr][4 * j + 2] = v.z; xv[rr][4 * j + 3] = v.w;
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!(c ? c1 : c0)) continue;
        const uint4 raw = *reinterpret_cast<const uint4*>(data + (wc + c * kConsumers) * kP1ColBytes + r * SZ);
        // the factor's 32-bit words in the same rotated chunk order
        uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
        if constexpr (NCH == 4) {
          if (rot & 1) { const uint32_t t = w[0]; w[0] = w[1]; w[1] = w[2]; w[2] = w[3]; w[3] = t; }
          if (rot & 2) { uint32_t t = w[0]; w[0] = w[2]; w[2] = t; t = w[1]; w[1] = w[3]; w[3] = t; }
        } else if constexpr (NCH == 2) {
          if (rot) { uint32_t t = w[0]; w[0] = w[2]; w[2] = t; t = w[1]; w[1] = w[3]; w[3] = t; }
        }
        float f[EPV];
        dec8<FMT>(make_uint2(w[0], w[1]), f);
        dec8<FMT>(make_uint2(w[2], w[3]), f + EPV / 2);
#pragma unroll
        for (int rr = 0; rr < NR; ++rr)
#pragma unroll
          for (int e = 0; e < EPV; ++e) acc[c][rr][e & 3] = fmaf(f[e], xv[rr][e], acc[c][rr][e & 3]);
      }
    }
  }
}

template <int NR>
__device__ __forceinline__ void p1_flush(const Meta& m, const StreamArgs& a, int wc, int lane,
                                         float (&acc)[2][NR][4], float (&acd)[2][NR][16]) {
  const int ncols = m.hi - m.lo;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int col = wc + c * kConsumers;
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
      if (m.fmt == 0) {
        float S = acd[c][rr][0], C = acd[c][rr][1];
#pragma unroll
        for (int q = 1; q < 8; ++q) dd_add(S, C, acd[c][rr][2 * q], acd[c][rr][2 * q + 1]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const float s2 = __shfl_xor_sync(0xffffffffu, S, off), c2 = __shfl_xor_sync(0xffffffffu, C, off);
          dd_add(S, C, s2, c2);
        }
        float th = S, tl = 0.f;  // renormalised: th = fl32(S + C), tl the rest
        dd_add(th, tl, C, 0.f);
        if (lane == 0 && col < ncols) {
          const int j = m.lo + col;
          if (m.mode == 0) {  // t of an fp64 block, kept as its two fp32 halves
            a.t64[m.toff + static_cast<int64_t>(j) * NR + rr] = make_float2(th, tl);
          } else {
            double* o = a.acc + static_cast<size_t>(rr) * a.npad + m.out_off + j;
            atomicAdd(o, f2d_scaled(th, m.e));
            if (tl != 0.f) atomicAdd(o, f2d_scaled(tl, m.e));
          }
        }
      } else {
        float s = (acc[c][rr][0] + acc[c][rr][1]) + (acc[c][rr][2] + acc[c][rr][3]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0 && col < ncols) a.t32[m.toff + static_cast<int64_t>(m.lo + col) * NR + rr] = s;
      }
    }
  }
}

// ---------------------------------------------------------------- phase 2
// Consumer thread c (0..127) owns 8 bytes of every column segment: rows
// 8c/sz .. 8c/sz + 8/sz - 1 of the item.  fp32 sums are taken per stage
// (16 columns) and added to the running total.
template <int FMT, int NR>
__device__ __forceinline__ void p2_consume_stage(const uint8_t* data, const Meta& m, const StreamArgs& a, int ct,
                                                 float (&acc)[8][NR], float (&accd)[NR][16]) {
  constexpr int SZ = Sz<FMT>::v;
  constexpr int RPT = 8 / SZ;  // rows per thread
  const int col0 = m.part * kP2Cols;
  if constexpr (FMT == 0) {
    // one row per thread; column c feeds the double-float chain c % 8:
    // (accd[rr][2q], accd[rr][2q+1]), q = c % 8
    auto column = [&](int c, float& S, float& C, int rr0) {
      const float2 f = *reinterpret_cast<const float2*>(data + c * kP2RowBytes + ct * 8);
      const float fh = f.x, fl = f.y;
      const int j = col0 + c;
      float th, tl;
      if (m.mode == 0) {
        const float2 t2 = __ldg(a.t64 + m.toff + static_cast<int64_t>(j) * NR + rr0);
        th = t2.x;
        tl = t2.y;
      } else {  // dense block: t_j = x_j (copy 0 of the input halves)
        const size_t o = static_cast<size_t>(rr0) * a.npad + m.in_off + j;
        th = __ldg(a.xs + o);
        tl = __ldg(a.xs_lo + o);
      }
      dd_acc(S, C, fh, fl, th, tl);
    };
    for (int c0 = 0; c0 < m.count; c0 += 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (c0 + q < m.count) {
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) column(c0 + q, accd[rr][2 * q], accd[rr][2 * q + 1], rr);
        }
      }
    }
  } else {
    float part[RPT][NR];
#pragma unroll
    for (int e = 0; e < RPT; ++e)
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) part[e][rr] = 0.f;
    const float* tp = a.t32 + m.toff;
#pragma unroll 4
    for (int c = 0; c < m.count; ++c) {
      const uint2 w = *reinterpret_cast<const uint2*>(data + c * kP2RowBytes + ct * 8);
      float f[RPT];
      dec8<FMT>(w, f);
      const int j = col0 + c;
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) {
        const float tj = __ldg(tp + static_cast<int64_t>(j) * NR + rr);
#pragma unroll
        for (int e = 0; e < RPT; ++e) part[e][rr] = fmaf(f[e], tj, part[e][rr]);
      }
    }
#pragma unroll
    for (int e = 0; e < RPT; ++e)
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) acc[e][rr] += part[e][rr];
  }
}

template <int NR>
__device__ __forceinline__ void p2_flush(const Meta& m, const StreamArgs& a, int ct, float (&acc)[8][NR],
                                         float (&accd)[NR][16]) {
  const int sz = fmt_size(m.fmt);
  const int rpt = 8 / sz;
  const int row0 = m.lo + ct * rpt;
  if (m.fmt == 0) {
    if (row0 < m.hi)
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) {
        float S = accd[rr][0], C = accd[rr][1];
#pragma unroll
        for (int q = 1; q < 8; ++q) dd_add(S, C, accd[rr][2 * q], accd[rr][2 * q + 1]);
        double* o = a.acc + static_cast<size_t>(rr) * a.npad + m.out_off + row0;
        atomicAdd(o, f2d_scaled(S, m.e));
        if (C != 0.f) atomicAdd(o, f2d_scaled(C, m.e));
      }
    return;
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    if (e >= rpt) break;
    const int row = row0 + e;
    if (row < m.hi)
#pragma unroll
      for (int rr = 0; rr < NR; ++rr)
        atomicAdd(a.acc + static_cast<size_t>(rr) * a.npad + m.out_off + row, f2d_scaled(acc[e][rr], m.e));
  }
}

template <int PHASE, int NR, unsigned FSET, int NST>
__device__ void consume(Smem<PHASE, FSET, NST>& sm, const StreamArgs& a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wc = warp - 1;           // consumer warp index
  const int ct = threadIdx.x - 32;   // consumer thread index (0..127)
  if constexpr (PHASE == 2) asm volatile("griddepcontrol.wait;" ::: "memory");  // t of phase 1
  int stage = 0;
  uint32_t par = 0;
  float acc1[2][NR][4];
  float acd1[2][NR][16];  // fp64 factors: double-float chains (phase 1)
  float acc2[8][NR];
  float acd2[NR][16];     // fp64 factors: double-float chains (phase 2)
  for (;;) {
    if (!mbar_wait(&sm.full[stage], par, a.status)) return;
    const Meta m = sm.meta[stage];
    if (m.item < 0) return;
    if (m.part == 0) {
      if constexpr (PHASE == 1) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) {
#pragma unroll
            for (int e = 0; e < 4; ++e) acc1[c][rr][e] = 0.f;
            if constexpr (FSET & 1u) {
#pragma unroll
              for (int e = 0; e < 16; ++e) acd1[c][rr][e] = 0.f;
            }
          }
      } else {
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
#pragma unroll
          for (int e = 0; e < 8; ++e) acc2[e][rr] = 0.f;
          if constexpr (FSET & 1u) {
#pragma unroll
            for (int e = 0; e < 16; ++e) acd2[rr][e] = 0.f;
          }
        }
      }
    }
    const uint8_t* data = sm.data[stage];
    if constexpr (PHASE == 1) {
      const float* xsm = reinterpret_cast<const float*>(sm.x[stage]);
      switch (m.fmt) {
        case 0: if constexpr (FSET & 1u) { p1_consume_stage<0, NR, XArea<FSET>::bytes>(data, xsm, m, a, wc, lane, acc1, acd1); break; } [[fallthrough]];
        case 1: if constexpr (FSET & 2u) { p1_consume_stage<1, NR, XArea<FSET>::bytes>(data, xsm, m, a, wc, lane, acc1, acd1); break; } [[fallthrough]];
        case 2: if constexpr (FSET & 4u) { p1_consume_stage<2, NR, XArea<FSET>::bytes>(data, xsm, m, a, wc, lane, acc1, acd1); break; } [[fallthrough]];
        case 3: if constexpr (FSET & 8u) { p1_consume_stage<3, NR, XArea<FSET>::bytes>(data, xsm, m, a, wc, lane, acc1, acd1); break; } [[fallthrough]];
        case 4: if constexpr (FSET & 16u) { p1_consume_stage<4, NR, XArea<FSET>::bytes>(data, xsm, m, a, wc, lane, acc1, acd1); break; } [[fallthrough]];
        default: if (lane == 0) atomicOr(a.status, 1);
      }
    } else {
      switch (m.fmt) {
        case 0: if constexpr (FSET & 1u) { p2_consume_stage<0, NR>(data, m, a, ct, acc2, acd2); break; } [[fallthrough]];
        case 1: if constexpr (FSET & 2u) { p2_consume_stage<1, NR>(data, m, a, ct, acc2, acd2); break; } [[fallthrough]];
        case 2: if constexpr (FSET & 4u) { p2_consume_stage<2, NR>(data, m, a, ct, acc2, acd2); break; } [[fallthrough]];
        case 3: if constexpr (FSET & 8u) { p2_consume_stage<3, NR>(data, m, a, ct, acc2, acd2); break; } [[fallthrough]];
        case 4: if constexpr (FSET & 16u) { p2_consume_stage<4, NR>(data, m, a, ct, acc2, acd2); break; } [[fallthrough]];
        default: if (lane == 0) atomicOr(a.status, 1);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[stage]);
    if (m.last) {
      if constexpr (PHASE == 1) p1_flush<NR>(m, a, wc, lane, acc1, acd1);
      else p2_flush<NR>(m, a, ct, acc2, acd2);
    }
    if (++stage == NST) {
      stage = 0;
      par ^= 1u;
    }
  }
}

// one pass by one CTA: barriers set up, then the producer warp and the
// consumer warps; every thread returns (also after a bounded wait expired)
template <int PHASE, int NR, unsigned FSET, int NST>
__device__ __forceinline__ void stream_body(uint8_t* smem_raw, const StreamArgs& a) {
  Smem<PHASE, FSET, NST>& sm = *reinterpret_cast<Smem<PHASE, FSET, NST>*>(smem_raw);
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], kConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (threadIdx.x < 32) produce<PHASE, FSET, NST>(sm, a);
  else consume<PHASE, NR, FSET, NST>(sm, a);
}

// after a pass in a kernel that reuses the shared memory: every thread is
// done with the barriers (no copy is in flight once the consumers have
// consumed every stage, or the producer has drained them after a timeout),
// so they are invalidated before the memory serves another purpose
template <int PHASE, unsigned FSET, int NST>
__device__ __forceinline__ void stream_teardown(uint8_t* smem_raw) {
  Smem<PHASE, FSET, NST>& sm = *reinterpret_cast<Smem<PHASE, FSET, NST>*>(smem_raw);
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < NST; ++s) {
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(saddr(&sm.full[s])) : "memory");
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(saddr(&sm.empty[s])) : "memory");
    }
  __syncthreads();
}

template <int PHASE, int NR, unsigned FSET, int NST>
__global__ void __launch_bounds__(kStreamThreads) stream_kernel(StreamArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  stream_body<PHASE, NR, FSET, NST>(smem_raw, a);
}

// launch with (pdl) or without programmatic stream serialization
template <class Kern>
cudaError_t launch_k(Kern k, int grid, size_t smem, cudaStream_t st, bool pdl, const StreamArgs& a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(kStreamThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, a);
}

template <int PHASE, int NR, unsigned FSET, int NST>
cudaError_t launch_one(const StreamArgs& a, int grid, cudaStream_t st, bool pdl) {
  const size_t smem = sizeof(Smem<PHASE, FSET, NST>);
  cudaError_t e = cudaFuncSetAttribute(stream_kernel<PHASE, NR, FSET, NST>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = launch_k(stream_kernel<PHASE, NR, FSET, NST>, grid, smem, st, pdl, a);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

template <int PHASE, int NR, unsigned FSET, int NST>
int occupancy_one() {
  const size_t smem = sizeof(Smem<PHASE, FSET, NST>);
  int b = 0;
  cudaFuncSetAttribute(stream_kernel<PHASE, NR, FSET, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, stream_kernel<PHASE, NR, FSET, NST>, kStreamThreads, smem);
  return (e != cudaSuccess || b < 1) ? 1 : b;
}

// one right-hand side: pipeline depths 3, 4 and 6 (the autotuner's choice);
// 2 and 4 right-hand sides: depth 4
template <int PHASE, unsigned FSET>
cudaError_t launch_stream_t(const StreamArgs& a, int grid, cudaStream_t st, bool pdl, int nst) {
  switch (a.nr) {
    case 1:
      if (nst == 3) return launch_one<PHASE, 1, FSET, 3>(a, grid, st, pdl);
      if (nst == 6) return launch_one<PHASE, 1, FSET, 6>(a, grid, st, pdl);
      return launch_one<PHASE, 1, FSET, kStages>(a, grid, st, pdl);
    case 2: return launch_one<PHASE, 2, FSET, kStages>(a, grid, st, pdl);
    case 4: return launch_one<PHASE, 4, FSET, kStages>(a, grid, st, pdl);
    default: return cudaErrorInvalidValue;
  }
}

template <int PHASE, unsigned FSET>
int stream_occupancy(int nr, int nst) {
  if (nr == 1) {
    if (nst == 3) return occupancy_one<PHASE, 1, FSET, 3>();
    if (nst == 6) return occupancy_one<PHASE, 1, FSET, 6>();
    return occupancy_one<PHASE, 1, FSET, kStages>();
  }
  if (nr == 2) return occupancy_one<PHASE, 2, FSET, kStages>();
  return occupancy_one<PHASE, 4, FSET, kStages>();
}

// The whole batch product in one persistent kernel (a cooperative launch:
// every CTA is resident, so the grid-wide barriers between the stages are
// safe): prep over all positions, phase 1, phase 2 and the output
// permutation.  Each stage's writes are visible to the next after the
// barrier; the input copies and t, read with non-coherent loads in phase 2,
// are written before that stage starts and not cached by it earlier.
template <unsigned FSET>
constexpr size_t batch_smem() {
  return sizeof(Smem<1, FSET, kStages>) > sizeof(Smem<2, FSET, kStages>) ? sizeof(Smem<1, FSET, kStages>)
                                                                         : sizeof(Smem<2, FSET, kStages>);
}

template <unsigned FSET>
__global__ void __launch_bounds__(kStreamThreads) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (!grid.is_valid()) {  // not a cooperative launch: no grid barrier may be used
    if (tid == 0) atomicOr(a.pass[0].status, 16);
    return;
  }
  const int64_t nth = static_cast<int64_t>(gridDim.x) * blockDim.x;
  if (tid < 2) *(tid == 0 ? a.pass[0].counter : a.pass[1].counter) = 0;
  for (int64_t p = tid; p < a.np; p += nth)
    batch_prep_position(p, a.x, a.xofs, a.perm, a.pofs, a.ns, a.count, a.np, const_cast<float*>(a.pass[0].xs),
                        const_cast<float*>(a.pass[0].xs_lo), a.pass[0].acc);
  grid.sync();
  if (a.pass[0].n_items > 0) {
    stream_body<1, 1, FSET, kStages>(smem_raw, a.pass[0]);
    stream_teardown<1, FSET, kStages>(smem_raw);
  }
  grid.sync();
  if (a.pass[1].n_items > 0) {
    stream_body<2, 1, FSET, kStages>(smem_raw, a.pass[1]);
    stream_teardown<2, FSET, kStages>(smem_raw);
  }
  grid.sync();
  for (int64_t p = tid; p < a.np; p += nth)
    batch_finish_position(p, a.pass[1].acc, a.xofs, a.perm, a.pofs, a.ns, a.count, a.y);
}

template <unsigned FSET>
int batch_occupancy() {
  const size_t smem = batch_smem<FSET>();
  int b = 0;
  cudaFuncSetAttribute(batch_kernel<FSET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_kernel<FSET>, kStreamThreads, smem);
  return e == cudaSuccess ? b : 0;
}

template <unsigned FSET>
cudaError_t launch_batch_t(const BatchArgs& a, int grid, cudaStream_t st) {
  const size_t smem = batch_smem<FSET>();
  cudaError_t e = cudaFuncSetAttribute(batch_kernel<FSET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(kStreamThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, batch_kernel<FSET>, a);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace

bool stream_depth_ok(int nst) { return nst == 3 || nst == 4 || nst == 6; }

cudaError_t launch_stream(int phase, unsigned fset, const StreamArgs& a, int grid, cudaStream_t st, bool pdl,
                          int nst) {
  if (a.n_items == 0) return cudaSuccess;
  if (phase == 1) pdl = false;  // phase 1 needs the prep launch complete before it starts
  if (!stream_depth_ok(nst)) nst = kStages;
  if (fset == kSetF64)
    return phase == 1 ? launch_stream_t<1, kSetF64>(a, grid, st, false, nst)
                      : launch_stream_t<2, kSetF64>(a, grid, st, pdl, nst);
  if (fset == kSetF32)
    return phase == 1 ? launch_stream_t<1, kSetF32>(a, grid, st, false, nst)
                      : launch_stream_t<2, kSetF32>(a, grid, st, pdl, nst);
  return phase == 1 ? launch_stream_t<1, kSetAll>(a, grid, st, false, nst)
                    : launch_stream_t<2, kSetAll>(a, grid, st, pdl, nst);
}

int stream_blocks_per_sm(int phase, unsigned fset, int nr, int nst) {
  if (!stream_depth_ok(nst)) nst = kStages;
  if (fset == kSetF64) return phase == 1 ? stream_occupancy<1, kSetF64>(nr, nst) : stream_occupancy<2, kSetF64>(nr, nst);
  if (fset == kSetF32) return phase == 1 ? stream_occupancy<1, kSetF32>(nr, nst) : stream_occupancy<2, kSetF32>(nr, nst);
  return phase == 1 ? stream_occupancy<1, kSetAll>(nr, nst) : stream_occupancy<2, kSetAll>(nr, nst);
}

int batch_persistent_grid(unsigned fset, int sms) {
  const int occ = fset == kSetF64 ? batch_occupancy<kSetF64>()
                                  : (fset == kSetF32 ? batch_occupancy<kSetF32>() : batch_occupancy<kSetAll>());
  return occ * sms;
}

cudaError_t launch_batch_persistent(unsigned fset, const BatchArgs& a, int grid, cudaStream_t st) {
  if (grid < 1) return cudaErrorInvalidValue;
  if (fset == kSetF64) return launch_batch_t<kSetF64>(a, grid, st);
  if (fset == kSetF32) return launch_batch_t<kSetF32>(a, grid, st);
  return launch_batch_t<kSetAll>(a, grid, st);
}

int stream_rows_per_item(int fmt) { return kP2RowBytes / (fmt == 0 ? 8 : (fmt == 1 ? 4 : (fmt == 4 ? 1 : 2))); }
int stream_cols_per_item() { return kP1Cols; }

}  // namespace dev
}  // namespace hh
