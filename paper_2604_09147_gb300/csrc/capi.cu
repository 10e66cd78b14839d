// C-ABI of the H_h library (declarations and contracts in include/hh.h):
// handle life cycle, upload of the block tables into device descriptors,
// the warp work lists, and the launch sequence of one product.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/hh.h"
#include "hh_device.h"
#include "hh_host.h"

using hh::dev::Item;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

struct CudaError : std::runtime_error {
  explicit CudaError(const std::string& s) : std::runtime_error(s) {}
};

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw CudaError(std::string(what) + ": " + cudaGetErrorString(e));
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct hh_matrix {
  hh::HostMatrix H;
  hh::Summary S;
  int device = -1;
  int sms = 0;
  int64_t npad = 0;
  int64_t t32_elems = 0, t64_elems = 0;  // per right-hand side
  uint8_t* d_arena = nullptr;
  int32_t* d_perm = nullptr;
  int* d_status = nullptr;
  void* d_ws = nullptr;
  size_t ws_bytes = 0;
  double* d_stage = nullptr;  // hh_matvec_host staging buffers (2 x n x stage_cols)
  int stage_cols = 0;
  // streaming passes (stream.cu): descriptors and items per [direction][phase]
  hh::dev::StreamDesc* d_sdesc[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  Item* d_sitems[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int n_sitems[2][2] = {{0, 0}, {0, 0}};
  double* d_dense_pad = nullptr;  // dense blocks, column-major, ld rounded up to even
  int sgrid[3][5] = {};
  unsigned fset = hh::dev::kSetAll;  // kernel variant covering the formats present
};

namespace {

void free_device(hh_matrix* h) {
  if (h->device < 0) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  cudaFree(h->d_arena);
  cudaFree(h->d_perm);
  for (int d = 0; d < 2; ++d)
    for (int p = 0; p < 2; ++p) {
      cudaFree(h->d_sdesc[d][p]);
      cudaFree(h->d_sitems[d][p]);
    }
  cudaFree(h->d_dense_pad);
  cudaFree(h->d_status);
  cudaFree(h->d_ws);
  cudaFree(h->d_stage);
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
}

template <class T>
T* upload(const std::vector<T>& v) {
  T* p = nullptr;
  size_t bytes = std::max<size_t>(v.size() * sizeof(T), 256);
  ck(cudaMalloc(&p, bytes), "cudaMalloc");
  if (!v.empty()) ck(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "cudaMemcpy");
  return p;
}

int next_pow2_32(int64_t v) {
  int g = 1;
  while (g < v && g < 32) g <<= 1;
  return g;
}

// Descriptors and work items of the streaming passes (stream.cu).
void upload_stream(hh_matrix* h, const std::vector<int64_t>& toff) {
  using hh::dev::StreamDesc;
  const hh::HostMatrix& H = h->H;
  // dense blocks with an even leading dimension (16-byte aligned columns)
  std::vector<int64_t> doff(H.dense.size());
  int64_t dtot = 0;
  for (size_t q = 0; q < H.dense.size(); ++q) {
    doff[q] = dtot;
    dtot += ((H.dense[q].m + 1) / 2 * 2) * H.dense[q].n;
  }
  // each block scaled by a power of two so that its largest magnitude lies in
  // (1/2, 1] (exact; the kernels split fp64 values into fp32 halves)
  std::vector<double> dpad(static_cast<size_t>(dtot), 0.0);
  std::vector<int32_t> dexp(H.dense.size(), 0);
  for (size_t q = 0; q < H.dense.size(); ++q) {
    const hh::DenseBlock& D = H.dense[q];
    const int64_t ld = (D.m + 1) / 2 * 2;
    double mx = 0.0;
    for (int64_t i = 0; i < D.m * D.n; ++i) mx = std::max(mx, std::fabs(H.dense_data[D.d_off + i]));
    int ex = 0;
    if (mx > 0.0) {
      std::frexp(mx, &ex);  // mx = f 2^ex, f in [1/2, 1)
      while (std::ldexp(mx, -ex) > 1.0) ++ex;
    }
    dexp[q] = ex;
    for (int64_t c = 0; c < D.n; ++c)
      for (int64_t r = 0; r < D.m; ++r)
        dpad[doff[q] + c * ld + r] = std::ldexp(H.dense_data[D.d_off + c * D.m + r], -ex);
  }
  h->d_dense_pad = upload(dpad);
  const int cols1 = hh::dev::stream_cols_per_item();
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<StreamDesc> desc[2];
    struct Costed {
      Item it;
      double cost;
    };
    std::vector<Costed> items[2];
    auto add_cols = [&](int phase, int di, int64_t rows, int64_t cols, int sz) {
      for (int64_t j = 0; j < cols; j += cols1) {
        int64_t hi = std::min<int64_t>(cols, j + cols1);
        items[phase].push_back({{0, di, (int32_t)j, (int32_t)hi}, double(hi - j) * double(rows * sz)});
      }
    };
    auto add_rows = [&](int phase, int di, int64_t rows, int64_t cols, int fmt) {
      const int64_t rt = hh::dev::stream_rows_per_item(fmt);
      for (int64_t r = 0; r < rows; r += rt) {
        int64_t hi = std::min<int64_t>(rows, r + rt);
        items[phase].push_back({{0, di, (int32_t)r, (int32_t)hi}, double(hi - r) * double(cols * hh::fmt_bytes(fmt))});
      }
    };
    for (size_t b = 0; b < H.lr.size(); ++b) {
      const hh::LRBlock& B = H.lr[b];
      if (B.k == 0) continue;
      const uint8_t* U = h->d_arena + B.u_off;
      const uint8_t* V = h->d_arena + B.v_off;
      StreamDesc s1, s2;
      std::memset(&s1, 0, sizeof(s1));
      std::memset(&s2, 0, sizeof(s2));
      s1.f = dir == 0 ? V : U;
      s1.ld = dir == 0 ? B.ldv : B.ldu;
      s1.rows = (int32_t)(dir == 0 ? B.n : B.m);
      s1.cols = B.k;
      s1.fmt = B.fmt;
      s1.in_off = (int32_t)(dir == 0 ? B.col_off : B.row_off);
      s1.toff = toff[b];
      s2.f = dir == 0 ? U : V;
      s2.ld = dir == 0 ? B.ldu : B.ldv;
      s2.rows = (int32_t)(dir == 0 ? B.m : B.n);
      s2.cols = B.k;
      s2.fmt = B.fmt;
      s2.e = B.exp_u + B.exp_v;
      s2.out_off = (int32_t)(dir == 0 ? B.row_off : B.col_off);
      s2.toff = toff[b];
      desc[0].push_back(s1);
      add_cols(0, (int)desc[0].size() - 1, s1.rows, s1.cols, hh::fmt_bytes(B.fmt));
      desc[1].push_back(s2);
      add_rows(1, (int)desc[1].size() - 1, s2.rows, s2.cols, B.fmt);
    }
    for (size_t q = 0; q < H.dense.size(); ++q) {
      const hh::DenseBlock& D = H.dense[q];
      StreamDesc s;
      std::memset(&s, 0, sizeof(s));
      s.f = reinterpret_cast<const uint8_t*>(h->d_dense_pad + doff[q]);
      s.ld = (D.m + 1) / 2 * 2;
      s.rows = (int32_t)D.m;
      s.cols = (int32_t)D.n;
      s.fmt = hh::F64;
      s.mode = 1;
      s.e = dexp[q];
      if (dir == 0) {  // forward: phase 2, y[row_off + i] += sum_j D x[col_off + j]
        s.in_off = (int32_t)D.col_off;
        s.out_off = (int32_t)D.row_off;
        desc[1].push_back(s);
        add_rows(1, (int)desc[1].size() - 1, s.rows, s.cols, hh::F64);
      } else {         // transpose: phase 1, xbar[col_off + j] += sum_i D y[row_off + i]
        s.in_off = (int32_t)D.row_off;
        s.out_off = (int32_t)D.col_off;
        desc[0].push_back(s);
        add_cols(0, (int)desc[0].size() - 1, s.rows, s.cols, 8);
      }
    }
    for (int p = 0; p < 2; ++p) {
      std::stable_sort(items[p].begin(), items[p].end(),
                       [](const Costed& x, const Costed& y) { return x.cost > y.cost; });
      std::vector<Item> flat;
      for (auto& c : items[p]) flat.push_back(c.it);
      h->d_sdesc[dir][p] = upload(desc[p]);
      h->d_sitems[dir][p] = upload(flat);
      h->n_sitems[dir][p] = (int)flat.size();
    }
  }
}

void upload_matrix(hh_matrix* h, int device) {
  const hh::HostMatrix& H = h->H;
  ck(cudaSetDevice(device), "cudaSetDevice");
  h->device = device;
  ck(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device), "device attribute");
  h->d_arena = upload(H.arena);
  h->d_perm = upload(H.perm);
  h->npad = (H.n + 32 + 3) / 4 * 4;
  // t offsets per block (room for kMaxNR right-hand sides)
  std::vector<int64_t> toff(H.lr.size(), 0);
  h->t32_elems = h->t64_elems = 0;
  for (size_t b = 0; b < H.lr.size(); ++b) {
    int64_t& tot = H.lr[b].fmt == hh::F64 ? h->t64_elems : h->t32_elems;
    toff[b] = tot * hh::dev::kMaxNR;
    tot += H.lr[b].k;
  }
  upload_stream(h, toff);
  ck(cudaMalloc(&h->d_status, 256), "cudaMalloc");
  ck(cudaMemset(h->d_status, 0, 256), "cudaMemset");
  unsigned present = 0;
  for (const hh::LRBlock& B : H.lr) present |= 1u << B.fmt;
  h->fset = hh::dev::pass_set_for(present);
  for (int phase = 1; phase <= 2; ++phase)
    for (int nr : {1, 2, 4}) h->sgrid[phase][nr] = h->sms * hh::dev::stream_blocks_per_sm(phase, h->fset, nr);
  size_t ws = 0;
  hh_workspace_bytes(h, &ws);
  ck(cudaMalloc(&h->d_ws, ws), "cudaMalloc workspace");
  h->ws_bytes = ws;
  ck(cudaDeviceSynchronize(), "upload");
}

struct WsView {
  float* xs;
  float* xs_lo;
  double* acc;
  float* t32;
  float2* t64;
  int* counters;
};

size_t ws_layout(const hh_matrix* h, WsView* v, char* base) {
  const int R = hh::dev::kMaxNR;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return base ? base + o : nullptr;
  };
  float* xs = (float*)take(sizeof(float) * 4 * R * h->npad);
  float* xs_lo = (float*)take(sizeof(float) * 4 * R * h->npad);
  double* acc = (double*)take(sizeof(double) * R * h->npad);
  float* t32 = (float*)take(sizeof(float) * std::max<int64_t>(1, h->t32_elems * R));
  float2* t64 = (float2*)take(sizeof(float2) * std::max<int64_t>(1, h->t64_elems * R));
  int* counters = (int*)take(256);
  if (v) *v = {xs, xs_lo, acc, t32, t64, counters};
  return off;
}

int run_product(hh_matrix* h, int dir, const double* in, double* out, int nrhs, int64_t ld_in,
                int64_t ld_out, void* ws, size_t ws_bytes, cudaStream_t st, cudaEvent_t* ev = nullptr) {
  if (h->device < 0) return fail(HH_ENOTSUP, "handle has no device data (built with device = -1)");
  if (!in || !out || nrhs < 1 || ld_in < h->H.n || ld_out < h->H.n)
    return fail(HH_EINVAL, "bad vector arguments (null pointer, nrhs < 1 or ld < n)");
  const size_t span_in = (size_t)((nrhs - 1) * ld_in + h->H.n) * 8;
  const size_t span_out = (size_t)((nrhs - 1) * ld_out + h->H.n) * 8;
  const char* a0 = (const char*)in;
  const char* b0 = (const char*)out;
  if (a0 < b0 + span_out && b0 < a0 + span_in) return fail(HH_EINVAL, "input and output overlap");
  size_t need = ws_layout(h, nullptr, nullptr);
  if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return fail(HH_EINVAL, "workspace too small or misaligned");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess)
    return fail(HH_ECUDA, "cudaSetDevice failed");
  WsView w;
  ws_layout(h, &w, (char*)ws);
  for (int rb = 0; rb < nrhs;) {
    const int rem = nrhs - rb;
    const int nr = rem >= 4 ? 4 : (rem >= 2 ? 2 : 1);
    if (ev) cudaEventRecord(ev[0], st);
    cudaError_t e = hh::dev::launch_prep(in + (int64_t)rb * ld_in, ld_in, nr, h->d_perm, h->H.n, h->npad,
                                         w.xs, w.xs_lo, w.acc, st, w.counters);
    for (int phase = 1; phase <= 2 && e == cudaSuccess; ++phase) {
      if (ev) cudaEventRecord(ev[phase], st);
      hh::dev::StreamArgs s;
      std::memset(&s, 0, sizeof(s));
      s.desc = h->d_sdesc[dir][phase - 1];
      s.items = h->d_sitems[dir][phase - 1];
      s.n_items = h->n_sitems[dir][phase - 1];
      s.nr = nr;
      s.npad = h->npad;
      s.xs = w.xs;
      s.xs_lo = w.xs_lo;
      s.t32 = w.t32;
      s.t64 = w.t64;
      s.acc = w.acc;
      s.status = h->d_status;
      s.counter = w.counters + (phase - 1);
      int grid = std::max(1, std::min(h->sgrid[phase][nr], s.n_items));
      e = hh::dev::launch_stream(phase, h->fset, s, grid, st);
    }
    if (ev) cudaEventRecord(ev[3], st);
    if (e == cudaSuccess)
      e = hh::dev::launch_finish(w.acc, nr, h->d_perm, h->H.n, h->npad, out + (int64_t)rb * ld_out, ld_out, st);
    if (ev) cudaEventRecord(ev[4], st);
    if (e != cudaSuccess) {
      if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
      return fail(HH_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    }
    rb += nr;
  }
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  return HH_OK;
}

hh_matrix* make_handle() { return new (std::nothrow) hh_matrix(); }

int finish_construction(hh_matrix* h, int device, hh_handle* out) {
  try {
    h->S = hh::summarize(h->H);
    if (device >= 0) upload_matrix(h, device);
  } catch (const CudaError& e) {
    free_device(h);
    delete h;
    return fail(HH_ECUDA, e.what());
  } catch (const std::bad_alloc&) {
    free_device(h);
    delete h;
    return fail(HH_ENOMEM, "out of host memory");
  }
  *out = h;
  return HH_OK;
}

}  // namespace

extern "C" {

const char* hh_last_error(void) { return g_last_error.c_str(); }

int hh_build(const double* points, int64_t n, int dim, int kernel, double kernel_param, int leaf_size,
             double eta, int switch_level, double tol, uint32_t fmt_mask, uint64_t seed, int device,
             hh_handle* out) {
  if (!out) return fail(HH_EINVAL, "out is NULL");
  *out = nullptr;
  if (!points) return fail(HH_EINVAL, "points is NULL");
  if (device < -1) return fail(HH_EINVAL, "device must be >= -1");
  hh_matrix* h = make_handle();
  if (!h) return fail(HH_ENOMEM, "out of host memory");
  try {
    hh::BuildParams p{kernel, kernel_param, leaf_size, eta, switch_level, tol, fmt_mask, seed, 0};
    if (const char* t = std::getenv("HH_BUILD_THREADS")) p.threads = std::atoi(t);
    hh::build(points, n, dim, p, h->H);
  } catch (const std::domain_error& e) {
    delete h;
    return fail(HH_ENOTSUP, e.what());
  } catch (const std::invalid_argument& e) {
    delete h;
    return fail(HH_EINVAL, e.what());
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(HH_ENOMEM, "out of host memory during build");
  } catch (const std::exception& e) {
    delete h;
    return fail(HH_EINVAL, e.what());
  }
  return finish_construction(h, device, out);
}

int hh_load(const char* path, int device, hh_handle* out) {
  if (!out) return fail(HH_EINVAL, "out is NULL");
  *out = nullptr;
  if (!path) return fail(HH_EINVAL, "path is NULL");
  hh_matrix* h = make_handle();
  if (!h) return fail(HH_ENOMEM, "out of host memory");
  try {
    hh::load_file(path, h->H);
  } catch (const hh::IoError& e) {
    delete h;
    return fail(HH_EIO, e.what());
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(HH_ENOMEM, "out of host memory while loading");
  } catch (const std::exception& e) {
    delete h;
    return fail(HH_EINVAL, e.what());
  }
  return finish_construction(h, device, out);
}

int hh_reencode(hh_handle src, uint32_t fmt_mask, int device, hh_handle* out) {
  if (!out) return fail(HH_EINVAL, "out is NULL");
  *out = nullptr;
  if (!src) return fail(HH_EINVAL, "null handle");
  if (device < -1) return fail(HH_EINVAL, "device must be >= -1");
  hh_matrix* h = make_handle();
  if (!h) return fail(HH_ENOMEM, "out of host memory");
  try {
    int threads = 0;
    if (const char* t = std::getenv("HH_BUILD_THREADS")) threads = std::atoi(t);
    hh::reencode(src->H, fmt_mask, threads, h->H);
  } catch (const std::domain_error& e) {
    delete h;
    return fail(HH_ENOTSUP, e.what());
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(HH_ENOMEM, "out of host memory");
  } catch (const std::exception& e) {
    delete h;
    return fail(HH_EINVAL, e.what());
  }
  return finish_construction(h, device, out);
}

int hh_save(hh_handle h, const char* path) {
  if (!h || !path) return fail(HH_EINVAL, "null argument");
  try {
    hh::save_file(h->H, path);
  } catch (const std::exception& e) {
    return fail(HH_EIO, e.what());
  }
  return HH_OK;
}

int hh_info(hh_handle h, hh_info_t* o) {
  if (!h || !o) return fail(HH_EINVAL, "null argument");
  std::memset(o, 0, sizeof(*o));
  const hh::HostMatrix& H = h->H;
  const hh::Summary& S = h->S;
  o->n = H.n;
  o->dim = H.dim;
  o->L = H.L;
  o->ell = H.ell;
  o->leaf_size = H.leaf;
  o->kernel = H.kernel;
  o->device = h->device;
  o->eta = H.eta;
  o->tol = H.tol;
  o->kernel_param = H.kparam;
  o->n_lowrank = (int64_t)H.lr.size();
  o->n_dense = (int64_t)H.dense.size();
  for (int f = 0; f < hh::NFMT; ++f) {
    o->blocks_per_fmt[f] = S.blocks_per_fmt[f];
    o->factor_bytes_per_fmt[f] = S.bytes_per_fmt[f];
  }
  o->dense_bytes = S.dense_bytes;
  o->u_bytes = S.u_bytes;
  o->v_bytes = S.v_bytes;
  o->max_rank = S.max_rank;
  o->storage_amp = S.storage_amp;
  o->storage_fp64 = S.storage_fp64;
  o->bytes_per_matvec = S.bytes_per_matvec;
  o->flops_per_matvec = S.flops_per_matvec;
  o->norm_ht = H.norm_ht;
  for (size_t l = 0; l < S.csp.size() && l < HH_MAX_LEVELS; ++l) o->csp[l] = S.csp[l];
  o->bound_thm42 = S.bound42;
  o->bound_thm44 = S.bound44;
  o->bound_rounding = S.bound_round;
  o->build_seconds = H.build_seconds;
  return HH_OK;
}

int hh_perm(hh_handle h, int32_t* perm) {
  if (!h || !perm) return fail(HH_EINVAL, "null argument");
  std::memcpy(perm, h->H.perm.data(), h->H.perm.size() * sizeof(int32_t));
  return HH_OK;
}

int hh_workspace_bytes(hh_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(HH_EINVAL, "null argument");
  *bytes = ws_layout(h, nullptr, nullptr);
  return HH_OK;
}

int hh_matvec(hh_handle h, const double* x, double* y, int nrhs, int64_t ldx, int64_t ldy, void* stream) {
  if (!h) return fail(HH_EINVAL, "null handle");
  return run_product(h, 0, x, y, nrhs, ldx, ldy, h->d_ws, h->ws_bytes, (cudaStream_t)stream);
}

int hh_matvec_T(hh_handle h, const double* ybar, double* xbar, int nrhs, int64_t ldy, int64_t ldx,
                void* stream) {
  if (!h) return fail(HH_EINVAL, "null handle");
  return run_product(h, 1, ybar, xbar, nrhs, ldy, ldx, h->d_ws, h->ws_bytes, (cudaStream_t)stream);
}

int hh_matvec_ws(hh_handle h, int transpose, const double* in, double* out, int nrhs, int64_t ld_in,
                 int64_t ld_out, void* workspace, size_t workspace_bytes, void* stream) {
  if (!h) return fail(HH_EINVAL, "null handle");
  return run_product(h, transpose ? 1 : 0, in, out, nrhs, ld_in, ld_out, workspace, workspace_bytes,
                     (cudaStream_t)stream);
}

int hh_matvec_timed(hh_handle h, int transpose, const double* in, double* out, int nrhs, int64_t ld_in,
                    int64_t ld_out, void* stream, float* ms) {
  if (!h || !ms) return fail(HH_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > hh::dev::kMaxNR || nrhs == 3) return fail(HH_EINVAL, "nrhs must be 1, 2 or 4");
  if (h->device < 0) return fail(HH_ENOTSUP, "handle has no device data");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  cudaEvent_t ev[5];
  int made = 0;
  for (; made < 5; ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
  int rc = made == 5 ? HH_OK : fail(HH_ECUDA, "cudaEventCreate failed");
  if (rc == HH_OK)
    rc = run_product(h, transpose ? 1 : 0, in, out, nrhs, ld_in, ld_out, h->d_ws, h->ws_bytes,
                     (cudaStream_t)stream, ev);
  if (rc == HH_OK && cudaEventSynchronize(ev[4]) != cudaSuccess) rc = fail(HH_ECUDA, "event synchronize failed");
  for (int i = 0; rc == HH_OK && i < 4; ++i)
    if (cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]) != cudaSuccess) rc = fail(HH_ECUDA, "event timing failed");
  for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  return rc;
}

int hh_matvec_host(hh_handle h, int transpose, const double* x_host, double* y_host, int nrhs,
                   void* stream) {
  if (!h || !x_host || !y_host || nrhs < 1) return fail(HH_EINVAL, "bad arguments");
  if (h->device < 0) return fail(HH_ENOTSUP, "handle has no device data");
  cudaStream_t st = (cudaStream_t)stream;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  const int64_t n = h->H.n;
  if (h->stage_cols < nrhs) {
    cudaStreamSynchronize(st);
    cudaFree(h->d_stage);
    h->d_stage = nullptr;
    h->stage_cols = 0;
    if (cudaMalloc(&h->d_stage, sizeof(double) * 2 * n * nrhs) != cudaSuccess) {
      if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
      return fail(HH_ENOMEM, "cannot allocate staging buffers");
    }
    h->stage_cols = nrhs;
  }
  double* dx = h->d_stage;
  double* dy = h->d_stage + n * h->stage_cols;
  int rc = HH_OK;
  if (cudaMemcpyAsync(dx, x_host, sizeof(double) * n * nrhs, cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = fail(HH_ECUDA, "host-to-device copy failed");
  if (rc == HH_OK) rc = run_product(h, transpose ? 1 : 0, dx, dy, nrhs, n, n, h->d_ws, h->ws_bytes, st);
  if (rc == HH_OK &&
      cudaMemcpyAsync(y_host, dy, sizeof(double) * n * nrhs, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = fail(HH_ECUDA, "device-to-host copy failed");
  if (rc == HH_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(HH_ECUDA, "stream synchronize failed");
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  return rc;
}

int hh_matvec_batched(const hh_handle* hs, int count, const double* const* xs, double* const* ys,
                      void* stream) {
  if (count < 0 || (count > 0 && (!hs || !xs || !ys))) return fail(HH_EINVAL, "bad batch arguments");
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return fail(HH_EINVAL, "null handle in batch");
    if (i > 0 && hs[i]->device != hs[0]->device) return fail(HH_EINVAL, "handles on different devices");
  }
  for (int i = 0; i < count; ++i) {
    int rc = hh_matvec(hs[i], xs[i], ys[i], 1, hs[i]->H.n, hs[i]->H.n, stream);
    if (rc != HH_OK) return rc;
  }
  return HH_OK;
}

int hh_sync_status(hh_handle h, void* stream) {
  if (!h) return fail(HH_EINVAL, "null handle");
  if (h->device < 0) return HH_OK;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  int word = 0;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(&word, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return fail(HH_ECUDA, std::string("sync failed: ") + cudaGetErrorString(e));
  if (word & 4) return fail(HH_ETIMEOUT, "a bounded device wait expired (status word " + std::to_string(word) + ")");
  if (word != 0) return fail(HH_EDEVICE, "device status word " + std::to_string(word));
  return HH_OK;
}

void hh_free(hh_handle h) {
  if (!h) return;
  free_device(h);
  delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free product (hh_matvec_noalloc, see include/hh.h).
//
// Some callers cannot allocate device memory at call time: a host framework
// that owns every device allocation (a serving runtime with a fixed memory
// budget, a plugin host), or a latency-critical loop in which cudaMalloc's
// implicit device synchronisation is not acceptable.  For them the product's
// scratch (shifted input copies, output accumulator, t arenas for one
// right-hand side) lives in one fixed file-scope device array that every GPU
// holds from the moment it loads this library until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};  // device address of g_noalloc_scratch per device

// Device address of the scratch array on the current device (looked up once
// per device; host code must not use the symbol itself as an address).
int noalloc_scratch(int device, void** ptr) {
  if (device < 0 || device >= kNoAllocMaxDevices) return fail(HH_ENOTSUP, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(HH_ECUDA, std::string("cudaGetSymbolAddress(scratch) failed: ") + cudaGetErrorString(e));
    g_noalloc_addr[device] = p;
  }
  *ptr = g_noalloc_addr[device];
  return HH_OK;
}

}  // namespace

extern "C" int hh_matvec_noalloc(hh_handle h, int transpose, const double* in, double* out, void* stream) {
  if (!h || !in || !out) return fail(HH_EINVAL, "null argument");
  // scratch for one right-hand side, in the layout of the handle workspace
  const int64_t npad = (h->H.n + 32 + 3) / 4 * 4;
  int64_t t32 = 0, t64 = 0;
  for (const hh::LRBlock& b : h->H.lr) (b.fmt == hh::F64 ? t64 : t32) += b.k;
  const size_t need = align256(sizeof(float) * 4 * npad) + align256(sizeof(float) * 4 * npad) +
                      align256(sizeof(double) * npad) +
                      align256(sizeof(float) * std::max<int64_t>(1, t32 * hh::dev::kMaxNR)) +
                      align256(sizeof(float2) * std::max<int64_t>(1, t64 * hh::dev::kMaxNR)) + 256;
  if (need > kNoAllocScratchBytes)
    return fail(HH_EINVAL, "hh_matvec_noalloc: this matrix needs " + std::to_string(need) +
                               " bytes of scratch, more than the fixed " +
                               std::to_string(kNoAllocScratchBytes) + " bytes; use hh_matvec or hh_matvec_ws");
  if (h->device < 0) return fail(HH_ENOTSUP, "handle has no device data (built with device = -1)");
  const char* a0 = (const char*)in;
  const char* b0 = (const char*)out;
  const size_t span = (size_t)h->H.n * sizeof(double);
  if (a0 < b0 + span && b0 < a0 + span) return fail(HH_EINVAL, "input and output overlap");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess) return fail(HH_ECUDA, "cudaSetDevice failed");
  void* base = nullptr;
  int rc = noalloc_scratch(h->device, &base);
  if (rc == HH_OK) {
    char* p = (char*)base;
    float* xs = (float*)p;
    p += align256(sizeof(float) * 4 * npad);
    float* xs_lo = (float*)p;
    p += align256(sizeof(float) * 4 * npad);
    double* acc = (double*)p;
    p += align256(sizeof(double) * npad);
    float* tt32 = (float*)p;
    p += align256(sizeof(float) * std::max<int64_t>(1, t32 * hh::dev::kMaxNR));
    float2* tt64 = (float2*)p;
    const int dir = transpose ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    int* counters = (int*)(p + align256(sizeof(float2) * std::max<int64_t>(1, t64 * hh::dev::kMaxNR)));
    cudaError_t e = hh::dev::launch_prep(in, h->H.n, 1, h->d_perm, h->H.n, npad, xs, xs_lo, acc, st, counters);
    for (int phase = 1; phase <= 2 && e == cudaSuccess; ++phase) {
      hh::dev::StreamArgs s;
      std::memset(&s, 0, sizeof(s));
      s.desc = h->d_sdesc[dir][phase - 1];
      s.items = h->d_sitems[dir][phase - 1];
      s.n_items = h->n_sitems[dir][phase - 1];
      s.nr = 1;
      s.npad = npad;
      s.xs = xs;
      s.xs_lo = xs_lo;
      s.t32 = tt32;
      s.t64 = tt64;
      s.acc = acc;  // cleared by the prep launch on every call
      s.status = h->d_status;
      s.counter = counters + (phase - 1);
      int grid = std::max(1, std::min(h->sgrid[phase][1], s.n_items));
      e = hh::dev::launch_stream(phase, h->fset, s, grid, st);
    }
    if (e == cudaSuccess) e = hh::dev::launch_finish(acc, 1, h->d_perm, h->H.n, npad, out, h->H.n, st);
    if (e != cudaSuccess) rc = fail(HH_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  }
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  return rc;
}
