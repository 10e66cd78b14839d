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

using hh::dev::BlkDesc;
using hh::dev::DenseDesc;
using hh::dev::Item;
using hh::dev::PassArgs;

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
  double* d_dense = nullptr;
  int32_t* d_perm = nullptr;
  BlkDesc* d_blk[2] = {nullptr, nullptr};
  DenseDesc* d_dns[2] = {nullptr, nullptr};
  Item* d_items[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int n_items[2][2] = {{0, 0}, {0, 0}};
  int* d_status = nullptr;
  void* d_ws = nullptr;
  size_t ws_bytes = 0;
  double* d_stage = nullptr;  // hh_matvec_host staging buffers (2 x n x stage_cols)
  int stage_cols = 0;
  int grid[3][5] = {};  // [phase][nr]
  unsigned fset = hh::dev::kSetAll;  // kernel variant covering the formats present
};

namespace {

void free_device(hh_matrix* h) {
  if (h->device < 0) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  cudaFree(h->d_arena);
  cudaFree(h->d_dense);
  cudaFree(h->d_perm);
  for (int d = 0; d < 2; ++d) {
    cudaFree(h->d_blk[d]);
    cudaFree(h->d_dns[d]);
    for (int p = 0; p < 2; ++p) cudaFree(h->d_items[d][p]);
  }
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

// Work lists of one direction (0: forward, 1: transpose).
void make_items(const hh::HostMatrix& H, int dir, std::vector<Item>& p1, std::vector<Item>& p2) {
  struct Costed {
    Item it;
    double cost;
  };
  std::vector<Costed> c1, c2;
  for (size_t b = 0; b < H.lr.size(); ++b) {
    const hh::LRBlock& B = H.lr[b];
    if (B.k == 0) continue;
    const int sz = hh::fmt_bytes(B.fmt);
    const int64_t n1 = dir == 0 ? B.n : B.m;
    const int64_t n2 = dir == 0 ? B.m : B.n;
    // phase 1: columns of f1, about 32 KB of factor data per item
    const int vw1 = 16 / sz;
    const int C1 = 32 / next_pow2_32((n1 + vw1 - 1) / vw1);
    int64_t cols = std::max<int64_t>(1, 32768 / std::max<int64_t>(1, n1 * sz));
    cols = std::max<int64_t>(C1, cols / C1 * C1);
    for (int64_t j = 0; j < B.k; j += cols) {
      int64_t hi = std::min<int64_t>(B.k, j + cols);
      c1.push_back({{0, (int32_t)b, (int32_t)j, (int32_t)hi}, double(hi - j) * double(n1 * sz)});
    }
    // phase 2: rows of f2, one 16-byte vector per lane (8 bytes for e4m3)
    const int lb = B.fmt == hh::E4M3 ? 8 : 16;
    const int64_t rows = 32 * (lb / sz);
    for (int64_t r = 0; r < n2; r += rows) {
      int64_t hi = std::min<int64_t>(n2, r + rows);
      c2.push_back({{1, (int32_t)b, (int32_t)r, (int32_t)hi}, double(hi - r) * double(B.k * sz)});
    }
  }
  for (size_t d = 0; d < H.dense.size(); ++d) {
    const hh::DenseBlock& D = H.dense[d];
    if (dir == 0) {
      for (int64_t r = 0; r < D.m; r += 32) {
        int64_t hi = std::min<int64_t>(D.m, r + 32);
        c2.push_back({{2, (int32_t)d, (int32_t)r, (int32_t)hi}, double(hi - r) * double(D.n * 8)});
      }
    } else {
      const int C = 32 / next_pow2_32(D.m);
      const int64_t cols = std::max<int64_t>(C, 8);
      for (int64_t c = 0; c < D.n; c += cols) {
        int64_t hi = std::min<int64_t>(D.n, c + cols);
        c2.push_back({{3, (int32_t)d, (int32_t)c, (int32_t)hi}, double(hi - c) * double(D.m * 8)});
      }
    }
  }
  auto by_cost = [](const Costed& a, const Costed& b) { return a.cost > b.cost; };
  std::stable_sort(c1.begin(), c1.end(), by_cost);
  std::stable_sort(c2.begin(), c2.end(), by_cost);
  p1.clear();
  p2.clear();
  for (auto& c : c1) p1.push_back(c.it);
  for (auto& c : c2) p2.push_back(c.it);
}

void upload_matrix(hh_matrix* h, int device) {
  const hh::HostMatrix& H = h->H;
  ck(cudaSetDevice(device), "cudaSetDevice");
  h->device = device;
  ck(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device), "device attribute");
  h->d_arena = upload(H.arena);
  h->d_dense = upload(H.dense_data);
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
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<BlkDesc> bd(H.lr.size());
    for (size_t b = 0; b < H.lr.size(); ++b) {
      const hh::LRBlock& B = H.lr[b];
      const uint8_t* U = h->d_arena + B.u_off;
      const uint8_t* V = h->d_arena + B.v_off;
      BlkDesc& d = bd[b];
      std::memset(&d, 0, sizeof(d));
      d.f1 = dir == 0 ? V : U;
      d.f2 = dir == 0 ? U : V;
      d.ld1 = dir == 0 ? B.ldv : B.ldu;
      d.ld2 = dir == 0 ? B.ldu : B.ldv;
      d.n1 = (int32_t)(dir == 0 ? B.n : B.m);
      d.n2 = (int32_t)(dir == 0 ? B.m : B.n);
      d.c1 = (int32_t)(dir == 0 ? B.col_off : B.row_off);
      d.c2 = (int32_t)(dir == 0 ? B.row_off : B.col_off);
      d.k = B.k;
      d.fmt = B.fmt;
      d.e = B.exp_u + B.exp_v;
      d.toff = toff[b];
    }
    h->d_blk[dir] = upload(bd);
    std::vector<DenseDesc> dd(H.dense.size());
    for (size_t q = 0; q < H.dense.size(); ++q) {
      const hh::DenseBlock& D = H.dense[q];
      dd[q].d = h->d_dense + D.d_off;
      dd[q].ld = D.m;
      dd[q].m = (int32_t)D.m;
      dd[q].n = (int32_t)D.n;
      dd[q].r0 = (int32_t)(dir == 0 ? D.row_off : D.row_off);
      dd[q].c0 = (int32_t)(dir == 0 ? D.col_off : D.col_off);
    }
    h->d_dns[dir] = upload(dd);
    std::vector<Item> p1, p2;
    make_items(H, dir, p1, p2);
    h->d_items[dir][0] = upload(p1);
    h->d_items[dir][1] = upload(p2);
    h->n_items[dir][0] = (int)p1.size();
    h->n_items[dir][1] = (int)p2.size();
  }
  ck(cudaMalloc(&h->d_status, 256), "cudaMalloc");
  ck(cudaMemset(h->d_status, 0, 256), "cudaMemset");
  unsigned present = 0;
  for (const hh::LRBlock& B : H.lr) present |= 1u << B.fmt;
  h->fset = hh::dev::pass_set_for(present);
  for (int phase = 1; phase <= 2; ++phase)
    for (int nr : {1, 2, 4}) h->grid[phase][nr] = h->sms * hh::dev::pass_blocks_per_sm(phase, h->fset, nr);
  size_t ws = 0;
  hh_workspace_bytes(h, &ws);
  ck(cudaMalloc(&h->d_ws, ws), "cudaMalloc workspace");
  h->ws_bytes = ws;
  ck(cudaDeviceSynchronize(), "upload");
}

struct WsView {
  float* xs;
  double* xs64;
  double* acc;
  float* t32;
  double* t64;
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
  double* xs64 = (double*)take(sizeof(double) * 2 * R * h->npad);
  double* acc = (double*)take(sizeof(double) * R * h->npad);
  float* t32 = (float*)take(sizeof(float) * std::max<int64_t>(1, h->t32_elems * R));
  double* t64 = (double*)take(sizeof(double) * std::max<int64_t>(1, h->t64_elems * R));
  if (v) *v = {xs, xs64, acc, t32, t64};
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
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.blk = h->d_blk[dir];
    a.dns = h->d_dns[dir];
    a.nr = nr;
    a.npad = h->npad;
    a.xs = w.xs;
    a.xs64 = w.xs64;
    a.t32 = w.t32;
    a.t64 = w.t64;
    a.acc = w.acc;
    a.status = h->d_status;
    if (ev) cudaEventRecord(ev[0], st);
    cudaError_t e = hh::dev::launch_prep(in + (int64_t)rb * ld_in, ld_in, nr, h->d_perm, h->H.n, h->npad,
                                         w.xs, w.xs64, w.acc, st);
    for (int phase = 1; phase <= 2 && e == cudaSuccess; ++phase) {
      if (ev) cudaEventRecord(ev[phase], st);
      a.items = h->d_items[dir][phase - 1];
      a.n_items = h->n_items[dir][phase - 1];
      int grid = std::min(h->grid[phase][nr], (a.n_items + 7) / 8);
      if (grid < 1) grid = 1;
      e = hh::dev::launch_pass(phase, h->fset, a, grid, st);
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
  const size_t need = align256(sizeof(float) * 4 * npad) + align256(sizeof(double) * 2 * npad) +
                      align256(sizeof(double) * npad) +
                      align256(sizeof(float) * std::max<int64_t>(1, t32 * hh::dev::kMaxNR)) +
                      align256(sizeof(double) * std::max<int64_t>(1, t64 * hh::dev::kMaxNR));
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
    double* xs64 = (double*)p;
    p += align256(sizeof(double) * 2 * npad);
    double* acc = (double*)p;
    p += align256(sizeof(double) * npad);
    float* tt32 = (float*)p;
    p += align256(sizeof(float) * std::max<int64_t>(1, t32 * hh::dev::kMaxNR));
    double* tt64 = (double*)p;
    const int dir = transpose ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.blk = h->d_blk[dir];
    a.dns = h->d_dns[dir];
    a.nr = 1;
    a.npad = npad;
    a.xs = xs;
    a.xs64 = xs64;
    a.t32 = tt32;
    a.t64 = tt64;
    a.acc = acc;  // cleared by the prep launch on every call
    a.status = h->d_status;
    cudaError_t e = hh::dev::launch_prep(in, h->H.n, 1, h->d_perm, h->H.n, npad, xs, xs64, acc, st);
    for (int phase = 1; phase <= 2 && e == cudaSuccess; ++phase) {
      a.items = h->d_items[dir][phase - 1];
      a.n_items = h->n_items[dir][phase - 1];
      int grid = std::max(1, std::min(h->grid[phase][1], (a.n_items + 7) / 8));
      e = hh::dev::launch_pass(phase, h->fset, a, grid, st);
    }
    if (e == cudaSuccess) e = hh::dev::launch_finish(acc, 1, h->d_perm, h->H.n, npad, out, h->H.n, st);
    if (e != cudaSuccess) rc = fail(HH_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  }
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  return rc;
}
