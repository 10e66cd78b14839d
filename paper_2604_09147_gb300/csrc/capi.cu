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

// Descriptors and work items of the two streaming passes (stream.cu) for one
// direction, with the kernel variant and grid sizes that fit them.
struct StreamSet {
  hh::dev::StreamDesc* d_desc[2] = {nullptr, nullptr};  // [phase]
  Item* d_items[2] = {nullptr, nullptr};
  int n_items[2] = {0, 0};
  unsigned fset = hh::dev::kSetAll;
  unsigned present = 0;  // formats of the low-rank blocks in the set (bit f)
  int grid[3][5] = {};   // [phase][nr]
  int depth[3] = {4, 4, 4};  // [phase] pipeline depth of one-column launches (hh_autotune's choice)
  // host copies (batches concatenate them)
  std::vector<hh::dev::StreamDesc> h_desc[2];
  std::vector<Item> h_items[2];
  std::vector<double> h_cost[2];
};

// Work tables of the tensor-core path (tc.cu) for one direction, and the
// factor panels packed for it (allocated and packed on the first
// tensor-core product in that direction).
struct TcSet {
  hh::dev::TcPiece* d_pieces = nullptr;
  hh::dev::TcGroup* d_groups = nullptr;
  hh::dev::TcTile* d_tiles = nullptr;
  hh::dev::TcEntry* d_entries = nullptr;
  int n_pieces = 0, n_groups = 0, n_tiles = 0, n_entries = 0;
  int64_t t_bytes = 0;                  // T images of all pieces
  int64_t part_floats = 0;              // partial sums of the split groups
  int n_cnt = 0;                        // arrival counters (four per split group)
  int64_t n_blocks = 0, factor_bytes = 0;
  int64_t img_bytes = 0;                // packed panels: groups, then entries
  uint8_t* d_img = nullptr;
};

// Work tables of the CUDA-core products for many right-hand sides (mr.cu)
// for one direction.
struct MrSet {
  hh::dev::TcPiece* d_pieces = nullptr;
  hh::dev::TcGroup* d_groups = nullptr;
  hh::dev::TcTile* d_tiles = nullptr;
  hh::dev::TcEntry* d_entries = nullptr;
  int n_pieces = 0, n_groups = 0, n_tiles = 0;
  int64_t t_floats = 0;
  // dense blocks on the tensor cores (dense_tc.cu): 128-row tiles, their
  // entries, and the digit panels and row exponents (allocated and packed
  // on the first many-column product in this direction)
  hh::dev::TcTile* d_dtiles = nullptr;
  hh::dev::TdEntry* d_dentries = nullptr;
  int n_dtiles = 0, n_dentries = 0;
  int64_t dimg_bytes = 0;
  int64_t dx_bytes = 0;        // the input's digit panels of every entry (two passes)
  int64_t dense_tc_elems = 0;  // 128 x 16 per k-step of every entry
  uint8_t* d_dimg = nullptr;
  int32_t* d_drexp = nullptr;
};

struct hh_matrix {
  hh::HostMatrix H;
  hh::Summary S;
  int device = -1;
  int sms = 0;
  int64_t npad = 0;
  int64_t t32_elems = 0, t64_elems = 0;  // per right-hand side
  uint8_t* d_arena = nullptr;
  int32_t* d_perm = nullptr;
  int32_t* d_iperm = nullptr;  // caller position -> tree position
  int* d_status = nullptr;
  void* d_ws = nullptr;
  size_t ws_bytes = 0;
  double* d_stage = nullptr;  // hh_matvec_host staging buffers (2 x n x stage_cols)
  int stage_cols = 0;
  double* d_dense_pad = nullptr;  // dense blocks, column-major, ld rounded up to even
  StreamSet ss[2];     // [direction]: every block on the streaming passes
  StreamSet ss_rest[2];  // [direction]: the blocks the tensor-core path leaves to them
  TcSet tc[2];         // [direction]
  MrSet mr[2];         // [direction]
  void* d_tc_ws = nullptr;  // tensor-core workspace, allocated on first use
  size_t tc_ws_bytes = 0;
  std::vector<int64_t> doff;   // dense block offsets in d_dense_pad
  std::vector<int32_t> dexp;   // and their scale exponents
  int split_len = hh::dev::kTcSplitPositions;  // positions of a many-column phase-1 item
  int64_t item_bytes = int64_t(64) << 10;      // factor bytes of a streaming phase-1 item (hh_autotune)
  int blocks_per_sm[2][3] = {};                // streaming grid per [direction][phase] (0: occupancy)
  int tuned = 0;
};

namespace {

// the many-column tables of one direction (and the packed panels)
void free_many(hh_matrix* h, int d) {
  TcSet& ts = h->tc[d];
  cudaFree(ts.d_pieces);
  cudaFree(ts.d_groups);
  cudaFree(ts.d_tiles);
  cudaFree(ts.d_entries);
  cudaFree(ts.d_img);
  MrSet& ms = h->mr[d];
  cudaFree(ms.d_pieces);
  cudaFree(ms.d_groups);
  cudaFree(ms.d_tiles);
  cudaFree(ms.d_entries);
  cudaFree(ms.d_dtiles);
  cudaFree(ms.d_dentries);
  cudaFree(ms.d_dimg);
  cudaFree(ms.d_drexp);
  ts = TcSet();
  ms = MrSet();
}

void free_device(hh_matrix* h) {
  if (h->device < 0) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  cudaFree(h->d_arena);
  cudaFree(h->d_perm);
  cudaFree(h->d_iperm);
  for (int d = 0; d < 2; ++d) {
    for (int p = 0; p < 2; ++p) {
      cudaFree(h->ss[d].d_desc[p]);
      cudaFree(h->ss[d].d_items[p]);
      cudaFree(h->ss_rest[d].d_desc[p]);
      cudaFree(h->ss_rest[d].d_items[p]);
    }
    free_many(h, d);
  }
  cudaFree(h->d_tc_ws);
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

// Dense blocks with an even leading dimension (16-byte aligned columns), each
// scaled by a power of two so that its largest magnitude lies in (1/2, 1]
// (exact; upload_matrix then turns every value into a pair of fp32 halves).
void upload_dense(hh_matrix* h, std::vector<int64_t>& doff, std::vector<int32_t>& dexp) {
  const hh::HostMatrix& H = h->H;
  doff.assign(H.dense.size(), 0);
  dexp.assign(H.dense.size(), 0);
  int64_t dtot = 0;
  for (size_t q = 0; q < H.dense.size(); ++q) {
    doff[q] = dtot;
    dtot += ((H.dense[q].m + 1) / 2 * 2) * H.dense[q].n;
  }
  std::vector<double> dpad(static_cast<size_t>(dtot), 0.0);
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
}

// Descriptors and work items of the streaming passes (stream.cu) for one
// direction: every dense block and the low-rank blocks `take` selects.
void build_stream_set(hh_matrix* h, int dir, const std::vector<int64_t>& toff, const std::vector<int64_t>& doff,
                      const std::vector<int32_t>& dexp, const std::vector<char>& take, bool with_dense,
                      StreamSet& out) {
  using hh::dev::StreamDesc;
  const hh::HostMatrix& H = h->H;
  const int cols1 = hh::dev::stream_cols_per_item();
  std::vector<StreamDesc> desc[2];
  struct Costed {
    Item it;
    double cost;
  };
  std::vector<Costed> items[2];
  // phase-1 items: whole groups of cols1 columns, as many groups (at most 8)
  // as make about h->item_bytes of factor bytes (64 KB unless hh_autotune
  // chose otherwise), so that short columns do not pay the per-item
  // scheduling latency every stage
  auto add_cols = [&](int phase, int di, int64_t rows, int64_t cols, int sz) {
    const int64_t group_bytes = std::max<int64_t>(1, int64_t(cols1) * rows * sz);
    const int64_t groups = std::max<int64_t>(1, std::min<int64_t>(8, (h->item_bytes + group_bytes - 1) / group_bytes));
    const int64_t per = cols1 * groups;
    for (int64_t j = 0; j < cols; j += per) {
      int64_t hi = std::min<int64_t>(cols, j + per);
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
  unsigned present = 0;
  for (size_t b = 0; b < H.lr.size(); ++b) {
    const hh::LRBlock& B = H.lr[b];
    if (B.k == 0 || !take[b]) continue;
    present |= 1u << B.fmt;
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
  for (size_t q = 0; q < H.dense.size() && with_dense; ++q) {
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
    std::vector<double> cost;
    for (auto& c : items[p]) {
      flat.push_back(c.it);
      cost.push_back(c.cost);
    }
    out.d_desc[p] = upload(desc[p]);
    out.d_items[p] = upload(flat);
    out.n_items[p] = (int)flat.size();
    out.h_desc[p] = desc[p];
    out.h_items[p] = flat;
    out.h_cost[p] = cost;
  }
  out.present = present;
  out.fset = hh::dev::pass_set_for(present);
  for (int phase = 1; phase <= 2; ++phase)
    for (int nr : {1, 2, 4})
      out.grid[phase][nr] = h->sms * hh::dev::stream_blocks_per_sm(phase, out.fset, nr, nr == 1 ? out.depth[phase] : 4);
}

// Formats the tensor-core path takes and the most ranks of one piece.
bool tc_format(int fmt) { return fmt == hh::F32 || fmt == hh::F16 || fmt == hh::BF16 || fmt == hh::E4M3; }
int tc_piece_cap(int) { return hh::dev::kTcGroupRanks; }
int64_t align128(int64_t v) { return (v + 127) / 128 * 128; }

// A block goes to the tensor cores when its format is one they take and both
// of its clusters start at a tree position that is a multiple of 16 (the
// operand images are built in 16-position blocks).
bool tc_eligible(const hh::LRBlock& B) {
  return B.k > 0 && tc_format(B.fmt) && B.row_off % 16 == 0 && B.col_off % 16 == 0;
}

// Work tables of the tensor-core path for one direction: pieces of at most
// kTcGroupRanks ranks, grouped by (input cluster, format) into phase-1 groups
// of at most kTcGroupRanks ranks and split into items of at most split_len
// positions, and the kTcRows-row output tiles of phase 2 with the piece rows
// that fall in them; the byte offsets of every group's and entry's packed
// panel (16-position blocks x factor slices x nk rows x 32 B; 16-rank steps x
// factor slices x 4 KB).
void build_tc_set(hh_matrix* h, int dir, TcSet& out) {
  using namespace hh::dev;
  const hh::HostMatrix& H = h->H;
  const int split_len = h->split_len;
  struct Key {
    int64_t in_off, rows;
    int fmt;
    bool operator<(const Key& o) const {
      if (in_off != o.in_off) return in_off < o.in_off;
      if (rows != o.rows) return rows < o.rows;
      return fmt < o.fmt;
    }
  };
  std::vector<std::pair<Key, TcPiece>> raw;
  for (const hh::LRBlock& B : H.lr) {
    if (!tc_eligible(B)) continue;
    const int sz = hh::fmt_bytes(B.fmt);
    const uint8_t* U = h->d_arena + B.u_off;
    const uint8_t* V = h->d_arena + B.v_off;
    const uint8_t* f1 = dir == 0 ? V : U;
    const uint8_t* f2 = dir == 0 ? U : V;
    const int64_t ld1 = dir == 0 ? B.ldv : B.ldu, ld2 = dir == 0 ? B.ldu : B.ldv;
    out.n_blocks += 1;
    out.factor_bytes += (B.m + B.n) * int64_t(B.k) * sz;
    for (int r0 = 0; r0 < B.k; r0 += tc_piece_cap(B.fmt)) {
      TcPiece q;
      std::memset(&q, 0, sizeof(q));
      q.k = std::min(tc_piece_cap(B.fmt), B.k - r0);
      q.kp = (q.k + 15) / 16 * 16;
      q.f1 = f1 + int64_t(r0) * ld1 * sz;
      q.f2 = f2 + int64_t(r0) * ld2 * sz;
      q.ld1 = ld1;
      q.ld2 = ld2;
      q.rows1 = (int32_t)(dir == 0 ? B.n : B.m);
      q.rows2 = (int32_t)(dir == 0 ? B.m : B.n);
      q.in_off = (int32_t)(dir == 0 ? B.col_off : B.row_off);
      q.out_off = (int32_t)(dir == 0 ? B.row_off : B.col_off);
      q.fmt = B.fmt;
      q.e = B.exp_u + B.exp_v;
      raw.push_back({Key{q.in_off, q.rows1, q.fmt}, q});
    }
  }
  std::stable_sort(raw.begin(), raw.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  std::vector<TcPiece> pieces;
  struct CGroup {
    TcGroup g;
    double cost;
  };
  std::vector<CGroup> groups;
  int64_t toff = 0;
  for (size_t i = 0; i < raw.size();) {
    size_t j = i;
    while (j < raw.size() && !(raw[i].first < raw[j].first) && !(raw[j].first < raw[i].first)) ++j;
    // pieces [i, j) share the input cluster and the format: pack into groups;
    // their items are listed split-major (every group's first position
    // range, then every group's second, ...), so that items taken at the
    // same time read the same input blocks, which then stay in L2 (the cost
    // sort below keeps this order among items of equal cost)
    std::vector<TcGroup> gl;
    for (size_t t = i; t < j;) {
      TcGroup g;
      std::memset(&g, 0, sizeof(g));
      g.first = (int32_t)pieces.size();
      g.fmt = raw[t].second.fmt;
      g.in_off = raw[t].second.in_off;
      g.rows = raw[t].second.rows1;
      const int cap = tc_piece_cap(g.fmt);
      while (t < j && g.nk + raw[t].second.kp <= cap) {
        TcPiece q = raw[t].second;
        q.col = g.nk;
        q.toff = toff;
        toff += int64_t(hh::dev::tc_input_slices(q.fmt)) * (q.kp / 16) * 4096;
        g.nk += q.kp;
        g.count += 1;
        pieces.push_back(q);
        ++t;
      }
      const int nsplit = (g.rows + split_len - 1) / split_len;
      g.nsplit = nsplit;
      if (nsplit > 1) {
        g.gid = out.n_cnt / 4;
        out.n_cnt += 4;
        g.poff = out.part_floats;  // nsplit consecutive [128][nk] partial sums
        out.part_floats += int64_t(nsplit) * 128 * g.nk;
      }
      g.img = out.img_bytes;
      out.img_bytes += align128(int64_t((g.rows + 15) / 16) * hh::dev::tc_factor_slices(g.fmt) * g.nk * 32);
      gl.push_back(g);
    }
    const int nsplit = gl.empty() ? 0 : gl.front().nsplit;  // the groups of a key share the cluster
    for (int sp = 0; sp < nsplit; ++sp)
      for (const TcGroup& g : gl) {
        TcGroup gs = g;
        gs.split = sp;
        gs.p0 = sp * split_len;
        gs.p1 = std::min(g.rows, (sp + 1) * split_len);
        if (nsplit > 1) {
          // a group's split items are consecutive in the partial-sum arena
          gs.poff = g.poff + int64_t(sp) * 128 * g.nk;
        }
        groups.push_back({gs, double((gs.p1 - gs.p0 + 15) / 16) *
                                   double(hh::dev::tc_factor_slices(g.fmt) * g.nk * 32 + hh::dev::tc_input_slices(g.fmt) * 4096)});
      }
    i = j;
  }
  std::stable_sort(groups.begin(), groups.end(), [](const CGroup& x, const CGroup& y) { return x.cost > y.cost; });
  // phase-2 tiles over every piece
  const int64_t ntiles = (H.n + kTcRows - 1) / kTcRows;
  std::vector<std::vector<TcEntry>> per_tile(static_cast<size_t>(ntiles));
  for (size_t pi = 0; pi < pieces.size(); ++pi) {
    const TcPiece& q = pieces[pi];
    const int64_t lo = q.out_off, hi = int64_t(q.out_off) + q.rows2;
    for (int64_t t = lo / kTcRows; t * kTcRows < hi; ++t) {
      const int64_t r0 = t * kTcRows, a = std::max(lo, r0), b = std::min(hi, r0 + kTcRows);
      per_tile[t].push_back(
          TcEntry{(int32_t)pi, (int32_t)(a - lo), (int32_t)(a - r0), (int32_t)(b - a), 0, q.toff, q.kp / 16, q.fmt});
    }
  }
  struct CTile {
    TcTile t;
    double cost;
  };
  std::vector<CTile> tiles;
  std::vector<TcEntry> entries;
  for (int64_t t = 0; t < ntiles; ++t) {
    if (per_tile[t].empty()) continue;
    TcTile tl{};
    tl.row0 = (int32_t)(t * kTcRows);
    tl.rows = (int32_t)std::min<int64_t>(kTcRows, H.n - t * kTcRows);
    tl.first = (int32_t)entries.size();
    tl.count = (int32_t)per_tile[t].size();
    tl.nst = 0;
    tl.chunk = kTcChunk16;
    double cost = 0;
    for (TcEntry e : per_tile[t]) {
      const TcPiece& q = pieces[e.piece];
      const int64_t step = int64_t(hh::dev::tc_factor_slices(q.fmt)) * 4096;
      e.img = out.img_bytes;
      out.img_bytes += (q.kp / 16) * step;
      entries.push_back(e);
      tl.nst += (q.kp / 16 + kTcKSteps - 1) / kTcKSteps;
      tl.chunk = std::min(tl.chunk, q.fmt == hh::F32 ? kTcChunkF32 : kTcChunk16);
      cost += double(q.kp / 16) * double(step + hh::dev::tc_input_slices(q.fmt) * 4096);
    }
    tiles.push_back({tl, cost});
  }
  std::stable_sort(tiles.begin(), tiles.end(), [](const CTile& x, const CTile& y) { return x.cost > y.cost; });
  std::vector<TcGroup> gflat;
  for (auto& g : groups) gflat.push_back(g.g);
  std::vector<TcTile> tflat;
  for (auto& t : tiles) tflat.push_back(t.t);
  out.d_pieces = upload(pieces);
  out.n_pieces = (int)pieces.size();
  out.d_groups = upload(gflat);
  out.d_tiles = upload(tflat);
  out.d_entries = upload(entries);
  out.n_groups = (int)gflat.size();
  out.n_tiles = (int)tflat.size();
  out.n_entries = (int)entries.size();
  out.t_bytes = toff;
}

// Output tiles of `rows` rows over the output ranges [out_off, out_off +
// rows2) of the given pieces, each tile with the piece rows that fall in it,
// sorted by cost (sum of cost_of(piece) * rows in the tile) descending.
template <class CostFn>
void build_tiles(int64_t n, int rows, const std::vector<hh::dev::TcPiece>& pieces, CostFn cost_of,
                 std::vector<hh::dev::TcTile>& tiles_out, std::vector<hh::dev::TcEntry>& entries) {
  using namespace hh::dev;
  const int64_t ntiles = (n + rows - 1) / rows;
  std::vector<std::vector<TcEntry>> per_tile(static_cast<size_t>(ntiles));
  for (size_t pi = 0; pi < pieces.size(); ++pi) {
    const TcPiece& q = pieces[pi];
    const int64_t lo = q.out_off, hi = int64_t(q.out_off) + q.rows2;
    for (int64_t t = lo / rows; t * rows < hi; ++t) {
      const int64_t r0 = t * rows, a = std::max(lo, r0), b = std::min(hi, r0 + rows);
      per_tile[t].push_back(TcEntry{(int32_t)pi, (int32_t)(a - lo), (int32_t)(a - r0), (int32_t)(b - a)});
    }
  }
  std::vector<std::pair<TcTile, double>> tiles;
  for (int64_t t = 0; t < ntiles; ++t) {
    if (per_tile[t].empty()) continue;
    TcTile tl{};
    tl.row0 = (int32_t)(t * rows);
    tl.rows = (int32_t)std::min<int64_t>(rows, n - t * rows);
    tl.first = (int32_t)entries.size();
    tl.count = (int32_t)per_tile[t].size();
    double cost = 0;
    for (const TcEntry& e : per_tile[t]) {
      entries.push_back(e);
      cost += cost_of(pieces[e.piece]) * rows;
    }
    tiles.push_back({tl, cost});
  }
  std::stable_sort(tiles.begin(), tiles.end(), [](const auto& x, const auto& y) { return x.second > y.second; });
  for (auto& t : tiles) tiles_out.push_back(t.first);
}

// Work tables of the CUDA-core products for many right-hand sides for one
// direction: the low-rank blocks in fp32, fp16, bf16 or e4m3 that the tensor
// cores do not take, in pieces of at most kMrRanks ranks grouped by input
// cluster and format and split into ranges of at most kTcSplitPositions
// positions; the 128-row tiles of their phase 2; and the dense blocks in
// 64-row tiles.
void build_mr_set(hh_matrix* h, int dir, const std::vector<int64_t>& doff, const std::vector<int32_t>& dexp,
                  MrSet& out) {
  using namespace hh::dev;
  const hh::HostMatrix& H = h->H;
  struct Key {
    int64_t in_off, rows;
    int fmt;
    bool operator<(const Key& o) const {
      if (in_off != o.in_off) return in_off < o.in_off;
      if (rows != o.rows) return rows < o.rows;
      return fmt < o.fmt;
    }
  };
  std::vector<std::pair<Key, TcPiece>> raw;
  for (const hh::LRBlock& B : H.lr) {
    if (B.k == 0 || B.fmt == hh::F64 || tc_eligible(B)) continue;
    const int sz = hh::fmt_bytes(B.fmt);
    const uint8_t* U = h->d_arena + B.u_off;
    const uint8_t* V = h->d_arena + B.v_off;
    const uint8_t* f1 = dir == 0 ? V : U;
    const uint8_t* f2 = dir == 0 ? U : V;
    const int64_t ld1 = dir == 0 ? B.ldv : B.ldu, ld2 = dir == 0 ? B.ldu : B.ldv;
    for (int r0 = 0; r0 < B.k; r0 += kMrRanks) {
      TcPiece q;
      std::memset(&q, 0, sizeof(q));
      q.k = std::min(kMrRanks, B.k - r0);
      q.kp = (q.k + 3) / 4 * 4;
      q.f1 = f1 + int64_t(r0) * ld1 * sz;
      q.f2 = f2 + int64_t(r0) * ld2 * sz;
      q.ld1 = ld1;
      q.ld2 = ld2;
      q.rows1 = (int32_t)(dir == 0 ? B.n : B.m);
      q.rows2 = (int32_t)(dir == 0 ? B.m : B.n);
      q.in_off = (int32_t)(dir == 0 ? B.col_off : B.row_off);
      q.out_off = (int32_t)(dir == 0 ? B.row_off : B.col_off);
      q.fmt = B.fmt;
      q.e = B.exp_u + B.exp_v;
      raw.push_back({Key{q.in_off, q.rows1, q.fmt}, q});
    }
  }
  std::stable_sort(raw.begin(), raw.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  std::vector<TcPiece> pieces;
  std::vector<std::pair<TcGroup, double>> groups;
  for (size_t i = 0; i < raw.size();) {
    size_t j = i;
    while (j < raw.size() && !(raw[i].first < raw[j].first) && !(raw[j].first < raw[i].first)) ++j;
    for (size_t t = i; t < j;) {
      TcGroup g;
      std::memset(&g, 0, sizeof(g));
      g.first = (int32_t)pieces.size();
      g.fmt = raw[t].second.fmt;
      g.in_off = raw[t].second.in_off;
      g.rows = raw[t].second.rows1;
      while (t < j && g.nk + raw[t].second.kp <= kMrRanks) {
        TcPiece q = raw[t].second;
        q.col = g.nk;
        q.toff = out.t_floats;
        out.t_floats += int64_t(q.kp) * 128;
        g.nk += q.kp;
        g.count += 1;
        pieces.push_back(q);
        ++t;
      }
      g.nsplit = (g.rows + h->split_len - 1) / h->split_len;
      for (int sp = 0; sp < g.nsplit; ++sp) {
        TcGroup gs = g;
        gs.split = sp;
        gs.p0 = sp * h->split_len;
        gs.p1 = std::min(g.rows, (sp + 1) * h->split_len);
        groups.push_back({gs, double(gs.p1 - gs.p0) * g.nk * hh::fmt_bytes(g.fmt)});
      }
    }
    i = j;
  }
  std::stable_sort(groups.begin(), groups.end(), [](const auto& x, const auto& y) { return x.second > y.second; });
  std::vector<TcGroup> gflat;
  for (auto& g : groups) gflat.push_back(g.first);
  std::vector<TcTile> tiles;
  std::vector<TcEntry> entries;
  build_tiles(H.n, kMrRows, pieces, [](const TcPiece& q) { return double(q.kp) * hh::fmt_bytes(q.fmt); }, tiles,
              entries);
  out.d_pieces = upload(pieces);
  out.d_groups = upload(gflat);
  out.d_tiles = upload(tiles);
  out.d_entries = upload(entries);
  out.n_pieces = (int)pieces.size();
  out.n_groups = (int)gflat.size();
  out.n_tiles = (int)tiles.size();
  // dense blocks: 128-row tiles of the output, each block's share of a tile
  // cut into entries of at most kTdMaxK contracted positions
  std::vector<TcPiece> dp;
  for (size_t q = 0; q < H.dense.size(); ++q) {
    const hh::DenseBlock& D = H.dense[q];
    TcPiece p;
    std::memset(&p, 0, sizeof(p));
    p.f2 = reinterpret_cast<const uint8_t*>(h->d_dense_pad + doff[q]);
    p.ld2 = (D.m + 1) / 2 * 2;
    p.k = (int32_t)(dir == 0 ? D.n : D.m);
    p.kp = p.k;
    p.rows2 = (int32_t)(dir == 0 ? D.m : D.n);
    p.in_off = (int32_t)(dir == 0 ? D.col_off : D.row_off);
    p.out_off = (int32_t)(dir == 0 ? D.row_off : D.col_off);
    p.fmt = hh::F64;
    p.e = dexp[q];
    p.pad = dir;
    dp.push_back(p);
  }
  std::vector<TcTile> dt;
  std::vector<TcEntry> de;
  build_tiles(H.n, kTcRows, dp, [](const TcPiece& q) { return double(q.k) * 8; }, dt, de);
  std::vector<TdEntry> te;
  for (TcTile& t : dt) {
    const int first = (int)te.size();
    for (int i = 0; i < t.count; ++i) {
      const TcEntry& e = de[size_t(t.first + i)];
      const TcPiece& p = dp[size_t(e.piece)];
      for (int k0 = 0; k0 < p.k; k0 += kTdMaxK) {
        TdEntry x;
        std::memset(&x, 0, sizeof(x));
        x.d = reinterpret_cast<const float2*>(p.f2);
        x.ld = p.ld2;
        x.img = out.dimg_bytes;
        x.src = e.src;
        x.dst = e.dst;
        x.nrows = e.nrows;
        x.k0 = k0;
        x.kc = std::min(kTdMaxK, p.k - k0);
        x.in_off = p.in_off + k0;
        x.e = p.e;
        x.trans = p.pad;
        // the first entry of the tile over these rows stores, later ones add
        x.first = 1;
        for (int q = first; q < (int)te.size(); ++q)
          if (te[size_t(q)].dst < x.dst + x.nrows && x.dst < te[size_t(q)].dst + te[size_t(q)].nrows) x.first = 0;
        x.xoff = out.dx_bytes;
        out.dimg_bytes += int64_t((x.kc + 15) / 16) * kTdStepBytes;
        out.dx_bytes += int64_t((x.kc + 15) / 16) * 2 * kTdXStepBytes;
        out.dense_tc_elems += int64_t((x.kc + 15) / 16) * 128 * 16;
        te.push_back(x);
      }
    }
    t.first = first;
    t.count = (int)te.size() - first;
  }
  out.d_dtiles = upload(dt);
  out.d_dentries = upload(te);
  out.n_dtiles = (int)dt.size();
  out.n_dentries = (int)te.size();
}

// ---------------------------------------------------------------------------
// Allocation-free product (hh_matvec_noalloc, see include/hh.h).
//
// Some callers cannot allocate device memory at call time: a host framework
// that owns every device allocation (a serving runtime with a fixed memory
// budget, a plugin host), or a latency-critical loop in which cudaMalloc's
// implicit device synchronisation is not acceptable.  For them the product's
// scratch (shifted input copies, output accumulator, t arenas for one
// right-hand side) lives in one fixed file-scope device array.  A GPU holds
// it from the first matrix built or loaded on it (upload_matrix resolves its
// address, which loads this file's device module) until the process exits,
// so that no hh_matvec_noalloc call loads a module or reserves memory.

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

// streaming grid of one direction and phase (defined below)
void set_stream_grid(hh_matrix* h, int dir, int phase, int c, int depth = 4);

void upload_matrix(hh_matrix* h, int device) {
  const hh::HostMatrix& H = h->H;
  ck(cudaSetDevice(device), "cudaSetDevice");
  h->device = device;
  ck(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device), "device attribute");
  {
    // the allocation-free product's scratch array: resolved here, once per
    // device, so that hh_matvec_noalloc never loads a module (a failure is
    // reported by that call instead)
    void* scratch = nullptr;
    if (noalloc_scratch(device, &scratch) != HH_OK) g_last_error.clear();
  }
  h->d_arena = upload(H.arena);
  h->d_perm = upload(H.perm);
  {
    std::vector<int32_t> iperm(H.perm.size());
    for (size_t p = 0; p < H.perm.size(); ++p) iperm[static_cast<size_t>(H.perm[p])] = static_cast<int32_t>(p);
    h->d_iperm = upload(iperm);
  }
  h->npad = (H.n + 32 + 3) / 4 * 4;
  // t offsets per block (room for kMaxNR right-hand sides)
  std::vector<int64_t> toff(H.lr.size(), 0);
  h->t32_elems = h->t64_elems = 0;
  for (size_t b = 0; b < H.lr.size(); ++b) {
    int64_t& tot = H.lr[b].fmt == hh::F64 ? h->t64_elems : h->t32_elems;
    toff[b] = tot * hh::dev::kMaxNR;
    tot += H.lr[b].k;
  }
  std::vector<int64_t>& doff = h->doff;
  std::vector<int32_t>& dexp = h->dexp;
  upload_dense(h, doff, dexp);
  // the device form of fp64 data: every fp64 factor and dense block becomes
  // float2 pairs (hi, lo) in place, once (the host arena keeps fp64)
  {
    std::vector<int64_t> spans;
    for (const hh::LRBlock& B : H.lr)
      if (B.fmt == hh::F64 && B.k > 0) {
        spans.insert(spans.end(), {B.u_off, B.ldu * B.k});
        spans.insert(spans.end(), {B.v_off, B.ldv * B.k});
      }
    int64_t* d_spans = upload(spans);
    cudaError_t e = hh::dev::launch_presplit_f64(h->d_arena, d_spans, (int)(spans.size() / 2), 0);
    const int64_t dtot = H.dense.empty() ? 0 : doff.back() + (H.dense.back().m + 1) / 2 * 2 * H.dense.back().n;
    std::vector<int64_t> dspan = {0, dtot};
    int64_t* d_dspan = upload(dspan);
    if (e == cudaSuccess)
      e = hh::dev::launch_presplit_f64(reinterpret_cast<uint8_t*>(h->d_dense_pad), d_dspan, dtot > 0 ? 1 : 0, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_spans);
    cudaFree(d_dspan);
    ck(e, "fp64 device form");
  }
  // with many right-hand sides the streaming passes keep only the fp64
  // low-rank blocks; the tensor cores and mr.cu take the rest
  // positions of one many-column phase-1 item (HH_TC_SPLIT_POSITIONS, a
  // positive multiple of 16, overrides; hh_autotune may change it)
  if (const char* e = std::getenv("HH_TC_SPLIT_POSITIONS")) {
    const int v = std::atoi(e);
    if (v >= 16 && v % 16 == 0) h->split_len = v;
  }
  // the streaming launch shape hh_autotune would choose, fixed from the
  // environment (for profiling runs): HH_STREAM_ITEM_BYTES (phase-1 item
  // size), HH_STREAM_DEPTH (3, 4 or 6 stages) and HH_STREAM_CTAS (per SM)
  if (const char* e = std::getenv("HH_STREAM_ITEM_BYTES")) {
    const long long v = std::atoll(e);
    if (v >= 1024) h->item_bytes = v;
  }
  std::vector<char> all(H.lr.size(), 1), rest(H.lr.size(), 0);
  for (size_t b = 0; b < H.lr.size(); ++b) rest[b] = H.lr[b].fmt == hh::F64;
  for (int dir = 0; dir < 2; ++dir) {
    build_stream_set(h, dir, toff, doff, dexp, all, true, h->ss[dir]);
    build_stream_set(h, dir, toff, doff, dexp, rest, false, h->ss_rest[dir]);
    build_tc_set(h, dir, h->tc[dir]);
    build_mr_set(h, dir, doff, dexp, h->mr[dir]);
  }
  {
    const char* ed = std::getenv("HH_STREAM_DEPTH");
    const char* ec = std::getenv("HH_STREAM_CTAS");
    if (ed || ec) {
      const int depth = ed ? std::atoi(ed) : 4, ctas = ec ? std::atoi(ec) : 16;
      for (int dir = 0; dir < 2; ++dir)
        for (int phase = 1; phase <= 2; ++phase) set_stream_grid(h, dir, phase, std::max(1, ctas), depth);
    }
  }
  ck(cudaMalloc(&h->d_status, 256), "cudaMalloc");
  ck(cudaMemset(h->d_status, 0, 256), "cudaMemset");
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

// Workspace of the streaming passes for up to R right-hand sides per launch
// sequence: shifted input copies and output accumulator for R columns; the t
// arenas always for kMaxNR (the descriptors' t offsets are laid out for it).
size_t ws_layout(const hh_matrix* h, WsView* v, char* base, int R = hh::dev::kMaxNR) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return base ? base + o : nullptr;
  };
  float* xs = (float*)take(sizeof(float) * 4 * R * h->npad);
  float* xs_lo = (float*)take(sizeof(float) * 4 * R * h->npad);
  double* acc = (double*)take(sizeof(double) * R * h->npad);
  float* t32 = (float*)take(sizeof(float) * std::max<int64_t>(1, h->t32_elems * hh::dev::kMaxNR));
  float2* t64 = (float2*)take(sizeof(float2) * std::max<int64_t>(1, h->t64_elems * hh::dev::kMaxNR));
  int* counters = (int*)take(256);
  if (v) *v = {xs, xs_lo, acc, t32, t64, counters};
  return off;
}

// prep -> phase 1 -> phase 2 of the streaming passes over the blocks of `set`
// for nr <= 4 right-hand sides; the products are added into acc [nr][npad]
// (cleared by the prep launch).
cudaError_t run_stream(hh_matrix* h, const StreamSet& set, const double* in, int64_t ld_in, int nr, double* acc,
                       const WsView& w, cudaStream_t st, cudaEvent_t* ev, bool clear_acc = true) {
  if (ev) cudaEventRecord(ev[0], st);
  cudaError_t e = hh::dev::launch_prep(in, ld_in, nr, h->d_perm, h->H.n, h->npad, w.xs, w.xs_lo,
                                       clear_acc ? acc : nullptr, st, w.counters);
  bool p1 = false;  // phase 1 launched: phase 2 may follow it as a programmatic dependent
  for (int phase = 1; phase <= 2 && e == cudaSuccess; ++phase) {
    if (ev) cudaEventRecord(ev[phase], st);
    hh::dev::StreamArgs s;
    std::memset(&s, 0, sizeof(s));
    s.desc = set.d_desc[phase - 1];
    s.items = set.d_items[phase - 1];
    s.n_items = set.n_items[phase - 1];
    s.nr = nr;
    s.npad = h->npad;
    s.xs = w.xs;
    s.xs_lo = w.xs_lo;
    s.t32 = w.t32;
    s.t64 = w.t64;
    s.acc = acc;
    s.status = h->d_status;
    s.counter = w.counters + (phase - 1);
    if (s.n_items == 0) continue;
    int grid = std::max(1, std::min(set.grid[phase][nr], s.n_items));
    e = hh::dev::launch_stream(phase, set.fset, s, grid, st, p1 && !ev, set.depth[phase]);
    p1 = phase == 1;
  }
  return e;
}

// Right-hand-side count from which hh_matvec / hh_matvec_T use the tensor
// cores (HH_TC_MIN_NRHS overrides; 0 disables the path): the many-column
// sequence costs about the same for 5 to 32 columns, the streaming passes
// one pass per 4 columns.
int tc_min_nrhs() {
  static const int v = [] {
    const char* s = std::getenv("HH_TC_MIN_NRHS");
    return s ? std::atoi(s) : 5;
  }();
  return v;
}

struct TcWs {
  uint8_t* ximg;
  uint8_t* timg;
  float* part;
  int* cnt;
  double* acc;
  int64_t nblk;
  float* xh;   // fp32 input images [npad][128] (mr.cu)
  float* xl;
  float* t32;  // T of the CUDA-core pieces
  uint8_t* xdig;  // the input's digit panels of the dense blocks (dense_tc.cu)
  int32_t* bexp;  // and their column exponents
  double* xt;     // the input in tree order [128][npad]
};

size_t tc_ws_layout(const hh_matrix* h, TcWs* v, char* base) {
  const int64_t nblk = (h->npad + 15) / 16 + 4;
  const int64_t tb = std::max(h->tc[0].t_bytes, h->tc[1].t_bytes);  // [direction]
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return base ? base + o : nullptr;
  };
  const int64_t pf = std::max(h->tc[0].part_floats, h->tc[1].part_floats);
  const int nc = std::max(h->tc[0].n_cnt, h->tc[1].n_cnt);
  uint8_t* ximg = (uint8_t*)take(size_t(3) * nblk * 4096);  // [block][three bf16 slices][4 KB]
  uint8_t* timg = (uint8_t*)take(std::max<size_t>(256, size_t(tb)));
  float* part = (float*)take(sizeof(float) * std::max<int64_t>(64, pf));
  int* cnt = (int*)take(sizeof(int) * std::max(64, nc + 2));  // split-group counters, then 2 work counters
  double* acc = (double*)take(sizeof(double) * hh::dev::kTcMaxRhs * h->npad);
  float* xh = (float*)take(sizeof(float) * 128 * h->npad);
  float* xl = (float*)take(sizeof(float) * 128 * h->npad);
  const int64_t tf = std::max(h->mr[0].t_floats, h->mr[1].t_floats);
  float* t32 = (float*)take(sizeof(float) * std::max<int64_t>(64, tf));
  const int64_t dx = std::max(h->mr[0].dx_bytes, h->mr[1].dx_bytes);
  const int64_t de = std::max(h->mr[0].n_dentries, h->mr[1].n_dentries);
  uint8_t* xdig = (uint8_t*)take(std::max<size_t>(256, size_t(dx)));
  int32_t* bexp = (int32_t*)take(sizeof(int32_t) * 128 * std::max<int64_t>(1, de));
  double* xt = (double*)take(sizeof(double) * hh::dev::kTcMaxRhs * h->npad);
  if (v) *v = {ximg, timg, part, cnt, acc, nblk, xh, xl, t32, xdig, bexp, xt};
  return off;
}

// Product for nrhs <= 128 right-hand sides in one pass over the blocks:
// input images, the dense blocks (first: they store into the cleared
// accumulator), the streaming passes over the fp64 low-rank blocks (chunks
// of up to 4 right-hand sides), the CUDA-core and tensor-core phases 1, the
// CUDA-core and tensor-core phases 2, and the output permutation.  With ev
// (9 events) every launch is bracketed: [0] images, [1] dense blocks,
// [2] streaming passes, [3] CUDA-core phase 1, [4] tensor-core phase 1,
// [5] CUDA-core phase 2, [6] tensor-core phase 2, [7] output permutation,
// [8] end.
cudaError_t run_tc(hh_matrix* h, int dir, const double* in, double* out, int nr, int64_t ld_in, int64_t ld_out,
                   const WsView& w, const TcWs& t, cudaStream_t st, cudaEvent_t* ev = nullptr) {
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], st);
  };
  mark(0);
  const TcSet& ts = h->tc[dir];
  const MrSet& ms = h->mr[dir];
  // clears the split-group counters and, after them, the two work counters
  cudaError_t e = hh::dev::launch_tc_prep(in, ld_in, nr, h->d_perm, h->H.n, t.nblk, t.ximg, t.acc, h->npad, t.cnt,
                                          ts.n_cnt + 2, t.xh, t.xl, h->npad, t.t32, ms.t_floats, t.xt, st);
  mark(1);
  {
    hh::dev::TdArgs d;
    std::memset(&d, 0, sizeof(d));
    d.tiles = ms.d_dtiles;
    d.entries = ms.d_dentries;
    d.n_tiles = ms.n_dtiles;
    d.nr = nr;
    d.img = ms.d_dimg;
    d.rexp = ms.d_drexp;
    d.xh = t.xh;
    d.xl = t.xl;
    d.xdig = t.xdig;
    d.bexp = t.bexp;
    d.acc = t.acc;
    d.npad = h->npad;
    d.status = h->d_status;
    if (e == cudaSuccess) e = hh::dev::launch_td_prep(d, ms.n_dentries, st);
    if (e == cudaSuccess) e = hh::dev::launch_td(d, h->sms, st);
  }
  const StreamSet& rest = h->ss_rest[dir];
  mark(2);
  if (rest.n_items[0] + rest.n_items[1] > 0)
    for (int rb = 0; rb < nr && e == cudaSuccess;) {
      const int rem = nr - rb, c = rem >= 4 ? 4 : (rem >= 2 ? 2 : 1);
      // the accumulator already holds the dense blocks' results
      e = run_stream(h, rest, in + int64_t(rb) * ld_in, ld_in, c, t.acc + int64_t(rb) * h->npad, w, st, nullptr,
                     false);
      rb += c;
    }
  hh::dev::TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.pieces = ts.d_pieces;
  a.groups = ts.d_groups;
  a.tiles = ts.d_tiles;
  a.entries = ts.d_entries;
  a.n_groups = ts.n_groups;
  a.n_tiles = ts.n_tiles;
  a.img = ts.d_img;
  a.nr = nr;
  a.rp = (nr + 15) / 16 * 16;
  a.ximg = t.ximg;
  a.nblk = t.nblk;
  a.timg = t.timg;
  a.part = t.part;
  a.cnt = t.cnt;
  a.n_cnt = ts.n_cnt;
  a.work = t.cnt + ts.n_cnt;
  a.acc = t.acc;
  a.npad = h->npad;
  a.status = h->d_status;
  hh::dev::MrArgs m;
  std::memset(&m, 0, sizeof(m));
  m.pieces = ms.d_pieces;
  m.groups = ms.d_groups;
  m.tiles = ms.d_tiles;
  m.entries = ms.d_entries;
  m.n_groups = ms.n_groups;
  m.n_tiles = ms.n_tiles;
  m.nr = nr;
  m.rp = nr <= 32 ? 32 : (nr <= 64 ? 64 : 128);
  m.xh = t.xh;
  m.xl = t.xl;
  m.t32 = t.t32;
  m.acc = t.acc;
  m.npad = h->npad;
  m.status = h->d_status;
  mark(3);
  if (e == cudaSuccess) e = hh::dev::launch_mr(1, m, st);
  mark(4);
  if (e == cudaSuccess) e = hh::dev::launch_tc(1, a, h->sms, st);
  mark(5);
  if (e == cudaSuccess) e = hh::dev::launch_mr(2, m, st);
  mark(6);
  if (e == cudaSuccess) e = hh::dev::launch_tc(2, a, h->sms, st);
  mark(7);
  if (e == cudaSuccess) e = hh::dev::launch_finish(t.acc, nr, h->d_iperm, h->H.n, h->npad, out, ld_out, st);
  mark(8);
  return e;
}

// path: kStreamOnly (every column through the streaming passes), kAuto (the
// many-right-hand-side sequence from tc_min_nrhs() columns on), kMany (that
// sequence for any nrhs).  ev: 5 events for the streaming sequence (one chunk
// of up to 4 columns), 9 for the many-right-hand-side sequence (one chunk of
// up to 128 columns).
enum Path { kStreamOnly = 0, kAuto = 1, kMany = 2 };

int run_product(hh_matrix* h, int dir, const double* in, double* out, int nrhs, int64_t ld_in,
                int64_t ld_out, void* ws, size_t ws_bytes, cudaStream_t st, cudaEvent_t* ev = nullptr,
                Path path = kStreamOnly) {
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
  const int tmin = tc_min_nrhs();
  const bool use_tc = path == kMany || (path == kAuto && tmin > 0 && nrhs >= tmin);
  TcWs t{};
  if (use_tc) {
    const size_t tneed = tc_ws_layout(h, nullptr, nullptr);
    if (h->tc_ws_bytes < tneed) {
      cudaStreamSynchronize(st);
      cudaFree(h->d_tc_ws);
      h->d_tc_ws = nullptr;
      h->tc_ws_bytes = 0;
      if (cudaMalloc(&h->d_tc_ws, tneed) != cudaSuccess) {
        if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
        return fail(HH_ENOMEM, "cannot allocate the tensor-core workspace");
      }
      h->tc_ws_bytes = tneed;
    }
    tc_ws_layout(h, &t, (char*)h->d_tc_ws);
    MrSet& ms = h->mr[dir];
    if (!ms.d_dimg && ms.dimg_bytes > 0) {
      cudaStreamSynchronize(st);
      if (cudaMalloc(&ms.d_dimg, size_t(ms.dimg_bytes)) != cudaSuccess ||
          cudaMalloc(&ms.d_drexp, sizeof(int32_t) * 128 * size_t(ms.n_dentries)) != cudaSuccess) {
        cudaFree(ms.d_dimg);
        ms.d_dimg = nullptr;
        ms.d_drexp = nullptr;
        if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
        return fail(HH_ENOMEM, "cannot allocate the dense-block digit panels");
      }
      const cudaError_t pe = hh::dev::launch_td_pack(ms.d_dentries, ms.n_dentries, ms.d_dimg, ms.d_drexp, st);
      if (pe != cudaSuccess) {
        if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
        return fail(HH_ECUDA, std::string("dense panel packing failed: ") + cudaGetErrorString(pe));
      }
    }
    TcSet& ts = h->tc[dir];
    if (!ts.d_img && ts.img_bytes > 0) {
      cudaStreamSynchronize(st);
      if (cudaMalloc(&ts.d_img, size_t(ts.img_bytes)) != cudaSuccess) {
        ts.d_img = nullptr;
        if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
        return fail(HH_ENOMEM, "cannot allocate the packed tensor-core panels");
      }
      const cudaError_t pe = hh::dev::launch_tc_pack(ts.d_pieces, ts.d_groups, ts.n_groups, ts.d_entries,
                                                     ts.n_entries, ts.d_img, st);
      if (pe != cudaSuccess) {
        if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
        return fail(HH_ECUDA, std::string("panel packing failed: ") + cudaGetErrorString(pe));
      }
    }
  }
  for (int rb = 0; rb < nrhs;) {
    const int rem = nrhs - rb;
    cudaError_t e;
    int nr;
    if (use_tc) {
      nr = std::min(rem, hh::dev::kTcMaxRhs);
      e = run_tc(h, dir, in + (int64_t)rb * ld_in, out + (int64_t)rb * ld_out, nr, ld_in, ld_out, w, t, st, ev);
    } else {
      nr = rem >= 4 ? 4 : (rem >= 2 ? 2 : 1);
      e = run_stream(h, h->ss[dir], in + (int64_t)rb * ld_in, ld_in, nr, w.acc, w, st, ev);
      if (ev) cudaEventRecord(ev[3], st);
      if (e == cudaSuccess)
        e = hh::dev::launch_finish(w.acc, nr, h->d_iperm, h->H.n, h->npad, out + (int64_t)rb * ld_out, ld_out, st);
      if (ev) cudaEventRecord(ev[4], st);
    }
    if (e != cudaSuccess) {
      if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
      return fail(HH_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    }
    rb += nr;
  }
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  return HH_OK;
}

// Rebuild the many-column tables (tensor-core and CUDA-core) with the
// handle's current split length.
void rebuild_many(hh_matrix* h) {
  for (int d = 0; d < 2; ++d) {
    free_many(h, d);
    build_tc_set(h, d, h->tc[d]);
    build_mr_set(h, d, h->doff, h->dexp, h->mr[d]);
  }
}

// Streaming grid of one direction and phase: c CTAs per SM (clamped to the
// occupancy of each column count).
void set_stream_grid(hh_matrix* h, int dir, int phase, int c, int depth) {
  StreamSet& ss = h->ss[dir];
  ss.depth[phase] = depth;
  for (int nr : {1, 2, 4}) {
    const int occ = hh::dev::stream_blocks_per_sm(phase, ss.fset, nr, nr == 1 ? depth : 4);
    ss.grid[phase][nr] = h->sms * std::max(1, std::min(c, occ));
  }
  h->blocks_per_sm[dir][phase] = c;
}

// the streaming tables of both directions again (after h->item_bytes changed);
// the launch choices of the previous tables are kept
void rebuild_stream_sets(hh_matrix* h) {
  const hh::HostMatrix& H = h->H;
  std::vector<int64_t> toff(H.lr.size(), 0);
  int64_t t32 = 0, t64 = 0;
  for (size_t b = 0; b < H.lr.size(); ++b) {
    int64_t& tot = H.lr[b].fmt == hh::F64 ? t64 : t32;
    toff[b] = tot * hh::dev::kMaxNR;
    tot += H.lr[b].k;
  }
  std::vector<char> all(H.lr.size(), 1), rest(H.lr.size(), 0);
  for (size_t b = 0; b < H.lr.size(); ++b) rest[b] = H.lr[b].fmt == hh::F64;
  for (int dir = 0; dir < 2; ++dir) {
    StreamSet old = h->ss[dir];
    for (int p = 0; p < 2; ++p) {
      cudaFree(h->ss[dir].d_desc[p]);
      cudaFree(h->ss[dir].d_items[p]);
      cudaFree(h->ss_rest[dir].d_desc[p]);
      cudaFree(h->ss_rest[dir].d_items[p]);
    }
    h->ss[dir] = StreamSet();
    h->ss_rest[dir] = StreamSet();
    build_stream_set(h, dir, toff, h->doff, h->dexp, all, true, h->ss[dir]);
    build_stream_set(h, dir, toff, h->doff, h->dexp, rest, false, h->ss_rest[dir]);
    for (int phase = 1; phase <= 2; ++phase)
      if (h->blocks_per_sm[dir][phase] > 0) set_stream_grid(h, dir, phase, h->blocks_per_sm[dir][phase], old.depth[phase]);
  }
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
  return hh_build_ex(points, n, dim, kernel, kernel_param, leaf_size, eta, switch_level, tol, fmt_mask, seed,
                     HH_TREE_KD, device, out);
}

static int build_common(const double* points, int64_t n, int dim, int kernel, double kernel_param, int leaf_size,
                        double eta, int switch_level, double tol, uint32_t fmt_mask, uint64_t seed, int tree,
                        int compress_device, int device, hh_handle* out);

int hh_build_ex(const double* points, int64_t n, int dim, int kernel, double kernel_param, int leaf_size,
                double eta, int switch_level, double tol, uint32_t fmt_mask, uint64_t seed, int tree, int device,
                hh_handle* out) {
  return build_common(points, n, dim, kernel, kernel_param, leaf_size, eta, switch_level, tol, fmt_mask, seed, tree,
                      -1, device, out);
}

int hh_build_dev(const double* points, int64_t n, int dim, int kernel, double kernel_param, int leaf_size,
                 double eta, int switch_level, double tol, uint32_t fmt_mask, uint64_t seed, int tree, int device,
                 hh_handle* out) {
  if (device < 0) return fail(HH_EINVAL, "hh_build_dev needs a device >= 0");
  return build_common(points, n, dim, kernel, kernel_param, leaf_size, eta, switch_level, tol, fmt_mask, seed, tree,
                      device, device, out);
}

static int build_common(const double* points, int64_t n, int dim, int kernel, double kernel_param, int leaf_size,
                        double eta, int switch_level, double tol, uint32_t fmt_mask, uint64_t seed, int tree,
                        int compress_device, int device, hh_handle* out) {
  if (!out) return fail(HH_EINVAL, "out is NULL");
  if (tree != HH_TREE_KD && tree != HH_TREE_2D) return fail(HH_EINVAL, "unknown tree kind");
  *out = nullptr;
  if (!points) return fail(HH_EINVAL, "points is NULL");
  if (device < -1) return fail(HH_EINVAL, "device must be >= -1");
  hh_matrix* h = make_handle();
  if (!h) return fail(HH_ENOMEM, "out of host memory");
  try {
    hh::BuildParams p{kernel, kernel_param, leaf_size, eta, switch_level, tol, fmt_mask, seed, 0, tree};
    p.device = compress_device;
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
  } catch (const std::runtime_error& e) {
    delete h;
    const bool dev = std::string(e.what()).rfind("device compression", 0) == 0;
    return fail(dev ? HH_ECUDA : HH_EINVAL, e.what());
  } catch (const std::exception& e) {
    delete h;
    return fail(HH_EINVAL, e.what());
  }
  return finish_construction(h, device, out);
}

int hh_optimal_switch_level(const double* points, int64_t n, int dim, int kernel, double kernel_param,
                            int leaf_size, double eta, double tol, uint32_t fmt_mask, uint64_t seed, int tree,
                            int* ell_star, int* depth, double* gains) {
  return hh_optimal_switch_level_dev(points, n, dim, kernel, kernel_param, leaf_size, eta, tol, fmt_mask, seed, tree,
                                     -1, ell_star, depth, gains);
}

int hh_optimal_switch_level_dev(const double* points, int64_t n, int dim, int kernel, double kernel_param,
                                int leaf_size, double eta, double tol, uint32_t fmt_mask, uint64_t seed, int tree,
                                int device, int* ell_star, int* depth, double* gains) {
  if (!points || !ell_star) return fail(HH_EINVAL, "points or ell_star is NULL");
  if (tree != HH_TREE_KD && tree != HH_TREE_2D) return fail(HH_EINVAL, "unknown tree kind");
  if (device < -1) return fail(HH_EINVAL, "device must be >= -1");
  try {
    hh::BuildParams p{kernel, kernel_param, leaf_size, eta, 0, tol, fmt_mask, seed, 0, tree};
    p.device = device;
    if (const char* e = std::getenv("HH_BUILD_THREADS")) p.threads = std::atoi(e);
    std::vector<double> g;
    int L = 0;
    const int ell = hh::optimal_switch_level(points, n, dim, p, g, L);
    if (L >= HH_MAX_LEVELS) return fail(HH_EINVAL, "tree deeper than HH_MAX_LEVELS - 1");
    *ell_star = ell;
    if (depth) *depth = L;
    if (gains)
      for (int l = 0; l < HH_MAX_LEVELS; ++l) gains[l] = l <= L ? g[static_cast<size_t>(l)] : std::nan("");
  } catch (const std::bad_alloc&) {
    return fail(HH_ENOMEM, "out of host memory during the level search");
  } catch (const std::exception& e) {
    return fail(HH_EINVAL, e.what());
  }
  return HH_OK;
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

int hh_shard_plan(hh_handle h, int nranks, int64_t* bounds) {
  if (!h || nranks < 1 || !bounds) return fail(HH_EINVAL, "null handle or bounds, or nranks < 1");
  try {
    std::vector<int64_t> b;
    hh::shard_plan(h->H, nranks, b);
    std::copy(b.begin(), b.end(), bounds);
  } catch (const std::bad_alloc&) {
    return fail(HH_ENOMEM, "out of host memory");
  } catch (const std::exception& e) {
    return fail(HH_EINVAL, e.what());
  }
  return HH_OK;
}

int hh_shard(hh_handle h, int64_t p0, int64_t p1, int device, hh_handle* out) {
  if (!h || !out) return fail(HH_EINVAL, "null handle or output");
  if (p0 < 0 || p1 < p0 || p1 > h->H.n) return fail(HH_EINVAL, "shard range outside [0, n]");
  hh_matrix* s = make_handle();
  if (!s) return fail(HH_ENOMEM, "out of host memory");
  try {
    hh::make_shard(h->H, p0, p1, s->H);
  } catch (const std::bad_alloc&) {
    delete s;
    return fail(HH_ENOMEM, "out of host memory");
  } catch (const std::exception& e) {
    delete s;
    return fail(HH_EINVAL, e.what());
  }
  return finish_construction(s, device, out);
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
  for (const hh::LRBlock& B : H.lr) {
    if (B.k == 0) continue;
    if (tc_eligible(B)) {
      o->tc_blocks += 1;
      o->tc_factor_bytes += (B.m + B.n) * int64_t(B.k) * hh::fmt_bytes(B.fmt);
      o->tc_u_elems += B.m * int64_t(B.k);
      o->tc_v_elems += B.n * int64_t(B.k);
    } else if (B.fmt != hh::F64) {
      o->mr_u_elems += B.m * int64_t(B.k);
      o->mr_v_elems += B.n * int64_t(B.k);
    }
  }
  for (const hh::DenseBlock& D : H.dense) o->dense_elems += D.m * D.n;
  o->tuned = h->tuned;
  o->split_positions = h->split_len;
  for (int d = 0; d < 2; ++d)
    for (int p = 1; p <= 2; ++p) o->blocks_per_sm[2 * d + p - 1] = h->blocks_per_sm[d][p];
  for (int d = 0; d < 2; ++d)
    o->tc_panel_bytes[d] = (h->tc[d].d_img ? h->tc[d].img_bytes : 0) + (h->mr[d].d_dimg ? h->mr[d].dimg_bytes : 0);
  o->tree_step = H.step;
  o->build_device = H.build_device;
  o->build_fallback = H.build_fallback;
  o->build_device_seconds = H.build_device_seconds;
  o->dense_tc_elems = h->mr[0].dense_tc_elems;
  for (int d = 0; d < 2; ++d)
    for (int p = 1; p <= 2; ++p) o->stream_depth[2 * d + p - 1] = h->ss[d].depth[p];
  o->item_bytes = h->item_bytes;
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
  return run_product(h, 0, x, y, nrhs, ldx, ldy, h->d_ws, h->ws_bytes, (cudaStream_t)stream, nullptr, kAuto);
}

int hh_matvec_T(hh_handle h, const double* ybar, double* xbar, int nrhs, int64_t ldy, int64_t ldx,
                void* stream) {
  if (!h) return fail(HH_EINVAL, "null handle");
  return run_product(h, 1, ybar, xbar, nrhs, ldy, ldx, h->d_ws, h->ws_bytes, (cudaStream_t)stream, nullptr, kAuto);
}

int hh_solve_cg(hh_handle h, const double* b, double* x, double shift, double rtol, int max_iter, int* iters,
                double* relres, void* stream) {
  if (!h || !b || !x) return fail(HH_EINVAL, "null argument");
  if (h->device < 0) return fail(HH_ENOTSUP, "handle has no device data (built with device = -1)");
  if (max_iter < 0 || !(rtol >= 0.0)) return fail(HH_EINVAL, "max_iter < 0 or rtol < 0");
  const int64_t n = h->H.n;
  const size_t nb = static_cast<size_t>(n) * sizeof(double);
  if ((const char*)b < (const char*)x + nb && (const char*)x < (const char*)b + nb)
    return fail(HH_EINVAL, "b and x overlap");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  double* scratch = nullptr;  // r, p, q, dot partials, the solver's device scalars
  const size_t state_doubles = (sizeof(hh::dev::CgState) + sizeof(double) - 1) / sizeof(double);
  if (cudaMalloc(&scratch, 3 * nb + sizeof(double) * (hh::dev::kDotBlocks + state_doubles)) != cudaSuccess) {
    if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
    return fail(HH_ENOMEM, "cannot allocate the solver vectors");
  }
  double* r = scratch;
  double* p = r + n;
  double* q = p + n;
  double* part = q + n;
  hh::dev::CgState* dstate = reinterpret_cast<hh::dev::CgState*>(part + hh::dev::kDotBlocks);
  std::vector<double> hpart(hh::dev::kDotBlocks);
  int rc = HH_OK;
  cudaError_t e = cudaSuccess;
  auto dot = [&](const double* u, const double* v) {  // on the host: the start of the solve only
    double s = 0.0;
    if (e == cudaSuccess) e = hh::dev::launch_dot(u, v, n, part, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hpart.data(), part, sizeof(double) * hh::dev::kDotBlocks,
                                              cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (double v2 : hpart) s += v2;  // block order: deterministic, as the device sums them
    return s;
  };
  auto apply = [&](const double* in, double* out) {  // out = (A_h + shift I) in
    if (e != cudaSuccess || rc != HH_OK) return;
    rc = run_product(h, 0, in, out, 1, n, n, h->d_ws, h->ws_bytes, st);
    if (rc == HH_OK && shift != 0.0) e = hh::dev::launch_shift(out, in, shift, n, st);
  };
  // r = b - (A + shift I) x, p = r
  apply(x, q);
  if (e == cudaSuccess && rc == HH_OK) e = cudaMemcpyAsync(r, b, nb, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && rc == HH_OK) e = hh::dev::launch_shift(r, q, -1.0, n, st);
  if (e == cudaSuccess && rc == HH_OK) e = cudaMemcpyAsync(p, r, nb, cudaMemcpyDeviceToDevice, st);
  const double bnorm = std::sqrt(dot(b, b));
  double rr = dot(r, r);
  // iterations run on the device scalars (alpha, beta, the convergence and
  // breakdown tests in one-thread kernels); the host reads them back every
  // kCheck iterations, and iterations past the stop leave x untouched, so
  // the result and the count are those of testing every iteration
  constexpr int kCheck = 8;
  hh::dev::CgState hs{};
  hs.rr = rr;
  hs.threshold = rtol * bnorm;
  hs.done = (max_iter == 0 || !(std::sqrt(rr) > rtol * bnorm)) ? 1.0 : 0.0;
  hs.max_iter = max_iter;
  if (e == cudaSuccess && rc == HH_OK)
    e = cudaMemcpyAsync(dstate, &hs, sizeof(hs), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int launched = 0;
  while (rc == HH_OK && e == cudaSuccess && hs.done == 0.0 && launched < max_iter) {
    const int batch = std::min(kCheck, max_iter - launched);
    for (int j = 0; j < batch && rc == HH_OK && e == cudaSuccess; ++j) {
      apply(p, q);
      if (rc != HH_OK || e != cudaSuccess) break;
      e = hh::dev::launch_dot(p, q, n, part, st);
      if (e == cudaSuccess) e = hh::dev::launch_cg_alpha(part, dstate, st);
      if (e == cudaSuccess) e = hh::dev::launch_cg_step(x, r, p, q, dstate, n, st);
      if (e == cudaSuccess) e = hh::dev::launch_dot(r, r, n, part, st);
      if (e == cudaSuccess) e = hh::dev::launch_cg_beta(part, dstate, st);
      if (e == cudaSuccess) e = hh::dev::launch_cg_dir(p, r, dstate, n, st);
    }
    launched += batch;
    if (e == cudaSuccess && rc == HH_OK) e = cudaMemcpyAsync(&hs, dstate, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  const int it = static_cast<int>(hs.iters);
  rr = hs.rr;
  if (rc == HH_OK && e == cudaSuccess && hs.breakdown != 0.0)
    rc = fail(HH_EINVAL, "conjugate gradients broke down: p^T (A + shift I) p <= 0");
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(scratch);
  if (rc == HH_OK && e != cudaSuccess) rc = fail(HH_ECUDA, std::string("solver launch failed: ") + cudaGetErrorString(e));
  if (iters) *iters = it;
  if (relres) *relres = bnorm > 0.0 ? std::sqrt(rr) / bnorm : 0.0;
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  return rc;
}

int hh_matvec_ws(hh_handle h, int transpose, const double* in, double* out, int nrhs, int64_t ld_in,
                 int64_t ld_out, void* workspace, size_t workspace_bytes, void* stream) {
  if (!h) return fail(HH_EINVAL, "null handle");
  return run_product(h, transpose ? 1 : 0, in, out, nrhs, ld_in, ld_out, workspace, workspace_bytes,
                     (cudaStream_t)stream);
}

// CUDA events around one product (n_ev = 5 for the streaming sequence, 9 for
// the many-right-hand-side sequence); writes the n_ev - 1 intervals to ms.
static int timed_product(hh_handle h, int dir, const double* in, double* out, int nrhs, int64_t ld_in, int64_t ld_out,
                  void* stream, float* ms, int n_ev, bool many) {
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  cudaEvent_t ev[9];
  int made = 0;
  for (; made < n_ev; ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
  int rc = made == n_ev ? HH_OK : fail(HH_ECUDA, "cudaEventCreate failed");
  if (rc == HH_OK)
    rc = run_product(h, dir, in, out, nrhs, ld_in, ld_out, h->d_ws, h->ws_bytes, (cudaStream_t)stream, ev,
                     many ? kMany : kStreamOnly);
  if (rc == HH_OK && cudaEventSynchronize(ev[n_ev - 1]) != cudaSuccess) rc = fail(HH_ECUDA, "event synchronize failed");
  for (int i = 0; rc == HH_OK && i < n_ev - 1; ++i)
    if (cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]) != cudaSuccess) rc = fail(HH_ECUDA, "event timing failed");
  for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  return rc;
}

int hh_matvec_timed(hh_handle h, int transpose, const double* in, double* out, int nrhs, int64_t ld_in,
                    int64_t ld_out, void* stream, float* ms) {
  if (!h || !ms) return fail(HH_EINVAL, "null argument");
  if (h->device < 0) return fail(HH_ENOTSUP, "handle has no device data");
  if (nrhs < 1 || nrhs > hh::dev::kMaxNR || nrhs == 3) return fail(HH_EINVAL, "nrhs must be 1, 2 or 4");
  return timed_product(h, transpose ? 1 : 0, in, out, nrhs, ld_in, ld_out, stream, ms, 5, false);
}

int hh_matvec_stages(hh_handle h, int transpose, const double* in, double* out, int nrhs, int64_t ld_in,
                     int64_t ld_out, void* stream, float* ms) {
  if (!h || !ms) return fail(HH_EINVAL, "null argument");
  if (h->device < 0) return fail(HH_ENOTSUP, "handle has no device data");
  if (nrhs < 1 || nrhs > hh::dev::kTcMaxRhs) return fail(HH_EINVAL, "nrhs must be between 1 and 128");
  return timed_product(h, transpose ? 1 : 0, in, out, nrhs, ld_in, ld_out, stream, ms, 9, true);
}

int hh_autotune(hh_handle h, int nrhs_many) {
  if (!h) return fail(HH_EINVAL, "null handle");
  if (h->device < 0) return fail(HH_ENOTSUP, "handle has no device data");
  if (nrhs_many < 0 || nrhs_many > hh::dev::kTcMaxRhs) return fail(HH_EINVAL, "nrhs_many must be in [0, 128]");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  const int64_t n = h->H.n;
  const int cols = std::max(4, nrhs_many);
  double* x = nullptr;
  double* y = nullptr;
  cudaStream_t st = nullptr;
  int rc = HH_OK;
  if (cudaMalloc(&x, sizeof(double) * n * cols) != cudaSuccess ||
      cudaMalloc(&y, sizeof(double) * n * cols) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
    rc = fail(HH_ENOMEM, "cannot allocate autotuning buffers");
  if (rc == HH_OK && cudaMemsetAsync(x, 0x3f, sizeof(double) * n * cols, st) != cudaSuccess)  // entries ~4.8e-4
    rc = fail(HH_ECUDA, "cudaMemsetAsync failed");
  float ms[8];
  // streaming passes, one column: (1) the factor bytes of a phase-1 item
  // (the work decomposition; both directions' whole products timed);
  // (2) per direction and phase, the pipeline depth and the CTAs per SM
  auto product_ms = [&](int reps) {
    float t = 1e30f;
    for (int rep = 0; rep < reps && rc == HH_OK; ++rep) {
      float sum = 0.f;
      for (int dir = 0; dir < 2 && rc == HH_OK; ++dir) {
        rc = timed_product(h, dir, x, y, 1, n, n, st, ms, 5, false);
        for (int q = 0; q < 4; ++q) sum += ms[q];
      }
      if (rep >= 1) t = std::min(t, sum);
    }
    return t;
  };
  if (rc == HH_OK) {
    int64_t best_b = h->item_bytes;
    float best = 1e30f;
    for (int64_t ib : {int64_t(16) << 10, int64_t(64) << 10, int64_t(256) << 10}) {
      h->item_bytes = ib;
      try {
        rebuild_stream_sets(h);
      } catch (const std::exception& e) {
        rc = fail(HH_ECUDA, e.what());
        break;
      }
      const float t = product_ms(4);
      if (rc == HH_OK && t < best) {
        best = t;
        best_b = ib;
      }
    }
    h->item_bytes = best_b;
    try {
      rebuild_stream_sets(h);
    } catch (const std::exception& e) {
      if (rc == HH_OK) rc = fail(HH_ECUDA, e.what());
    }
  }
  for (int dir = 0; dir < 2 && rc == HH_OK; ++dir)
    for (int phase = 1; phase <= 2 && rc == HH_OK; ++phase) {
      int best_c = 0, best_d = 4;
      float best = 1e30f;
      for (int depth : {4, 3, 6}) {
        const int occ = hh::dev::stream_blocks_per_sm(phase, h->ss[dir].fset, 1, depth);
        for (int c = 1; c <= occ && rc == HH_OK; ++c) {
          set_stream_grid(h, dir, phase, c, depth);
          float t = 1e30f;
          for (int rep = 0; rep < 6 && rc == HH_OK; ++rep) {
            rc = timed_product(h, dir, x, y, 1, n, n, st, ms, 5, false);
            if (rep >= 1) t = std::min(t, ms[phase]);
          }
          if (t < best) {
            best = t;
            best_c = c;
            best_d = depth;
          }
        }
      }
      set_stream_grid(h, dir, phase, best_c > 0 ? best_c : 1, best_d);
    }
  // many columns: the position split of the phase-1 items
  if (rc == HH_OK && nrhs_many > 0) {
    int best_s = h->split_len;
    float best = 1e30f;
    for (int split : {1024, 2048, 4096, 8192, 16384, 32768, 65536}) {
      h->split_len = split;
      try {
        rebuild_many(h);
      } catch (const std::exception& e) {
        rc = fail(HH_ECUDA, e.what());
        break;
      }
      float t = 1e30f;
      for (int rep = 0; rep < 4 && rc == HH_OK; ++rep) {
        rc = timed_product(h, 0, x, y, nrhs_many, n, n, st, ms, 9, true);
        float sum = 0.f;
        for (int k = 0; k < 8; ++k) sum += ms[k];
        if (rep >= 1) t = std::min(t, sum);
      }
      if (rc != HH_OK) break;
      if (t < best) {
        best = t;
        best_s = split;
      }
    }
    h->split_len = best_s;
    try {
      rebuild_many(h);
    } catch (const std::exception& e) {
      if (rc == HH_OK) rc = fail(HH_ECUDA, e.what());
    }
  }
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaFree(x);
  cudaFree(y);
  if (rc == HH_OK) h->tuned = 1;
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
  if (rc == HH_OK)
    rc = run_product(h, transpose ? 1 : 0, dx, dy, nrhs, n, n, h->d_ws, h->ws_bytes, st, nullptr, kAuto);
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
  if (word & (4 | 8)) return fail(HH_ETIMEOUT, "a bounded device wait expired (status word " + std::to_string(word) + ")");
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
// Batches of independent matrices (hh_batch_*, see include/hh.h): the
// streaming tables of every matrix concatenated over one position space, so
// that one product of the whole batch is four launches whatever the count.
struct hh_batch_s {
  std::vector<hh_matrix*> mats;
  int device = -1;
  int sms = 0;
  int count = 0;
  int64_t np = 0;                 // concatenated positions
  std::vector<int64_t> offsets;   // caller-order vector offsets, count + 1
  int64_t* d_xofs = nullptr;
  int64_t* d_pofs = nullptr;
  int64_t* d_ns = nullptr;
  int32_t* d_perm = nullptr;
  StreamSet ss[2];
  void* d_ws = nullptr;
  float* xs = nullptr;
  float* xs_lo = nullptr;
  double* acc = nullptr;
  float* t32 = nullptr;
  float2* t64 = nullptr;
  int* counters = nullptr;
  int persistent = 1;             // one cooperative kernel per product (0: prep, two passes, finish)
  int pgrid[2] = {0, 0};          // its co-resident grid per direction
  cudaStream_t cap = nullptr;     // private stream for graph capture
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  const double* gx[2] = {nullptr, nullptr};
  double* gy[2] = {nullptr, nullptr};
};

namespace {

void free_batch(hh_batch_s* b) {
  if (b->device < 0) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != b->device) cudaSetDevice(b->device);
  for (int d = 0; d < 2; ++d) {
    for (int p = 0; p < 2; ++p) {
      cudaFree(b->ss[d].d_desc[p]);
      cudaFree(b->ss[d].d_items[p]);
    }
    if (b->gexec[d]) cudaGraphExecDestroy(b->gexec[d]);
  }
  cudaFree(b->d_xofs);
  cudaFree(b->d_pofs);
  cudaFree(b->d_ns);
  cudaFree(b->d_perm);
  cudaFree(b->d_ws);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (cur >= 0 && cur != b->device) cudaSetDevice(cur);
}

// one batch product: the persistent kernel, or prep, phase 1, phase 2, finish
cudaError_t batch_launches(hh_batch_s* b, int dir, const double* x, double* y, cudaStream_t st) {
  if (b->persistent && b->pgrid[dir] > 0) {
    hh::dev::BatchArgs ba;
    std::memset(&ba, 0, sizeof(ba));
    for (int phase = 1; phase <= 2; ++phase) {
      const StreamSet& set = b->ss[dir];
      hh::dev::StreamArgs& a = ba.pass[phase - 1];
      a.desc = set.d_desc[phase - 1];
      a.items = set.d_items[phase - 1];
      a.n_items = set.n_items[phase - 1];
      a.nr = 1;
      a.npad = b->np;
      a.xs = b->xs;
      a.xs_lo = b->xs_lo;
      a.t32 = b->t32;
      a.t64 = b->t64;
      a.acc = b->acc;
      a.status = b->mats[0]->d_status;
      a.counter = b->counters + (phase - 1);
    }
    ba.x = x;
    ba.y = y;
    ba.xofs = b->d_xofs;
    ba.perm = b->d_perm;
    ba.pofs = b->d_pofs;
    ba.ns = b->d_ns;
    ba.count = b->count;
    ba.np = b->np;
    return hh::dev::launch_batch_persistent(b->ss[dir].fset, ba, b->pgrid[dir], st);
  }
  cudaError_t e = hh::dev::launch_batch_prep(x, b->d_xofs, b->d_perm, b->d_pofs, b->d_ns, b->count, b->np, b->xs,
                                             b->xs_lo, b->acc, b->counters, st);
  bool p1 = false;
  for (int phase = 1; phase <= 2 && e == cudaSuccess; ++phase) {
    const StreamSet& set = b->ss[dir];
    hh::dev::StreamArgs a;
    std::memset(&a, 0, sizeof(a));
    a.desc = set.d_desc[phase - 1];
    a.items = set.d_items[phase - 1];
    a.n_items = set.n_items[phase - 1];
    a.nr = 1;
    a.npad = b->np;
    a.xs = b->xs;
    a.xs_lo = b->xs_lo;
    a.t32 = b->t32;
    a.t64 = b->t64;
    a.acc = b->acc;
    a.status = b->mats[0]->d_status;
    a.counter = b->counters + (phase - 1);
    if (a.n_items == 0) continue;
    const int grid = std::max(1, std::min(set.grid[phase][1], a.n_items));
    e = hh::dev::launch_stream(phase, set.fset, a, grid, st, p1);
    p1 = phase == 1;
  }
  if (e == cudaSuccess)
    e = hh::dev::launch_batch_finish(b->acc, b->d_xofs, b->d_perm, b->d_pofs, b->d_ns, b->count, b->np, y, st);
  return e;
}

}  // namespace

extern "C" {

int hh_batch_create(const hh_handle* hs, int count, hh_batch* out) {
  if (!out) return fail(HH_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !hs) return fail(HH_EINVAL, "need at least one handle");
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return fail(HH_EINVAL, "null handle in batch");
    if (hs[i]->device < 0) return fail(HH_ENOTSUP, "handle without device data in batch");
    if (hs[i]->device != hs[0]->device) return fail(HH_EINVAL, "handles on different devices");
  }
  hh_batch_s* b = new (std::nothrow) hh_batch_s();
  if (!b) return fail(HH_ENOMEM, "out of host memory");
  int cur = -1;
  cudaGetDevice(&cur);
  try {
    ck(cudaSetDevice(hs[0]->device), "cudaSetDevice");
    b->device = hs[0]->device;
    b->sms = hs[0]->sms;
    b->count = count;
    std::vector<int64_t> pofs(count + 1, 0), ns(count, 0);
    b->offsets.assign(count + 1, 0);
    int64_t t32 = 0, t64 = 0;
    std::vector<int64_t> t32o(count), t64o(count);
    for (int i = 0; i < count; ++i) {
      hh_matrix* h = hs[i];
      b->mats.push_back(h);
      ns[i] = h->H.n;
      pofs[i + 1] = pofs[i] + h->npad;
      b->offsets[i + 1] = b->offsets[i] + h->H.n;
      t32o[i] = t32;
      t64o[i] = t64;
      t32 += h->t32_elems;
      t64 += h->t64_elems;
    }
    b->np = pofs[count];
    if (b->np + 64 > (int64_t(1) << 31)) throw std::invalid_argument("batch too large for 32-bit positions");
    std::vector<int32_t> perm(static_cast<size_t>(b->np), 0);
    for (int i = 0; i < count; ++i) std::copy(hs[i]->H.perm.begin(), hs[i]->H.perm.end(), perm.begin() + pofs[i]);
    b->d_xofs = upload(b->offsets);
    b->d_pofs = upload(pofs);
    b->d_ns = upload(ns);
    b->d_perm = upload(perm);
    for (int dir = 0; dir < 2; ++dir) {
      unsigned present = 0;
      for (int p = 0; p < 2; ++p) {
        std::vector<hh::dev::StreamDesc> desc;
        std::vector<std::pair<Item, double>> items;
        for (int i = 0; i < count; ++i) {
          const StreamSet& src = hs[i]->ss[dir];
          const int base = (int)desc.size();
          for (hh::dev::StreamDesc d : src.h_desc[p]) {
            d.in_off += (int32_t)pofs[i];
            d.out_off += (int32_t)pofs[i];
            if (d.mode == 0) d.toff += (d.fmt == hh::F64 ? t64o[i] : t32o[i]) * hh::dev::kMaxNR;
            desc.push_back(d);
          }
          for (size_t k = 0; k < src.h_items[p].size(); ++k) {
            Item it = src.h_items[p][k];
            it.idx += base;
            items.push_back({it, src.h_cost[p][k]});
          }
          present |= src.present;
        }
        std::stable_sort(items.begin(), items.end(), [](const auto& x, const auto& y) { return x.second > y.second; });
        std::vector<Item> flat;
        for (auto& it : items) flat.push_back(it.first);
        b->ss[dir].d_desc[p] = upload(desc);
        b->ss[dir].d_items[p] = upload(flat);
        b->ss[dir].n_items[p] = (int)flat.size();
      }
      b->ss[dir].present = present;
      b->ss[dir].fset = hh::dev::pass_set_for(present);
      for (int phase = 1; phase <= 2; ++phase)
        b->ss[dir].grid[phase][1] = b->sms * hh::dev::stream_blocks_per_sm(phase, b->ss[dir].fset, 1);
    }
    // workspace: shifted input copies, output accumulator, t arenas, counters
    size_t off = 0;
    auto take = [&](size_t bytes) {
      size_t o = off;
      off = align256(off + bytes);
      return o;
    };
    const size_t o_xs = take(sizeof(float) * 4 * b->np), o_lo = take(sizeof(float) * 4 * b->np);
    const size_t o_acc = take(sizeof(double) * b->np);
    const size_t o_t32 = take(sizeof(float) * std::max<int64_t>(1, t32 * hh::dev::kMaxNR));
    const size_t o_t64 = take(sizeof(float2) * std::max<int64_t>(1, t64 * hh::dev::kMaxNR));
    const size_t o_cnt = take(256);
    ck(cudaMalloc(&b->d_ws, off), "cudaMalloc batch workspace");
    char* w = static_cast<char*>(b->d_ws);
    b->xs = reinterpret_cast<float*>(w + o_xs);
    b->xs_lo = reinterpret_cast<float*>(w + o_lo);
    b->acc = reinterpret_cast<double*>(w + o_acc);
    b->t32 = reinterpret_cast<float*>(w + o_t32);
    b->t64 = reinterpret_cast<float2*>(w + o_t64);
    b->counters = reinterpret_cast<int*>(w + o_cnt);
    ck(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    // the persistent kernel needs cooperative launch and one co-resident grid
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device);
    const char* env = std::getenv("HH_BATCH_LAUNCHES");
    b->persistent = (coop && !(env && std::atoi(env) == 4)) ? 1 : 0;
    for (int d = 0; d < 2; ++d) b->pgrid[d] = hh::dev::batch_persistent_grid(b->ss[d].fset, b->sms);
  } catch (const CudaError& e) {
    free_batch(b);
    delete b;
    if (cur >= 0) cudaSetDevice(cur);
    return fail(HH_ECUDA, e.what());
  } catch (const std::bad_alloc&) {
    free_batch(b);
    delete b;
    if (cur >= 0) cudaSetDevice(cur);
    return fail(HH_ENOMEM, "out of host memory");
  } catch (const std::exception& e) {
    free_batch(b);
    delete b;
    if (cur >= 0) cudaSetDevice(cur);
    return fail(HH_EINVAL, e.what());
  }
  if (cur >= 0 && cur != b->device) cudaSetDevice(cur);
  *out = b;
  return HH_OK;
}

int hh_batch_offsets(hh_batch b, int64_t* offsets) {
  if (!b || !offsets) return fail(HH_EINVAL, "null argument");
  std::copy(b->offsets.begin(), b->offsets.end(), offsets);
  return HH_OK;
}

int hh_batch_matvec(hh_batch b, int transpose, const double* x, double* y, void* stream) {
  if (!b || !x || !y) return fail(HH_EINVAL, "null argument");
  const size_t span = static_cast<size_t>(b->offsets[b->count]) * sizeof(double);
  if ((const char*)x < (const char*)y + span && (const char*)y < (const char*)x + span)
    return fail(HH_EINVAL, "input and output overlap");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != b->device && cudaSetDevice(b->device) != cudaSuccess) return fail(HH_ECUDA, "cudaSetDevice failed");
  cudaError_t e = batch_launches(b, transpose ? 1 : 0, x, y, (cudaStream_t)stream);
  if (cur >= 0 && cur != b->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return fail(HH_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  return HH_OK;
}

int hh_batch_matvec_graph(hh_batch b, int transpose, const double* x, double* y, void* stream) {
  if (!b || !x || !y) return fail(HH_EINVAL, "null argument");
  const size_t span = static_cast<size_t>(b->offsets[b->count]) * sizeof(double);
  if ((const char*)x < (const char*)y + span && (const char*)y < (const char*)x + span)
    return fail(HH_EINVAL, "input and output overlap");
  const int dir = transpose ? 1 : 0;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != b->device && cudaSetDevice(b->device) != cudaSuccess) return fail(HH_ECUDA, "cudaSetDevice failed");
  int rc = HH_OK;
  if (!b->gexec[dir] || b->gx[dir] != x || b->gy[dir] != y) {
    if (b->gexec[dir]) {
      cudaStreamSynchronize((cudaStream_t)stream);
      cudaGraphExecDestroy(b->gexec[dir]);
      b->gexec[dir] = nullptr;
    }
    cudaError_t e = cudaSuccess, e2 = cudaSuccess;
    for (int attempt = 0; attempt < 2; ++attempt) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
      e2 = cudaSuccess;
      if (e == cudaSuccess) {
        e2 = batch_launches(b, dir, x, y, b->cap);
        e = cudaStreamEndCapture(b->cap, &g);
      }
      if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&b->gexec[dir], g, 0);
      if (g) cudaGraphDestroy(g);
      if ((e == cudaSuccess && e2 == cudaSuccess) || !b->persistent) break;
      // the cooperative kernel could not be captured: the four-launch sequence
      cudaGetLastError();
      b->gexec[dir] = nullptr;
      b->persistent = 0;
    }
    if (e != cudaSuccess || e2 != cudaSuccess) {
      b->gexec[dir] = nullptr;
      rc = fail(HH_ECUDA, std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    } else {
      b->gx[dir] = x;
      b->gy[dir] = y;
    }
  }
  if (rc == HH_OK && cudaGraphLaunch(b->gexec[dir], (cudaStream_t)stream) != cudaSuccess)
    rc = fail(HH_ECUDA, "cudaGraphLaunch failed");
  if (cur >= 0 && cur != b->device) cudaSetDevice(cur);
  return rc;
}

void hh_batch_free(hh_batch b) {
  if (!b) return;
  free_batch(b);
  delete b;
}

}  // extern "C"

extern "C" int hh_matvec_noalloc(hh_handle h, int transpose, const double* in, double* out, void* stream) {
  if (!h || !in || !out) return fail(HH_EINVAL, "null argument");
  if (h->device < 0) return fail(HH_ENOTSUP, "handle has no device data (built with device = -1)");
  // scratch for one right-hand side, in the layout of the handle workspace
  const size_t need = ws_layout(h, nullptr, nullptr, 1);
  if (need > kNoAllocScratchBytes)
    return fail(HH_EINVAL, "hh_matvec_noalloc: this matrix needs " + std::to_string(need) +
                               " bytes of scratch, more than the fixed " +
                               std::to_string(kNoAllocScratchBytes) + " bytes; use hh_matvec or hh_matvec_ws");
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
    WsView w;
    ws_layout(h, &w, (char*)base, 1);
    const int dir = transpose ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    // prep clears the accumulator and the work counters on every call
    cudaError_t e = run_stream(h, h->ss[dir], in, h->H.n, 1, w.acc, w, st, nullptr);
    if (e == cudaSuccess) e = hh::dev::launch_finish(w.acc, 1, h->d_iperm, h->H.n, h->npad, out, h->H.n, st);
    if (e != cudaSuccess) rc = fail(HH_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  }
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  return rc;
}
