// Serialized H_h file and layout validation.
//
// Little-endian layout, version 1 ("HHMATv01"):
//   magic 8 bytes; int64[16] {N, dim, L, ell, leaf, kernel, n_lr, n_dense,
//   fmt_mask, arena_bytes, dense_elems, n_nodes, seed, 0, 0, 0};
//   float64[8] {eta, tol, kernel_param, ||H~||_F, 0, 0, 0, 0};
//   points float64[N*dim] (user order); perm int32[N];
//   nodes n_nodes x {int64 off, int64 size, float64 lo[dim], float64 hi[dim]};
//   LRBlock[n_lr] (104 bytes each); DenseBlock[n_dense] (56 bytes each);
//   arena uint8[arena_bytes]; dense float64[dense_elems].
#include <cstdio>
#include <cstring>
#include <memory>
#include <stdexcept>

#include "hh_host.h"

namespace hh {

namespace {
const char kMagic[8] = {'H', 'H', 'M', 'A', 'T', 'v', '0', '1'};

struct File {
  FILE* f;
  explicit File(FILE* f_) : f(f_) {}
  ~File() {
    if (f) std::fclose(f);
  }
};

void wr(FILE* f, const void* p, size_t n) {
  if (n && std::fwrite(p, 1, n, f) != n) throw IoError("write failed");
}
void rd(FILE* f, void* p, size_t n) {
  if (n && std::fread(p, 1, n, f) != n) throw IoError("file truncated");
}
}  // namespace

void validate(const HostMatrix& h) {
  if (h.n < 1 || h.dim < 1 || h.dim > 3 || h.L < 0 || h.L > 46 || h.ell < 0 || h.ell > h.L)
    throw std::invalid_argument("bad header");
  if (h.step != 1 && h.step != h.dim) throw std::invalid_argument("bad tree step");
  if (h.L % h.step || h.ell % h.step) throw std::invalid_argument("levels are not tree levels");
  if ((int64_t)h.perm.size() != h.n || (int64_t)h.points.size() != h.n * h.dim)
    throw std::invalid_argument("bad point / permutation arrays");
  std::vector<char> seen(h.n, 0);
  for (int32_t p : h.perm) {
    if (p < 0 || p >= h.n || seen[p]) throw std::invalid_argument("perm is not a permutation");
    seen[p] = 1;
  }
  const int64_t nn = (int64_t(2) << h.L) - 1;
  if ((int64_t)h.node_off.size() != nn) throw std::invalid_argument("bad node table");
  auto check_range = [&](int level, int idx, int64_t off, int64_t size) {
    if (level < 0 || level > h.L || idx < 0 || idx >= (int64_t(1) << level))
      throw std::invalid_argument("bad cluster index");
    int64_t node = (int64_t(1) << level) - 1 + idx;
    if (h.node_off[node] != off || h.node_size[node] != size)
      throw std::invalid_argument("block range does not match its cluster");
    if (off < 0 || size < 0 || off + size > h.n) throw std::invalid_argument("block out of range");
  };
  for (const LRBlock& b : h.lr) {
    if (b.fmt < 0 || b.fmt >= NFMT || b.k < 0) throw std::invalid_argument("bad block format/rank");
    check_range(b.level, b.i, b.row_off, b.m);
    check_range(b.level, b.j, b.col_off, b.n);
    const int sz = fmt_bytes(b.fmt);
    if (b.ldu < b.m || b.ldv < b.n || (b.ldu * sz) % 16 || (b.ldv * sz) % 16)
      throw std::invalid_argument("bad leading dimension");
    if (b.u_off % 16 || b.v_off % 16 || b.u_off < 0 || b.v_off < 0 ||
        b.u_off + b.ldu * b.k * sz > (int64_t)h.arena.size() ||
        b.v_off + b.ldv * b.k * sz > (int64_t)h.arena.size())
      throw std::invalid_argument("factor outside the arena or misaligned");
    if (b.exp_u < -1100 || b.exp_u > 1100 || b.exp_v < -1100 || b.exp_v > 1100)
      throw std::invalid_argument("bad scale exponent");
  }
  for (const DenseBlock& d : h.dense) {
    check_range(d.level, d.i, d.row_off, d.m);
    check_range(d.level, d.j, d.col_off, d.n);
    if (d.d_off < 0 || d.d_off + d.m * d.n > (int64_t)h.dense_data.size())
      throw std::invalid_argument("dense block outside its arena");
  }
}

void save_file(const HostMatrix& h, const std::string& path) {
  File f(std::fopen(path.c_str(), "wb"));
  if (!f.f) throw IoError("cannot open " + path + " for writing");
  const int64_t nn = (int64_t)h.node_off.size();
  int64_t ints[16] = {h.n, h.dim, h.L, h.ell, h.leaf, h.kernel, (int64_t)h.lr.size(),
                      (int64_t)h.dense.size(), (int64_t)h.fmt_mask, (int64_t)h.arena.size(),
                      (int64_t)h.dense_data.size(), nn, (int64_t)h.seed, (int64_t)h.step, 0, 0};
  double reals[8] = {h.eta, h.tol, h.kparam, h.norm_ht, 0, 0, 0, 0};
  wr(f.f, kMagic, 8);
  wr(f.f, ints, sizeof(ints));
  wr(f.f, reals, sizeof(reals));
  wr(f.f, h.points.data(), h.points.size() * 8);
  wr(f.f, h.perm.data(), h.perm.size() * 4);
  for (int64_t q = 0; q < nn; ++q) {
    wr(f.f, &h.node_off[q], 8);
    wr(f.f, &h.node_size[q], 8);
    wr(f.f, &h.node_lo[q * h.dim], 8 * h.dim);
    wr(f.f, &h.node_hi[q * h.dim], 8 * h.dim);
  }
  wr(f.f, h.lr.data(), h.lr.size() * sizeof(LRBlock));
  wr(f.f, h.dense.data(), h.dense.size() * sizeof(DenseBlock));
  wr(f.f, h.arena.data(), h.arena.size());
  wr(f.f, h.dense_data.data(), h.dense_data.size() * 8);
}

void load_file(const std::string& path, HostMatrix& h) {
  File f(std::fopen(path.c_str(), "rb"));
  if (!f.f) throw IoError("cannot open " + path);
  char magic[8];
  rd(f.f, magic, 8);
  if (std::memcmp(magic, kMagic, 8) != 0) throw std::invalid_argument("not an H_h file");
  int64_t ints[16];
  double reals[8];
  rd(f.f, ints, sizeof(ints));
  rd(f.f, reals, sizeof(reals));
  h = HostMatrix();
  h.n = ints[0];
  h.dim = (int32_t)ints[1];
  h.L = (int32_t)ints[2];
  h.ell = (int32_t)ints[3];
  h.leaf = (int32_t)ints[4];
  h.kernel = (int32_t)ints[5];
  const int64_t nlr = ints[6], ndn = ints[7];
  h.fmt_mask = (uint32_t)ints[8];
  const int64_t abytes = ints[9], delems = ints[10], nn = ints[11];
  h.seed = (uint64_t)ints[12];
  h.step = ints[13] > 0 ? (int32_t)ints[13] : 1;  // files without the field hold a binary tree
  h.eta = reals[0];
  h.tol = reals[1];
  h.kparam = reals[2];
  h.norm_ht = reals[3];
  if (h.n < 1 || h.n > (int64_t(1) << 31) || h.dim < 1 || h.dim > 3 || h.L < 0 || h.L > 46 ||
      nn != (int64_t(2) << h.L) - 1 || nlr < 0 || ndn < 0 || abytes < 0 || delems < 0 ||
      nlr > (int64_t(1) << 40) || ndn > (int64_t(1) << 40))
    throw std::invalid_argument("bad H_h header");
  h.points.resize(h.n * h.dim);
  rd(f.f, h.points.data(), h.points.size() * 8);
  h.perm.resize(h.n);
  rd(f.f, h.perm.data(), h.perm.size() * 4);
  h.node_off.resize(nn);
  h.node_size.resize(nn);
  h.node_lo.resize(nn * h.dim);
  h.node_hi.resize(nn * h.dim);
  for (int64_t q = 0; q < nn; ++q) {
    rd(f.f, &h.node_off[q], 8);
    rd(f.f, &h.node_size[q], 8);
    rd(f.f, &h.node_lo[q * h.dim], 8 * h.dim);
    rd(f.f, &h.node_hi[q * h.dim], 8 * h.dim);
  }
  h.lr.resize(nlr);
  rd(f.f, h.lr.data(), nlr * sizeof(LRBlock));
  h.dense.resize(ndn);
  rd(f.f, h.dense.data(), ndn * sizeof(DenseBlock));
  h.arena.resize(abytes);
  rd(f.f, h.arena.data(), abytes);
  h.dense_data.resize(delems);
  rd(f.f, h.dense_data.data(), delems * 8);
  char extra;
  if (std::fread(&extra, 1, 1, f.f) != 0) throw std::invalid_argument("trailing bytes in H_h file");
  validate(h);
}

}  // namespace hh
