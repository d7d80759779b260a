// Checkpoint and restore of a handle's strip state at a strip boundary
// (sgdg_checkpoint / sgdg_restore / sgdg_checkpoint_verify).
//
// The strip scheme of Sect. 2 carries U^-_j from one strip to the next; the
// library also carries the last two strip solutions (warm starts), the next
// right-hand side, the start time of the next strip and, for Vlasov-Poisson
// handles, the field E per finest cell (Sect. 5.3).  A checkpoint holds all
// of it in FP64, so a restored handle continues exactly where the writer
// stopped.  Layout (native endianness, no padding):
//   "SGDGCKP2" | u64 problem hash | i64 n_coeffs | i64 n_spatial
//   | i32 flags[8] = {have_initial, first_strip, solved, nsolved, warm,
//                     has_prev2, has_guess, has_field}
//   | f64 t_now | rhs[n_coeffs] | u_sol[n_coeffs] | U_end[n_spatial]
//   | u_prev2[n_coeffs] if has_prev2 | guess[n_coeffs] if has_guess
//   | if has_field: i32 d, i32 ncells, i32 nverts, i32 updated,
//                   E[d][ncells], rho[nverts], phi[nverts]
//   | u64 FNV-1a 64 of every byte before it
// Restore reads and checks the whole file on the host (magic, sizes, the
// checksum, nothing after the trailer) before it touches the handle, so a
// truncated or corrupted file leaves the handle's state as it was.
#include <cstdio>
#include <cstring>
#include <memory>

#include "handle.h"

namespace sgdg {

namespace {

constexpr char kMagic[8] = {'S', 'G', 'D', 'G', 'C', 'K', 'P', '2'};

struct File {
  std::FILE* f = nullptr;
  explicit File(std::FILE* ff) : f(ff) {}
  ~File() { if (f) std::fclose(f); }
};

// writer that hashes what it writes
struct Writer {
  std::FILE* f;
  unsigned long long sum = kFnvBasis;
  bool put(const void* p, size_t n) {
    fnv1a64(sum, p, n);
    return std::fwrite(p, 1, n, f) == n;
  }
};

// reader that hashes what it reads
struct Reader {
  std::FILE* f;
  unsigned long long sum = kFnvBasis;
  bool get(void* p, size_t n) {
    if (std::fread(p, 1, n, f) != n) return false;
    fnv1a64(sum, p, n);
    return true;
  }
};

// device array -> file through a host bounce buffer
Status put_dev(Writer& w, const double* d, long long n) {
  std::vector<double> hbuf((size_t)n);
  if (n && cudaMemcpy(hbuf.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return {SGDG_ECUDA, "checkpoint: device-to-host copy"};
  if (!w.put(hbuf.data(), sizeof(double) * n)) return {SGDG_EIO, "checkpoint: write failed"};
  return {};
}

// the whole content of a checkpoint file, parsed and checked on the host
struct Content {
  unsigned long long hash = 0;
  long long nc = 0, ns = 0;
  int flags[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double t_now = 0.0;
  std::vector<double> rhs, u_sol, U_end, u_prev2, guess;
  int field_head[4] = {0, 0, 0, 0};
  std::vector<std::vector<double>> E;
  std::vector<double> rho, phi;
};

// sizes in a header are checked against what the file can hold before any
// buffer is sized from them
Status parse(const char* path, Content& c) {
  File F(std::fopen(path, "rb"));
  if (!F.f) return {SGDG_EIO, std::string("cannot open ") + path};
  if (std::fseek(F.f, 0, SEEK_END) != 0) return {SGDG_EIO, "cannot seek"};
  const long long fsize = std::ftell(F.f);
  std::rewind(F.f);
  Reader r{F.f};
  char magic[8];
  if (!r.get(magic, 8) || std::memcmp(magic, kMagic, 8) != 0) return {SGDG_EIO, "not a checkpoint file"};
  if (!r.get(&c.hash, 8) || !r.get(&c.nc, 8) || !r.get(&c.ns, 8) || !r.get(c.flags, sizeof(c.flags)) ||
      !r.get(&c.t_now, 8))
    return {SGDG_EIO, "file ends early"};
  const long long nvec = 2 + (c.flags[5] ? 1 : 0) + (c.flags[6] ? 1 : 0);
  if (c.nc < 0 || c.ns < 0 || c.nc > fsize / 8 || c.ns > fsize / 8 || nvec * c.nc + c.ns > fsize / 8)
    return {SGDG_EIO, "sizes in the header exceed the file"};
  auto vec = [&](std::vector<double>& v, long long n) {
    v.resize((size_t)n);
    return r.get(v.data(), sizeof(double) * (size_t)n);
  };
  if (!vec(c.rhs, c.nc) || !vec(c.u_sol, c.nc) || !vec(c.U_end, c.ns)) return {SGDG_EIO, "file ends early"};
  if (c.flags[5] && !vec(c.u_prev2, c.nc)) return {SGDG_EIO, "file ends early"};
  if (c.flags[6] && !vec(c.guess, c.nc)) return {SGDG_EIO, "file ends early"};
  if (c.flags[7]) {
    int* hd = c.field_head;
    if (!r.get(hd, sizeof(c.field_head))) return {SGDG_EIO, "file ends early"};
    if (hd[0] < 1 || hd[0] > kMaxDim || hd[1] < 0 || hd[2] < 0 ||
        (long long)hd[0] * hd[1] + 2LL * hd[2] > fsize / 8)
      return {SGDG_EIO, "field sizes in the file are invalid"};
    c.E.assign(hd[0], {});
    for (auto& e : c.E)
      if (!vec(e, hd[1])) return {SGDG_EIO, "file ends early"};
    if (!vec(c.rho, hd[2]) || !vec(c.phi, hd[2])) return {SGDG_EIO, "file ends early"};
  }
  const unsigned long long sum = r.sum;
  unsigned long long stored = 0;
  if (std::fread(&stored, 1, 8, F.f) != 8) return {SGDG_EIO, "file ends early (no checksum)"};
  if (stored != sum) return {SGDG_EIO, "checksum mismatch: the file is corrupted"};
  char extra;
  if (std::fread(&extra, 1, 1, F.f) != 0) return {SGDG_EIO, "bytes after the checksum"};
  return {};
}

Status upload(const double* src, double* d, long long n) {
  if (n && cudaMemcpy(d, src, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return {SGDG_ECUDA, "restore: host-to-device copy"};
  return {};
}

Status checkpoint(Handle& h, const char* path) {
  if (!h.have_initial) return {SGDG_EINVAL, "checkpoint: sgdg_set_initial was not called"};
  if (cudaSetDevice(h.cfg.device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return {SGDG_ECUDA, "checkpoint: synchronise"};
  File F(std::fopen(path, "wb"));
  if (!F.f) return {SGDG_EIO, std::string("checkpoint: cannot open ") + path};
  Writer w{F.f};
  const long long nc = h.n_coeffs, ns = h.n_spatial;
  const int flags[8] = {h.have_initial ? 1 : 0, h.first_strip ? 1 : 0, h.solved ? 1 : 0, h.nsolved, h.warm,
                        h.u_prev2 ? 1 : 0, h.guess ? 1 : 0, h.field ? 1 : 0};
  if (!w.put(kMagic, 8) || !w.put(&h.problem_hash, 8) || !w.put(&nc, 8) || !w.put(&ns, 8) ||
      !w.put(flags, sizeof(flags)) || !w.put(&h.t_now, 8))
    return {SGDG_EIO, "checkpoint: write failed"};
  Status st = put_dev(w, h.rhs, nc);
  if (!st.code) st = put_dev(w, h.u_sol, nc);
  if (!st.code) st = put_dev(w, h.U_end, ns);
  if (!st.code && h.u_prev2) st = put_dev(w, h.u_prev2, nc);
  if (!st.code && h.guess) st = put_dev(w, h.guess, nc);
  if (st.code) return st;
  if (h.field) {
    const Handle::Field& Fd = *h.field;
    const int head[4] = {h.d, (int)(Fd.E.empty() ? 0 : Fd.E[0].size()), (int)Fd.rho0.size(), Fd.updated ? 1 : 0};
    if (!w.put(head, sizeof(head))) return {SGDG_EIO, "checkpoint: write failed"};
    for (const auto& e : Fd.E)
      if (!w.put(e.data(), sizeof(double) * e.size())) return {SGDG_EIO, "checkpoint: write failed"};
    std::vector<double> rho = Fd.rho, phi = Fd.phi;
    rho.resize(head[2], 0.0);
    phi.resize(head[2], 0.0);
    if (!w.put(rho.data(), sizeof(double) * rho.size()) || !w.put(phi.data(), sizeof(double) * phi.size()))
      return {SGDG_EIO, "checkpoint: write failed"};
  }
  const unsigned long long sum = w.sum;
  if (std::fwrite(&sum, 1, 8, F.f) != 8) return {SGDG_EIO, "checkpoint: write failed"};
  if (std::fflush(F.f) != 0) return {SGDG_EIO, "checkpoint: flush failed"};
  return {};
}

Status restore(Handle& h, const char* path) {
  if (cudaSetDevice(h.cfg.device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return {SGDG_ECUDA, "restore: synchronise"};
  Content c;
  {
    Status st = parse(path, c);
    if (st.code) return {st.code, "restore: " + st.msg};
  }
  if (c.hash != h.problem_hash || c.nc != h.n_coeffs || c.ns != h.n_spatial)
    return {SGDG_EINVAL, "restore: the checkpoint belongs to a different problem"};
  if ((c.flags[7] != 0) != (h.field != nullptr))
    return {SGDG_EINVAL, "restore: Vlasov-Poisson state does not match the handle"};
  if (h.field) {
    const Handle::Field& Fd = *h.field;
    const int* hd = c.field_head;
    if (hd[0] != h.d || Fd.E.size() != (size_t)h.d || hd[1] != (int)Fd.E[0].size() ||
        hd[2] != (int)Fd.rho0.size())
      return {SGDG_EINVAL, "restore: field sizes differ from the handle's"};
    if (!hd[3] && Fd.updated)
      return {SGDG_EINVAL, "restore: the checkpoint predates any field update; restore it into a fresh handle"};
  }
  // everything is checked: from here on the handle takes the file's state
  const long long nc = c.nc, ns = c.ns;
  if (c.flags[5] && !h.u_prev2 && dev_alloc(h, (void**)&h.u_prev2, sizeof(double) * nc) != cudaSuccess)
    return {SGDG_ENOMEM, "restore: previous solution buffer"};
  if (c.flags[6] && !h.guess && dev_alloc(h, (void**)&h.guess, sizeof(double) * nc) != cudaSuccess)
    return {SGDG_ENOMEM, "restore: guess buffer"};
  Status st = upload(c.rhs.data(), h.rhs, nc);
  if (!st.code) st = upload(c.u_sol.data(), h.u_sol, nc);
  if (!st.code) st = upload(c.U_end.data(), h.U_end, ns);
  if (!st.code && c.flags[5]) st = upload(c.u_prev2.data(), h.u_prev2, nc);
  if (!st.code && c.flags[6]) st = upload(c.guess.data(), h.guess, nc);
  if (st.code) return st;
  if (h.field) {
    Handle::Field& Fd = *h.field;
    for (int i = 0; i < h.d; ++i) Fd.E[i].swap(c.E[i]);   // in place: the cell-field table points at these vectors
    Fd.rho.swap(c.rho);
    Fd.phi.swap(c.phi);
    Fd.updated = c.field_head[3] != 0;
    if (Fd.updated) {
      st = field_reassemble(h);
      if (st.code) return st;
    }
  }
  h.have_initial = c.flags[0] != 0;
  h.first_strip = c.flags[1] != 0;
  h.solved = c.flags[2] != 0;
  h.nsolved = c.flags[3];
  h.warm = c.flags[4];
  h.t_now = c.t_now;
  st = set_strip_time(h, c.t_now);   // time factors: the couplings of the next strip
  if (st.code) return st;
  if (cudaDeviceSynchronize() != cudaSuccess) return {SGDG_ECUDA, "restore: synchronise"};
  return {};
}

}  // namespace

}  // namespace sgdg

using namespace sgdg;

extern "C" {

sgdg_status sgdg_checkpoint(void* hp, const char* path) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (!path) {
    h->err = "checkpoint: null path";
    return SGDG_EINVAL;
  }
  Status st = checkpoint(*h, path);
  if (st.code) h->err = st.msg;
  return st.code;
}

sgdg_status sgdg_checkpoint_verify(const char* path, sgdg_checkpoint_info* info) {
  if (!path) return SGDG_EINVAL;
  Content c;
  Status st = parse(path, c);
  if (st.code) return st.code;
  if (info) {
    info->problem_hash = c.hash;
    info->n_coeffs = c.nc;
    info->n_spatial = c.ns;
    info->t_now = c.t_now;
    info->strips_solved = c.flags[3];
    info->has_field = c.flags[7];
  }
  return SGDG_OK;
}

sgdg_status sgdg_restore(void* hp, const char* path) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (!path) {
    h->err = "restore: null path";
    return SGDG_EINVAL;
  }
  Status st = restore(*h, path);
  if (st.code) h->err = st.msg;
  return st.code;
}

}  // extern "C"
