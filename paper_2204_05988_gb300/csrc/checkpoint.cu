// Checkpoint and restore of a handle's strip state at a strip boundary
// (sgdg_checkpoint / sgdg_restore).
//
// The strip scheme of Sect. 2 carries U^-_j from one strip to the next; the
// library also carries the last two strip solutions (warm starts), the next
// right-hand side, the start time of the next strip and, for Vlasov-Poisson
// handles, the field E per finest cell (Sect. 5.3).  A checkpoint holds all
// of it in FP64, so a restored handle continues exactly where the writer
// stopped.  Layout (native endianness, no padding):
//   "SGDGCKP1" | u64 problem hash | i64 n_coeffs | i64 n_spatial
//   | i32 flags[8] = {have_initial, first_strip, solved, nsolved, warm,
//                     has_prev2, has_guess, has_field}
//   | f64 t_now | rhs[n_coeffs] | u_sol[n_coeffs] | U_end[n_spatial]
//   | u_prev2[n_coeffs] if has_prev2 | guess[n_coeffs] if has_guess
//   | if has_field: i32 d, i32 ncells, i32 nverts, i32 updated,
//                   E[d][ncells], rho[nverts], phi[nverts]
#include <cstdio>
#include <cstring>
#include <memory>

#include "handle.h"

namespace sgdg {

namespace {

constexpr char kMagic[8] = {'S', 'G', 'D', 'G', 'C', 'K', 'P', '1'};

struct File {
  std::FILE* f = nullptr;
  explicit File(std::FILE* ff) : f(ff) {}
  ~File() { if (f) std::fclose(f); }
};

bool put(std::FILE* f, const void* p, size_t n) { return std::fwrite(p, 1, n, f) == n; }
bool get(std::FILE* f, void* p, size_t n) { return std::fread(p, 1, n, f) == n; }

// device array -> file through a host bounce buffer
Status put_dev(std::FILE* f, const double* d, long long n) {
  std::vector<double> hbuf((size_t)n);
  if (n && cudaMemcpy(hbuf.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return {SGDG_ECUDA, "checkpoint: device-to-host copy"};
  if (!put(f, hbuf.data(), sizeof(double) * n)) return {SGDG_EIO, "checkpoint: write failed"};
  return {};
}

Status get_dev(std::FILE* f, double* d, long long n) {
  std::vector<double> hbuf((size_t)n);
  if (!get(f, hbuf.data(), sizeof(double) * n)) return {SGDG_EIO, "restore: file ends early"};
  if (n && cudaMemcpy(d, hbuf.data(), sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return {SGDG_ECUDA, "restore: host-to-device copy"};
  return {};
}

Status checkpoint(Handle& h, const char* path) {
  if (!h.have_initial) return {SGDG_EINVAL, "checkpoint: sgdg_set_initial was not called"};
  if (cudaSetDevice(h.cfg.device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return {SGDG_ECUDA, "checkpoint: synchronise"};
  File F(std::fopen(path, "wb"));
  if (!F.f) return {SGDG_EIO, std::string("checkpoint: cannot open ") + path};
  const long long nc = h.n_coeffs, ns = h.n_spatial;
  const int flags[8] = {h.have_initial ? 1 : 0, h.first_strip ? 1 : 0, h.solved ? 1 : 0, h.nsolved, h.warm,
                        h.u_prev2 ? 1 : 0, h.guess ? 1 : 0, h.field ? 1 : 0};
  if (!put(F.f, kMagic, 8) || !put(F.f, &h.problem_hash, 8) || !put(F.f, &nc, 8) || !put(F.f, &ns, 8) ||
      !put(F.f, flags, sizeof(flags)) || !put(F.f, &h.t_now, 8))
    return {SGDG_EIO, "checkpoint: write failed"};
  Status st = put_dev(F.f, h.rhs, nc);
  if (!st.code) st = put_dev(F.f, h.u_sol, nc);
  if (!st.code) st = put_dev(F.f, h.U_end, ns);
  if (!st.code && h.u_prev2) st = put_dev(F.f, h.u_prev2, nc);
  if (!st.code && h.guess) st = put_dev(F.f, h.guess, nc);
  if (st.code) return st;
  if (h.field) {
    const Handle::Field& Fd = *h.field;
    const int head[4] = {h.d, (int)(Fd.E.empty() ? 0 : Fd.E[0].size()), (int)Fd.rho0.size(), Fd.updated ? 1 : 0};
    if (!put(F.f, head, sizeof(head))) return {SGDG_EIO, "checkpoint: write failed"};
    for (const auto& e : Fd.E)
      if (!put(F.f, e.data(), sizeof(double) * e.size())) return {SGDG_EIO, "checkpoint: write failed"};
    std::vector<double> rho = Fd.rho, phi = Fd.phi;
    rho.resize(head[2], 0.0);
    phi.resize(head[2], 0.0);
    if (!put(F.f, rho.data(), sizeof(double) * rho.size()) || !put(F.f, phi.data(), sizeof(double) * phi.size()))
      return {SGDG_EIO, "checkpoint: write failed"};
  }
  if (std::fflush(F.f) != 0) return {SGDG_EIO, "checkpoint: flush failed"};
  return {};
}

Status restore(Handle& h, const char* path) {
  if (cudaSetDevice(h.cfg.device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return {SGDG_ECUDA, "restore: synchronise"};
  File F(std::fopen(path, "rb"));
  if (!F.f) return {SGDG_EIO, std::string("restore: cannot open ") + path};
  char magic[8];
  unsigned long long hash = 0;
  long long nc = 0, ns = 0;
  int flags[8];
  double t_now = 0.0;
  if (!get(F.f, magic, 8) || std::memcmp(magic, kMagic, 8) != 0) return {SGDG_EIO, "restore: not a checkpoint file"};
  if (!get(F.f, &hash, 8) || !get(F.f, &nc, 8) || !get(F.f, &ns, 8) || !get(F.f, flags, sizeof(flags)) ||
      !get(F.f, &t_now, 8))
    return {SGDG_EIO, "restore: file ends early"};
  if (hash != h.problem_hash || nc != h.n_coeffs || ns != h.n_spatial)
    return {SGDG_EINVAL, "restore: the checkpoint belongs to a different problem"};
  if ((flags[7] != 0) != (h.field != nullptr))
    return {SGDG_EINVAL, "restore: Vlasov-Poisson state does not match the handle"};
  // buffers the state needs
  if (flags[5] && !h.u_prev2 && dev_alloc(h, (void**)&h.u_prev2, sizeof(double) * nc) != cudaSuccess)
    return {SGDG_ENOMEM, "restore: previous solution buffer"};
  if (flags[6] && !h.guess && dev_alloc(h, (void**)&h.guess, sizeof(double) * nc) != cudaSuccess)
    return {SGDG_ENOMEM, "restore: guess buffer"};
  Status st = get_dev(F.f, h.rhs, nc);
  if (!st.code) st = get_dev(F.f, h.u_sol, nc);
  if (!st.code) st = get_dev(F.f, h.U_end, ns);
  if (!st.code && flags[5]) st = get_dev(F.f, h.u_prev2, nc);
  if (!st.code && flags[6]) st = get_dev(F.f, h.guess, nc);
  if (st.code) return st;
  if (h.field) {
    Handle::Field& Fd = *h.field;
    int head[4];
    if (!get(F.f, head, sizeof(head))) return {SGDG_EIO, "restore: file ends early"};
    if (head[0] != h.d || Fd.E.size() != (size_t)h.d || head[1] != (int)Fd.E[0].size() ||
        head[2] != (int)Fd.rho0.size())
      return {SGDG_EINVAL, "restore: field sizes differ from the handle's"};
    if (!head[3] && Fd.updated)
      return {SGDG_EINVAL, "restore: the checkpoint predates any field update; restore it into a fresh handle"};
    std::vector<std::vector<double>> E(h.d, std::vector<double>(head[1]));
    std::vector<double> rho(head[2]), phi(head[2]);
    for (auto& e : E)
      if (!get(F.f, e.data(), sizeof(double) * e.size())) return {SGDG_EIO, "restore: file ends early"};
    if (!get(F.f, rho.data(), sizeof(double) * rho.size()) || !get(F.f, phi.data(), sizeof(double) * phi.size()))
      return {SGDG_EIO, "restore: file ends early"};
    for (int i = 0; i < h.d; ++i) Fd.E[i].swap(E[i]);   // in place: the cell-field table points at these vectors
    Fd.rho.swap(rho);
    Fd.phi.swap(phi);
    Fd.updated = head[3] != 0;
    if (Fd.updated) {
      st = field_reassemble(h);
      if (st.code) return st;
    }
  }
  h.have_initial = flags[0] != 0;
  h.first_strip = flags[1] != 0;
  h.solved = flags[2] != 0;
  h.nsolved = flags[3];
  h.warm = flags[4];
  h.t_now = t_now;
  {
    Status st = set_strip_time(h, t_now);   // time factors: the couplings of the next strip
    if (st.code) return st;
  }
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
