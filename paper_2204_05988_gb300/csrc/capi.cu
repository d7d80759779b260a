// C ABI of the sgdg library: set-up (hierarchies, FP64 assembly, term table,
// device upload) and the entry points declared in include/sgdg.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>

#include "handle.h"
#include "sweep.h"

namespace sgdg {

static std::mutex& registry_mutex() {
  static std::mutex m;
  return m;
}

// callers hold registry_mutex()
static std::vector<void*>& registry(Handle* h) {
  static std::map<Handle*, std::vector<void*>> reg;
  return reg[h];
}

// Every device allocation of a handle goes through here and is released in
// sgdg_destroy.  Batch members allocate lazily from their own host threads.
cudaError_t dev_alloc(Handle& h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  {
    std::lock_guard<std::mutex> lk(registry_mutex());
    if (h.budget && h.device_bytes + bytes > h.budget) return cudaErrorMemoryAllocation;   // over hbm_budget_bytes
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(registry_mutex());
    h.device_bytes += bytes;
    registry(&h).push_back(*p);
  }
  return e;
}

namespace {

#define SG_CU(x)                                                              \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) return {SGDG_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
#define SG_ST(x)                   \
  do {                             \
    Status s_ = (x);               \
    if (s_.code) return s_;        \
  } while (0)

template <typename T>
Status upload(Handle& h, T** dst, const T* src, size_t n) {
  if (dev_alloc(h, (void**)dst, sizeof(T) * n) != cudaSuccess) return {SGDG_ENOMEM, "device upload"};
  SG_CU(cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice));
  return {};
}

Status upload_vals(Handle& h, const std::vector<double>& v, double** d64, float** d32) {
  SG_ST(upload(h, d64, v.data(), v.size()));
  std::vector<float> f(v.begin(), v.end());
  SG_ST(upload(h, d32, f.data(), f.size()));
  return {};
}

}  // namespace

std::vector<int> ell_columns(const std::vector<int>& rowptr, const std::vector<int>& col, int w) {
  const int n = (int)rowptr.size() - 1;
  std::vector<int> out((size_t)n * w, 0);
  for (int r = 0; r < n; ++r) {
    const int b = rowptr[r], len = rowptr[r + 1] - b;
    for (int j = 0; j < w; ++j) out[(size_t)r * w + j] = len == 0 ? 0 : col[b + (j < len ? j : 0)];
  }
  return out;
}

std::vector<double> ell_values(const std::vector<int>& rowptr, const std::vector<double>& val, int w) {
  const int n = (int)rowptr.size() - 1;
  std::vector<double> out((size_t)n * w, 0.0);
  for (int r = 0; r < n; ++r) {
    const int b = rowptr[r], len = rowptr[r + 1] - b;
    for (int j = 0; j < len && j < w; ++j) out[(size_t)r * w + j] = val[b + j];
  }
  return out;
}

namespace {

// Stencil-slot offsets (dx, dy) of a 2-D lattice whose cells are cut along
// the (1, 1) diagonal, in the order of their lexicographic index offsets.
constexpr int kLatSlots = 7;
constexpr int kLatDx[kLatSlots] = {-1, 0, -1, 0, 1, 0, 1};
constexpr int kLatDy[kLatSlots] = {-1, -1, 0, 0, 0, 1, 1};

// The slot map of a level when it is such a lattice (empty otherwise).
std::vector<int> lattice_slots(const MeshLevel& lv, int d, int w, int* nx_out) {
  *nx_out = 0;
  if (d != 2 || w < 8 || lv.n < 4) return {};
  const Csr& P = lv.pattern;
  const double y0 = lv.coords[1];
  int nx = 0;
  while (nx < lv.n && lv.coords[2 * nx + 1] == y0) ++nx;
  if (nx < 2 || lv.n % nx) return {};
  const int ny = lv.n / nx;
  for (int k = 0; k < lv.n; ++k)
    if (lv.coords[2 * k] != lv.coords[2 * (k % nx)] || lv.coords[2 * k + 1] != lv.coords[2 * (k / nx * nx) + 1])
      return {};
  std::vector<int> pos((size_t)lv.n * w, -1);
  for (int k = 0; k < lv.n; ++k) {
    const int ix = k % nx, iy = k / nx;
    for (int p = P.rowptr[k]; p < P.rowptr[k + 1]; ++p) {
      const int c = P.col[p], dx = c % nx - ix, dy = c / nx - iy;
      int slot = -1;
      for (int q = 0; q < kLatSlots; ++q)
        if (kLatDx[q] == dx && kLatDy[q] == dy) slot = q;
      if (slot < 0) return {};
      pos[(size_t)k * w + slot] = p;
    }
    (void)ny;
  }
  *nx_out = nx;
  return pos;
}

}  // namespace

std::vector<int> pattern_ell_columns(const SideDev& sd, const Csr& P, int l) {
  const int w = sd.ell_w();
  if (l >= (int)sd.lat_nx.size() || !sd.lat_nx[l]) return ell_columns(P.rowptr, P.col, w);
  const std::vector<int>& pos = sd.lat_pos[l];
  std::vector<int> out((size_t)P.nrows * w);
  for (int r = 0; r < P.nrows; ++r)
    for (int s = 0; s < w; ++s) {
      const int p = pos[(size_t)r * w + s];
      out[(size_t)r * w + s] = p >= 0 ? P.col[p] : r;
    }
  return out;
}

Status upload_pattern_vals(Handle& h, const SideDev& sd, const Csr& P, int l, const std::vector<double>& val,
                           double** d64, float** d32) {
  const int w = sd.ell_w();
  if (l >= (int)sd.lat_nx.size() || !sd.lat_nx[l]) return upload_ell_vals(h, P.rowptr, val, w, d64, d32);
  const std::vector<int>& pos = sd.lat_pos[l];
  std::vector<double> e(pos.size(), 0.0);
  for (size_t i = 0; i < pos.size(); ++i)
    if (pos[i] >= 0) e[i] = val[pos[i]];
  const std::vector<float> f(e.begin(), e.end());
  if (!*d64) {
    SG_ST(upload(h, d64, e.data(), e.size()));
    SG_ST(upload(h, d32, f.data(), f.size()));
  } else {
    SG_CU(cudaMemcpy(*d64, e.data(), sizeof(double) * e.size(), cudaMemcpyHostToDevice));
    SG_CU(cudaMemcpy(*d32, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
  }
  return {};
}

Status upload_ell_vals(Handle& h, const std::vector<int>& rowptr, const std::vector<double>& val, int w,
                       double** d64, float** d32) {
  const std::vector<double> e = ell_values(rowptr, val, w);
  const std::vector<float> f(e.begin(), e.end());
  if (!*d64) {
    SG_ST(upload(h, d64, e.data(), e.size()));
    SG_ST(upload(h, d32, f.data(), f.size()));
  } else {
    SG_CU(cudaMemcpy(*d64, e.data(), sizeof(double) * e.size(), cudaMemcpyHostToDevice));
    SG_CU(cudaMemcpy(*d32, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
  }
  return {};
}

void factor_products(const Hierarchy& hi, const SideDev& sd, const std::vector<Csr>& X, FactorProducts& out) {
  const int L = hi.L;
  out.rf.assign(L, {});
  out.fp.assign(L + 1, {});
  for (int l = 0; l < L && sd.has_rf; ++l)
    product_values(hi.Rt[l], hi.Rt[l].val, X[l + 1], X[l + 1].val, sd.RF_pat[l], out.rf[l]);
  for (int l = 1; l <= L && sd.has_fp; ++l)
    product_values(X[l], X[l].val, hi.E[l - 1], hi.E[l - 1].val, sd.FP_pat[l], out.fp[l]);
}

Status upload_products(Handle& h, SideDev& sd, int f, const FactorProducts& pr) {
  for (int l = 0; l < (int)pr.rf.size() && sd.has_rf; ++l)
    SG_ST(upload_ell_vals(h, sd.RF_pat[l].rowptr, pr.rf[l], sd.rf_w(), &sd.v64.ell_RF[f][l], &sd.v32.ell_RF[f][l]));
  for (int l = 1; l < (int)pr.fp.size() && sd.has_fp; ++l)
    SG_ST(upload_ell_vals(h, sd.FP_pat[l].rowptr, pr.fp[l], sd.fp_w(), &sd.v64.ell_FP[f][l], &sd.v32.ell_FP[f][l]));
  return {};
}

Status upload_factor_products(Handle& h, const Hierarchy& hi, SideDev& sd, int f, const std::vector<Csr>& X) {
  FactorProducts pr;
  factor_products(hi, sd, X, pr);
  return upload_products(h, sd, f, pr);
}

namespace {

// Patterns of the factor-transfer products R_l F_{l+1} (with_rf) and
// F_l E_{l-1} (with_fp), shared by every factor of the side, in ELL form.
Status setup_products(Handle& h, const Hierarchy& hi, SideDev& sd, bool with_rf, bool with_fp) {
  const int L = hi.L;
  sd.has_rf = with_rf;
  sd.has_fp = with_fp;
  sd.RF_pat.assign(L, Csr());
  sd.FP_pat.assign(L + 1, Csr());
  sd.rf_row = sd.fp_row = 0;
  for (int l = 0; l < L && with_rf; ++l) {
    sd.RF_pat[l] = product_pattern(hi.Rt[l], hi.lev[l + 1].pattern);
    for (int r = 0; r < sd.RF_pat[l].nrows; ++r)
      sd.rf_row = std::max(sd.rf_row, sd.RF_pat[l].rowptr[r + 1] - sd.RF_pat[l].rowptr[r]);
  }
  for (int l = 1; l <= L && with_fp; ++l) {
    sd.FP_pat[l] = product_pattern(hi.lev[l].pattern, hi.E[l - 1]);
    for (int r = 0; r < sd.FP_pat[l].nrows; ++r)
      sd.fp_row = std::max(sd.fp_row, sd.FP_pat[l].rowptr[r + 1] - sd.FP_pat[l].rowptr[r]);
  }
  if (sd.rf_row > kMaxChainRow) return {SGDG_EINVAL, "restriction-factor product rows longer than 24 entries"};
  if (sd.fp_row > kMaxFinalRow) return {SGDG_EINVAL, "factor-prolongation product rows longer than 16 entries"};
  sd.rf_row = std::max(sd.rf_row, 1);
  sd.fp_row = std::max(sd.fp_row, 1);
  sd.RF_ell_col.assign(L, nullptr);
  sd.FP_ell_col.assign(L + 1, nullptr);
  for (int l = 0; l < L && with_rf; ++l) {
    const std::vector<int> c = ell_columns(sd.RF_pat[l].rowptr, sd.RF_pat[l].col, sd.rf_w());
    SG_ST(upload(h, &sd.RF_ell_col[l], c.data(), c.size()));
  }
  for (int l = 1; l <= L && with_fp; ++l) {
    const std::vector<int> c = ell_columns(sd.FP_pat[l].rowptr, sd.FP_pat[l].col, sd.fp_w());
    SG_ST(upload(h, &sd.FP_ell_col[l], c.data(), c.size()));
  }
  return {};
}

Status upload_side(Handle& h, const Hierarchy& hi, SideDev& sd) {
  const int L = hi.L;
  sd.n.resize(L + 1);
  sd.nnz.resize(L + 1);
  sd.rowptr.resize(L + 1);
  sd.col.resize(L + 1);
  const int w = sd.ell_w();
  sd.ell_col.resize(L + 1);
  sd.lat_nx.assign(L + 1, 0);
  sd.lat_pos.assign(L + 1, {});
  for (int l = 0; l <= L; ++l) {
    const Csr& P = hi.lev[l].pattern;
    sd.n[l] = P.nrows;
    sd.nnz[l] = P.nnz();
    SG_ST(upload(h, &sd.rowptr[l], P.rowptr.data(), P.rowptr.size()));
    SG_ST(upload(h, &sd.col[l], P.col.data(), P.col.size()));
    if (sd.lattice_ok) sd.lat_pos[l] = lattice_slots(hi.lev[l], hi.d, w, &sd.lat_nx[l]);
    const std::vector<int> ec = pattern_ell_columns(sd, P, l);
    SG_ST(upload(h, &sd.ell_col[l], ec.data(), ec.size()));
  }
  sd.lat_E.assign(L + 1, 0);
  for (int l = 1; l <= L; ++l) {
    const int nx = sd.lat_nx[l], nxc = sd.lat_nx[l - 1];
    if (!nx || !nxc || nxc != (nx + 1) / 2 || (hi.lev[l].n / nx + 1) / 2 != hi.lev[l - 1].n / nxc) continue;
    const Csr& E = hi.E[l - 1];
    bool ok = true;
    for (int k = 0; k < E.nrows && ok; ++k) {
      const int ix = k % nx, iy = k / nx;
      int want[2], nw = 0;
      if (!(ix & 1) && !(iy & 1)) want[nw++] = (iy / 2) * nxc + ix / 2;
      else if (!(iy & 1)) { want[nw++] = (iy / 2) * nxc + (ix - 1) / 2; want[nw++] = (iy / 2) * nxc + (ix + 1) / 2; }
      else if (!(ix & 1)) { want[nw++] = (iy - 1) / 2 * nxc + ix / 2; want[nw++] = (iy + 1) / 2 * nxc + ix / 2; }
      else { want[nw++] = (iy - 1) / 2 * nxc + (ix - 1) / 2; want[nw++] = (iy + 1) / 2 * nxc + (ix + 1) / 2; }
      const int len = E.rowptr[k + 1] - E.rowptr[k];
      if (len != nw) ok = false;
      for (int p = 0; p < len && ok; ++p)
        ok = E.col[E.rowptr[k] + p] == want[p] && E.val[E.rowptr[k] + p] == (nw == 1 ? 1.0 : 0.5);
    }
    sd.lat_E[l] = ok ? 1 : 0;
  }
  sd.E_rowptr.resize(L); sd.E_col.resize(L); sd.R_rowptr.resize(L); sd.R_col.resize(L); sd.inj.resize(L);
  sd.E_nnz.resize(L); sd.R_nnz.resize(L);
  sd.v64.E.resize(L); sd.v64.R.resize(L); sd.v32.E.resize(L); sd.v32.R.resize(L);
  sd.E_ell_col.resize(L); sd.R_ell_col.resize(L);
  sd.v64.ell_E.assign(L, nullptr); sd.v64.ell_R.assign(L, nullptr);
  sd.v32.ell_E.assign(L, nullptr); sd.v32.ell_R.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    const Csr& E = hi.E[l];
    const Csr& R = hi.Rt[l];
    sd.E_nnz[l] = E.nnz();
    sd.R_nnz[l] = R.nnz();
    SG_ST(upload(h, &sd.E_rowptr[l], E.rowptr.data(), E.rowptr.size()));
    SG_ST(upload(h, &sd.E_col[l], E.col.data(), E.col.size()));
    SG_ST(upload_vals(h, E.val, &sd.v64.E[l], &sd.v32.E[l]));
    SG_ST(upload(h, &sd.R_rowptr[l], R.rowptr.data(), R.rowptr.size()));
    SG_ST(upload(h, &sd.R_col[l], R.col.data(), R.col.size()));
    SG_ST(upload_vals(h, R.val, &sd.v64.R[l], &sd.v32.R[l]));
    const std::vector<int> eec = ell_columns(E.rowptr, E.col, kEllE);
    SG_ST(upload(h, &sd.E_ell_col[l], eec.data(), eec.size()));
    SG_ST(upload_ell_vals(h, E.rowptr, E.val, kEllE, &sd.v64.ell_E[l], &sd.v32.ell_E[l]));
    const std::vector<int> erc = ell_columns(R.rowptr, R.col, w);
    SG_ST(upload(h, &sd.R_ell_col[l], erc.data(), erc.size()));
    SG_ST(upload_ell_vals(h, R.rowptr, R.val, w, &sd.v64.ell_R[l], &sd.v32.ell_R[l]));
    SG_ST(upload(h, &sd.inj[l], hi.inj[l].data(), hi.inj[l].size()));
  }
  return {};
}

std::vector<Chain> make_chains(const std::vector<Term>& terms, bool by_v) {
  std::map<int, int> idx;
  std::vector<Chain> out;
  for (int t = 0; t < (int)terms.size(); ++t) {
    int key = by_v ? terms[t].v : terms[t].x;
    auto it = idx.find(key);
    if (it == idx.end()) {
      it = idx.emplace(key, (int)out.size()).first;
      Chain c;
      c.first = key;
      c.by_v = by_v;
      out.push_back(c);
    }
    out[it->second].terms.push_back(t);
  }
  return out;
}

void make_plan(Plan& p, const std::vector<Term>& terms) {
  p.terms = terms;
  std::vector<Chain> cv = make_chains(terms, true), cx = make_chains(terms, false);
  // the sweep applies V first in branch A and X first in branch B
  p.A = cv;
  p.B = cx;
  p.D = cv.size() <= cx.size() ? cv : cx;
}

// the problem identity of checkpoints: FNV-1a 64 over raw bytes
void fnv(unsigned long long& hsh, const void* p, size_t n) { fnv1a64(hsh, p, n); }

struct ErrStore {
  std::string msg;
};
ErrStore& global_err() {
  static ErrStore e;
  return e;
}

sgdg_status fail(Handle* h, const Status& st) {
  if (h) h->err = st.msg;
  global_err().msg = st.msg;
  return st.code;
}

Status create(const sgdg_config& cfg, const sgdg_coeffs& c, Handle& h) {
  if (cfg.mesh_x.dim != cfg.mesh_v.dim) return {SGDG_EINVAL, "mesh_x and mesh_v must have the same dimension"};
  if (cfg.mesh_x.dim < 1 || cfg.mesh_x.dim > kMaxDim) return {SGDG_EINVAL, "dimension must be 1, 2 or 3"};
  if (cfg.level_L < 0 || cfg.level_L >= kMaxLevels) return {SGDG_EINVAL, "level_L out of range 0..11"};
  if (2 * cfg.level_L + 2 > kMaxGrids) return {SGDG_EINVAL, "too many grids"};
  if (cfg.time_degree != 1) return {SGDG_EINVAL, "only time_degree 1 is supported"};
  if (!(cfg.dt > 0.0) || !(cfg.delta >= 0.0)) return {SGDG_EINVAL, "dt must be > 0 and delta >= 0"};
  if (cfg.precision == SGDG_BF16_STORE)
    return {SGDG_EINVAL, "BF16 storage is an apply precision, not a solver precision"};
  if (cfg.precision != SGDG_FP64 && cfg.precision != SGDG_MIXED_FP32) return {SGDG_EINVAL, "unknown precision"};
  if (cfg.restart < 1 || cfg.restart > 63 || cfg.inner_its < 1 || cfg.inner_its > 63)
    return {SGDG_EINVAL, "restart and inner_its must be in 1..63"};
  if (cfg.outer_method != SGDG_OUTER_FGMRES && cfg.outer_method != SGDG_OUTER_RICHARDSON)
    return {SGDG_EINVAL, "unknown outer_method"};
  if (c.n_u0 < 0 || (c.n_u0 > 0 && !c.u0)) return {SGDG_EINVAL, "bad u0 list"};
  {
    Status sm = validate_mesh(cfg.mesh_x);
    if (sm.code) return {sm.code, "mesh_x: " + sm.msg};
    sm = validate_mesh(cfg.mesh_v);
    if (sm.code) return {sm.code, "mesh_v: " + sm.msg};
  }
  {
    bool timed = c.sigma_t != nullptr;
    for (int p = 0; p < 2 * cfg.mesh_x.dim && p < 2 * kMaxDim; ++p) timed = timed || c.beta_t[p] != nullptr;
    if (timed && cfg.vlasov_poisson)
      return {SGDG_EINVAL, "time factors of beta or sigma are not combined with vlasov_poisson"};
    if (c.time_quad < 0 || c.time_quad > 8) return {SGDG_EINVAL, "time_quad must be in 0..8"};
  }
  h.cfg = cfg;
  h.d = cfg.mesh_x.dim;
  h.L = cfg.level_L;
  h.budget = cfg.hbm_budget_bytes;
  h.problem_hash = kFnvBasis;
  fnv(h.problem_hash, &h.d, sizeof(h.d));
  fnv(h.problem_hash, &h.L, sizeof(h.L));
  fnv(h.problem_hash, &cfg.dt, sizeof(cfg.dt));
  fnv(h.problem_hash, &cfg.delta, sizeof(cfg.delta));
  SG_CU(cudaSetDevice(cfg.device));
  Hierarchy hx, hv;
  {
    Status sv;   // the two level hierarchies are independent: build them side by side
    std::thread tv([&] { sv = build_hierarchy(cfg.mesh_v, h.L, hv); });
    Status sx = build_hierarchy(cfg.mesh_x, h.L, hx);
    tv.join();
    SG_ST(sx);
    SG_ST(sv);
  }
  SG_ST(build_terms(c, h.d, cfg.mesh_x, cfg.mesh_v, cfg.dt, cfg.delta, h.tt));
  // callback tables: ids 0 .. 2 kMaxDim - 1 beta components, then sigma
  SideFns fx, fv;
  for (int p = 0; p < 2 * kMaxDim; ++p) {
    fx.fn.push_back(p < 2 * h.d ? c.beta[p].fx : nullptr); fx.user.push_back(c.beta[p].ux);
    fv.fn.push_back(p < 2 * h.d ? c.beta[p].fv : nullptr); fv.user.push_back(c.beta[p].uv);
  }
  fx.fn.push_back(c.sigma.fx); fx.user.push_back(c.sigma.ux);
  fv.fn.push_back(c.sigma.fv); fv.user.push_back(c.sigma.uv);
  // make sure the plain mass factor exists on both sides
  FactorSpec mass;
  auto find_or_add = [&](std::vector<FactorSpec>& fs) {
    for (size_t i = 0; i < fs.size(); ++i)
      if (fs[i] == mass) return (int)i;
    fs.push_back(mass);
    return (int)fs.size() - 1;
  };
  h.X.mass = find_or_add(h.tt.xf);
  h.V.mass = find_or_add(h.tt.vf);
  // stiffness factors (d/dy_p, d/dy_p) of both sides for the H^1 Gram plan
  int kx[3] = {0, 0, 0}, kv[3] = {0, 0, 0};
  for (int p = 1; p <= h.d; ++p) {
    mass.test = mass.trial = p;
    kx[p - 1] = find_or_add(h.tt.xf);
    kv[p - 1] = find_or_add(h.tt.vf);
  }
  mass.test = mass.trial = 0;
  // the sweep kernels keep one matrix row of at most 16 entries (prolongation:
  // kProlongRow) in registers
  int side_maxrow[2] = {0, 0};
  for (int side = 0; side < 2; ++side) {
    const Hierarchy* hi = side == 0 ? &hx : &hv;
    auto maxrow = [](const Csr& A) {
      int m = 0;
      for (int i = 0; i < A.nrows; ++i) m = std::max(m, A.rowptr[i + 1] - A.rowptr[i]);
      return m;
    };
    for (const MeshLevel& lv : hi->lev) side_maxrow[side] = std::max(side_maxrow[side], maxrow(lv.pattern));
    for (const Csr& R : hi->Rt) side_maxrow[side] = std::max(side_maxrow[side], maxrow(R));
    if (side_maxrow[side] > 16) return {SGDG_EINVAL, "P1 pattern or restriction rows longer than 16 entries"};
    for (const Csr& E : hi->E)
      if (maxrow(E) > kProlongRow) return {SGDG_EINVAL, "prolongation rows with more than 2 entries"};
  }
  h.X.maxrow = side_maxrow[0];
  h.V.maxrow = side_maxrow[1];
  h.X.lattice_ok = true;   // the x side's dim-1 finals have a lattice kernel
  SG_ST(upload_side(h, hx, h.X));
  SG_ST(upload_side(h, hv, h.V));
  // the sweep uses R X (branch B's chain steps) and V E (branch B's final).
  // On 3D Kuhn lattices R X has rows of 65 entries: branch B then applies X
  // and R one after the other (apply.cu)
  SG_ST(setup_products(h, hx, h.X, h.d < 3, false));
  SG_ST(setup_products(h, hv, h.V, false, true));
  for (int side = 0; side < 2; ++side) {
    SideDev& sd = side == 0 ? h.X : h.V;
    const Hierarchy& hi = side == 0 ? hx : hv;
    const std::vector<FactorSpec>& fs = side == 0 ? h.tt.xf : h.tt.vf;
    const SideFns& fns = side == 0 ? fx : fv;
    sd.v64.ell_fac.assign(fs.size(), std::vector<double*>(h.L + 1, nullptr));
    sd.v32.ell_fac.assign(fs.size(), std::vector<float*>(h.L + 1, nullptr));
    sd.v64.ell_RF.assign(fs.size(), std::vector<double*>(h.L + 1, nullptr));
    sd.v32.ell_RF.assign(fs.size(), std::vector<float*>(h.L + 1, nullptr));
    sd.v64.ell_FP.assign(fs.size(), std::vector<double*>(h.L + 1, nullptr));
    sd.v32.ell_FP.assign(fs.size(), std::vector<float*>(h.L + 1, nullptr));
    for (size_t f = 0; f < fs.size(); ++f)
      for (int id : fs[f].wfn)
        if (!fns.fn[id]) return {SGDG_EINVAL, "factor references a missing coefficient function"};
    // FP64 assembly of every factor of the side on the host: the boundary-face
    // factors one by one, the volume factors together in one pass over the
    // finest cells (each coefficient callback once per quadrature point),
    // then all products with the transfers concurrently, one factor per
    // thread - the values do not depend on the thread count
    const int nf = (int)fs.size();
    std::vector<std::vector<Csr>> Xs(nf);
    std::vector<FactorProducts> Ps(nf);
    std::vector<Status> sts(nf);
    std::vector<FactorSpec> vspec;
    std::vector<int> vidx;
    for (int f = 0; f < nf; ++f) {
      if (fs[f].kind != 0) sts[f] = assemble_factor(hi, fns, fs[f], Xs[f]);
      else { vspec.push_back(fs[f]); vidx.push_back(f); }
    }
    {
      std::vector<std::vector<Csr>> Xv;
      SG_ST(assemble_volume(hi, fns, vspec, Xv));
      for (size_t k = 0; k < vidx.size(); ++k) Xs[vidx[k]] = std::move(Xv[k]);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int f = 0; f < nf; ++f)
      if (!sts[f].code) factor_products(hi, sd, Xs[f], Ps[f]);
    for (int f = 0; f < nf; ++f) SG_ST(sts[f]);
    for (size_t f = 0; f < fs.size(); ++f) {
      std::vector<Csr>& X = Xs[f];
      fnv(h.problem_hash, X[h.L].val.data(), sizeof(double) * X[h.L].val.size());
      fnv(h.problem_hash, X[h.L].col.data(), sizeof(int) * X[h.L].col.size());
      for (int l = 0; l <= h.L; ++l) {
        SG_ST(upload_pattern_vals(h, sd, hi.lev[l].pattern, l, X[l].val, &sd.v64.ell_fac[f][l],
                                  &sd.v32.ell_fac[f][l]));
      }
      SG_ST(upload_products(h, sd, (int)f, Ps[f]));
      if ((int)f == sd.mass) {
        sd.v64.dinv.resize(h.L + 1);
        sd.v32.dinv.resize(h.L + 1);
        for (int l = 0; l <= h.L; ++l) {
          std::vector<double> di(X[l].nrows);
          for (int i = 0; i < X[l].nrows; ++i) {
            double dd = 0.0;
            for (int p = X[l].rowptr[i]; p < X[l].rowptr[i + 1]; ++p)
              if (X[l].col[p] == i) dd = X[l].val[p];
            if (!(dd > 0.0)) return {SGDG_EINVAL, "mass matrix with a non-positive diagonal"};
            di[i] = 1.0 / dd;
          }
          SG_ST(upload_vals(h, di, &sd.v64.dinv[l], &sd.v32.dinv[l]));
        }
      }
      std::vector<Csr>().swap(Xs[f]);
      Ps[f] = FactorProducts();
    }
  }
  // grids, offsets
  const int L = h.L;
  h.n1.resize(L + 1);
  h.n2.resize(L + 1);
  h.off.assign(L + 2, 0);
  h.soff.assign(L + 2, 0);
  for (int l = 0; l <= L; ++l) {
    h.n1[l] = h.X.n[l];
    h.n2[l] = h.V.n[L - l];
    h.soff[l + 1] = h.soff[l] + (long long)h.n1[l] * h.n2[l];
    h.off[l + 1] = 2 * h.soff[l + 1];
  }
  for (int l = 0; l <= L; ++l)
    if ((long long)h.n1[l] * h.n2[l] >= (1LL << 31)) return {SGDG_EINVAL, "component grid with 2^31 or more nodes"};
  h.n_spatial = h.soff[L + 1];
  h.n_coeffs = h.off[L + 1];
  if (cfg.vlasov_poisson) SG_ST(field_setup(h, c, hx, hv, fx));
  long long tmp = 2;
  for (int i = 1; i <= L; ++i) tmp = std::max(tmp, 2LL * h.X.n[i - 1] * h.V.n[L - i]);
  for (int i = 0; i < L; ++i) tmp = std::max(tmp, 2LL * h.X.n[i + 1] * h.V.n[L - i]);
  h.tmp_elems = tmp;
  for (const Term& t : h.tt.terms) {
    fnv(h.problem_hash, t.tau, sizeof(t.tau));
    fnv(h.problem_hash, &t.x, sizeof(t.x));
    fnv(h.problem_hash, &t.v, sizeof(t.v));
  }
  make_plan(h.op, h.tt.terms);
  // time factors: the couplings of the first strip (0, dt)
  for (int p = 0; p < 2 * kMaxDim; ++p) h.coef_t.push_back({p < 2 * h.d ? c.beta_t[p] : nullptr, c.beta_ut[p]});
  h.coef_t.push_back({c.sigma_t, c.sigma_ut});
  h.time_quad = c.time_quad > 0 ? c.time_quad : 3;
  SG_ST(set_strip_time(h, 0.0));
  Term mt;
  mt.tau[0][0] = 1.0; mt.tau[0][1] = 0.0; mt.tau[1][0] = 0.0; mt.tau[1][1] = 1.0;
  mt.x = h.X.mass;
  mt.v = h.V.mass;
  make_plan(h.mass, std::vector<Term>{mt});
  {
    // H^1(I_j x Omega) Gram form in the Legendre time basis: M_t = dt diag(1, 1/3),
    // C_t = int eta_s' eta_s'' = diag(0, 4 / dt)
    const double dt = cfg.dt;
    std::vector<Term> g;
    Term t0 = mt;
    t0.tau[0][0] = dt;
    t0.tau[1][1] = dt / 3.0 + 4.0 / dt;
    g.push_back(t0);
    for (int p = 0; p < h.d; ++p) {
      Term a = mt, b = mt;
      a.tau[0][0] = b.tau[0][0] = dt;
      a.tau[1][1] = b.tau[1][1] = dt / 3.0;
      a.x = kx[p];
      b.v = kv[p];
      g.push_back(a);
      g.push_back(b);
    }
    make_plan(h.h1, g);
  }
  // u0 load vectors
  for (int k = 0; k < c.n_u0; ++k) {
    std::vector<std::vector<double>> lx, lv;
    SG_ST(load_vectors(hx, c.u0[k].fx, c.u0[k].ux, lx));
    SG_ST(load_vectors(hv, c.u0[k].fv, c.u0[k].uv, lv));
    h.u0x.push_back(lx);
    h.u0v.push_back(lv);
    h.u0coef.push_back(c.u0[k].coef);
  }
  // source f: the Kronecker terms of int_I (f, w + delta (d_t w + beta . grad w))
  // (Sect. 2, b_j): (f_k, phi)(g_k, psi) scaled by int ft (eta_s + delta eta_s'),
  // and per component beta_c = b_c(x) c_c(v) the term
  // delta (f_k b_c, D phi)(g_k c_c, D psi) scaled by int ft eta_s, D the
  // derivative along component c on its side
  if (c.n_f > 0) {
    if (cfg.vlasov_poisson) return {SGDG_EINVAL, "sources are not combined with vlasov_poisson"};
    if (!c.f) return {SGDG_EINVAL, "n_f > 0 with a NULL source array"};
    auto upload_levels = [&](const std::vector<std::vector<double>>& lv, std::vector<double*>& dst) -> Status {
      dst.assign(lv.size(), nullptr);
      for (size_t l = 0; l < lv.size(); ++l) SG_ST(upload(h, &dst[l], lv[l].data(), lv[l].size()));
      return {};
    };
    for (int k = 0; k < c.n_f; ++k) {
      const sgdg_source& f = c.f[k];
      h.src_t.push_back({f.ft, f.ut});
      Handle::SourceTerm t;
      t.src = k;
      t.kind = 0;
      t.coef = f.coef;
      std::vector<std::vector<double>> lx, lv;
      SG_ST(load_vectors_w(hx, {{f.fx, f.ux}}, 0, lx));
      SG_ST(load_vectors_w(hv, {{f.fv, f.uv}}, 0, lv));
      SG_ST(upload_levels(lx, t.lx));
      SG_ST(upload_levels(lv, t.lv));
      h.src_terms.push_back(t);
      for (int comp = 0; comp < 2 * h.d; ++comp) {
        const sgdg_product& b = c.beta[comp];
        if (b.coef == 0.0) continue;
        Handle::SourceTerm tb;
        tb.src = k;
        tb.kind = 1;
        tb.coef = f.coef * b.coef;
        if (c.beta_t[comp]) tb.tfn = comp;
        SG_ST(load_vectors_w(hx, {{f.fx, f.ux}, {b.fx, b.ux}}, comp < h.d ? comp + 1 : 0, lx));
        SG_ST(load_vectors_w(hv, {{f.fv, f.uv}, {b.fv, b.uv}}, comp >= h.d ? comp - h.d + 1 : 0, lv));
        SG_ST(upload_levels(lx, tb.lx));
        SG_ST(upload_levels(lv, tb.lv));
        h.src_terms.push_back(tb);
      }
    }
  }
  // inflow data g: -int_I <g, w>_{Gamma^-} (Sect. 2, b_j), per g term and
  // inflow part the load vectors of the part's x and v factors with the
  // extra weights gx, gv (row sums of the factor matrices: the P1 functions
  // sum to one), scaled by -int_I gt eta_s at every strip
  if (c.n_g > 0) {
    if (cfg.vlasov_poisson) return {SGDG_EINVAL, "inflow data are not combined with vlasov_poisson"};
    if (!c.g) return {SGDG_EINVAL, "n_g > 0 with a NULL inflow array"};
    const std::vector<InflowPart> parts = inflow_parts(c, h.d, cfg.mesh_x, cfg.mesh_v, true);
    auto row_sums = [](const std::vector<Csr>& X, std::vector<std::vector<double>>& out) {
      out.assign(X.size(), {});
      for (size_t l = 0; l < X.size(); ++l) {
        out[l].assign(X[l].nrows, 0.0);
        for (int i = 0; i < X[l].nrows; ++i)
          for (int p = X[l].rowptr[i]; p < X[l].rowptr[i + 1]; ++p) out[l][i] += X[l].val[p];
      }
    };
    for (int k = 0; k < c.n_g; ++k) {
      const sgdg_source& g = c.g[k];
      const int src = (int)h.src_t.size();
      h.src_t.push_back({g.ft, g.ut});
      SideFns gx = fx, gv = fv;   // id gid (after sigma): the g factors
      const int gid = (int)gx.fn.size();
      gx.fn.push_back(g.fx); gx.user.push_back(g.ux);
      gv.fn.push_back(g.fv); gv.user.push_back(g.uv);
      for (const InflowPart& ip : parts) {
        FactorSpec X = ip.x, V = ip.v;
        if (g.fx) { X.wfn.push_back(gid); std::sort(X.wfn.begin(), X.wfn.end()); }
        if (g.fv) { V.wfn.push_back(gid); std::sort(V.wfn.begin(), V.wfn.end()); }
        std::vector<Csr> AX, AV;
        SG_ST(assemble_factor(hx, gx, X, AX));
        SG_ST(assemble_factor(hv, gv, V, AV));
        std::vector<std::vector<double>> lx, lv;
        row_sums(AX, lx);
        row_sums(AV, lv);
        Handle::SourceTerm t;
        t.src = src;
        t.kind = 2;
        t.coef = g.coef * ip.scale;
        if (ip.gate_fn >= 0) {
          t.tfn = t.gate_fn = ip.gate_fn;
          t.gate_sign = ip.gate_sign;
          t.gate_coef = c.beta[ip.gate_fn].coef;
        }
        t.lx.assign(lx.size(), nullptr);
        t.lv.assign(lv.size(), nullptr);
        for (size_t l = 0; l < lx.size(); ++l) SG_ST(upload(h, &t.lx[l], lx[l].data(), lx[l].size()));
        for (size_t l = 0; l < lv.size(); ++l) SG_ST(upload(h, &t.lv[l], lv[l].data(), lv[l].size()));
        h.src_terms.push_back(t);
      }
    }
  }
  if (dev_alloc(h, (void**)&h.U_end, sizeof(double) * h.n_spatial) != cudaSuccess ||
      dev_alloc(h, (void**)&h.u_sol, sizeof(double) * h.n_coeffs) != cudaSuccess ||
      dev_alloc(h, (void**)&h.rhs, sizeof(double) * h.n_coeffs) != cudaSuccess)
    return {SGDG_ENOMEM, "state vectors"};
  SG_CU(cudaMemset(h.u_sol, 0, sizeof(double) * h.n_coeffs));
  SG_CU(cudaMemset(h.U_end, 0, sizeof(double) * h.n_spatial));
  SG_CU(cudaDeviceSynchronize());
  h.hx_host = std::make_shared<Hierarchy>(std::move(hx));
  h.hv_host = std::make_shared<Hierarchy>(std::move(hv));
  return {};
}

}  // namespace

void set_last_error(const std::string& msg) { global_err().msg = msg; }

}  // namespace sgdg

using namespace sgdg;

extern "C" {

sgdg_status sgdg_create(const sgdg_config* cfg, const sgdg_coeffs* coeffs, void** out) {
  if (!cfg || !coeffs || !out) return fail(nullptr, {SGDG_EINVAL, "null argument"});
  Handle* h = new Handle();
  Status st = create(*cfg, *coeffs, *h);
  if (st.code) {
    global_err().msg = st.msg;
    sgdg_destroy(h);
    return st.code;
  }
  *out = h;
  return SGDG_OK;
}

void sgdg_destroy(void* hp) {
  if (!hp) return;
  Handle* h = (Handle*)hp;
  cudaSetDevice(h->cfg.device);
  cudaDeviceSynchronize();
  solver_free(*h);
  for (cudaEvent_t e : h->ev_in) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_out) if (e) cudaEventDestroy(e);
  if (h->host_s) cudaStreamDestroy(h->host_s);
  if (h->host_c) cudaStreamDestroy(h->host_c);
  {
    std::lock_guard<std::mutex> lk(registry_mutex());
    for (void* p : registry(h)) cudaFree(p);
    registry(h).clear();
  }
  delete h;
}

sgdg_status sgdg_validate_mesh(const sgdg_mesh* m) {
  if (!m) return fail(nullptr, {SGDG_EINVAL, "null mesh"});
  const Status st = validate_mesh(*m);
  if (st.code) return fail(nullptr, st);
  return SGDG_OK;
}

const char* sgdg_last_error(const void* hp) {
  if (!hp) return global_err().msg.c_str();
  return ((const Handle*)hp)->err.c_str();
}

sgdg_status sgdg_get_info(const void* hp, sgdg_info* o) {
  if (!hp || !o) return SGDG_EINVAL;
  const Handle* h = (const Handle*)hp;
  o->L = h->L;
  o->d = h->d;
  o->R = 2;
  o->n_grids = h->L + 1;
  o->n_spatial = h->n_spatial;
  o->n_coeffs = h->n_coeffs;
  o->n_terms = (int)h->op.terms.size();
  o->n_x_factors = (int)h->tt.xf.size();
  o->n_v_factors = (int)h->tt.vf.size();
  o->device_bytes = (double)h->device_bytes;
  o->nnz_x = o->nnz_v = o->rows_x = o->rows_v = 0;
  for (int l = 0; l <= h->L; ++l) {
    o->nnz_x += h->X.nnz[l];
    o->nnz_v += h->V.nnz[l];
    o->rows_x += h->X.n[l];
    o->rows_v += h->V.n[l];
  }
  o->lattice_x_levels = 0;
  for (int nx : h->X.lat_nx) o->lattice_x_levels += nx > 0 ? 1 : 0;
  return SGDG_OK;
}

sgdg_status sgdg_grid_shape(const void* hp, int l, int* n1, int* n2, long long* offset) {
  if (!hp) return SGDG_EINVAL;
  const Handle* h = (const Handle*)hp;
  if (l < 0 || l > h->L) return SGDG_EINVAL;
  if (n1) *n1 = h->n1[l];
  if (n2) *n2 = h->n2[l];
  if (offset) *offset = h->off[l];
  return SGDG_OK;
}

sgdg_status sgdg_apply_operator(void* hp, const void* u, void* y, int prec, void* stream) {
  if (!hp || !u || !y) return fail((Handle*)hp, {SGDG_EINVAL, "null argument"});
  Handle* h = (Handle*)hp;
  cudaStream_t s = (cudaStream_t)stream;
  Status st;
  if (prec == SGDG_FP64) st = apply_plan<double>(*h, h->op, (const double*)u, (double*)y, s);
  else if (prec == SGDG_MIXED_FP32) st = apply_plan<float>(*h, h->op, (const float*)u, (float*)y, s);
  else if (prec == SGDG_BF16_STORE) st = apply_plan<Bf16>(*h, h->op, (const __nv_bfloat16*)u, (__nv_bfloat16*)y, s);
  else st = {SGDG_EINVAL, "unknown precision"};
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_apply_mass(void* hp, const void* u, void* y, int prec, void* stream) {
  if (!hp || !u || !y) return fail((Handle*)hp, {SGDG_EINVAL, "null argument"});
  Handle* h = (Handle*)hp;
  cudaStream_t s = (cudaStream_t)stream;
  Status st;
  if (prec == SGDG_FP64) st = apply_plan<double>(*h, h->mass, (const double*)u, (double*)y, s);
  else if (prec == SGDG_MIXED_FP32) st = apply_plan<float>(*h, h->mass, (const float*)u, (float*)y, s);
  else if (prec == SGDG_BF16_STORE)
    st = apply_plan<Bf16>(*h, h->mass, (const __nv_bfloat16*)u, (__nv_bfloat16*)y, s);
  else st = {SGDG_EINVAL, "unknown precision"};
  return st.code ? fail(h, st) : SGDG_OK;
}

namespace {

// The host-buffer apply is pipelined per grid: grid i's input is copied (and
// rounded to the precision's storage type) on a copy stream while earlier
// grids compute, and Y_i is converted and copied back as soon as the sweep
// has finished it.
struct HostApply {
  Handle* h = nullptr;
  int prec = SGDG_FP64;
  double* y = nullptr;
};

Status host_apply_done(void* ctx, int i) {
  HostApply& x = *(HostApply*)ctx;
  Handle& h = *x.h;
  const size_t off = (size_t)h.off[i], n = (size_t)(h.off[i + 1] - h.off[i]);
  double* out64 = (double*)h.b64.cvt_out;
  if (cudaEventRecord(h.ev_out[i], h.host_s) != cudaSuccess || cudaStreamWaitEvent(h.host_c, h.ev_out[i], 0) != cudaSuccess)
    return {SGDG_ECUDA, "host apply: event"};
  cudaError_t e = cudaSuccess;
  if (x.prec == SGDG_MIXED_FP32)
    e = vec_convert<float, double>((const float*)h.b32.cvt_out + off, out64 + off, (long long)n, h.host_c);
  else if (x.prec == SGDG_BF16_STORE)
    e = vec_convert<__nv_bfloat16, double>((const __nv_bfloat16*)h.b16.cvt_out + off, out64 + off, (long long)n,
                                           h.host_c);
  if (e != cudaSuccess) return {SGDG_ECUDA, "host apply: conversion"};
  if (cudaMemcpyAsync(x.y + off, out64 + off, 8 * n, cudaMemcpyDeviceToHost, h.host_c) != cudaSuccess)
    return {SGDG_ECUDA, "host apply: device-to-host copy"};
  return {};
}

}  // namespace

sgdg_status sgdg_apply_operator_host(void* hp, const double* u, double* y, int prec) {
  if (!hp || !u || !y) return fail((Handle*)hp, {SGDG_EINVAL, "null argument"});
  Handle* h = (Handle*)hp;
  if (prec != SGDG_FP64 && prec != SGDG_MIXED_FP32 && prec != SGDG_BF16_STORE)
    return fail(h, {SGDG_EINVAL, "unknown precision"});
  Handle::Bufs& b = h->b64;
  size_t n = (size_t)h->n_coeffs;
  if (!b.cvt_in) {
    if (dev_alloc(*h, &b.cvt_in, 8 * n) != cudaSuccess || dev_alloc(*h, &b.cvt_out, 8 * n) != cudaSuccess)
      return fail(h, {SGDG_ENOMEM, "host-apply buffers"});
  }
  if (prec != SGDG_FP64) {
    Handle::Bufs& bs = prec == SGDG_MIXED_FP32 ? h->b32 : h->b16;
    const size_t esz = prec == SGDG_MIXED_FP32 ? 4 : 2;
    if (!bs.cvt_in &&
        (dev_alloc(*h, &bs.cvt_in, esz * n) != cudaSuccess || dev_alloc(*h, &bs.cvt_out, esz * n) != cudaSuccess))
      return fail(h, {SGDG_ENOMEM, "host-apply buffers"});
  }
  if (!h->host_s) {
    if (cudaStreamCreateWithFlags(&h->host_s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->host_c, cudaStreamNonBlocking) != cudaSuccess)
      return fail(h, {SGDG_ECUDA, "host apply: streams"});
    h->ev_in.assign(h->L + 1, nullptr);
    h->ev_out.assign(h->L + 1, nullptr);
    for (int i = 0; i <= h->L; ++i)
      if (cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_out[i], cudaEventDisableTiming) != cudaSuccess)
        return fail(h, {SGDG_ECUDA, "host apply: events"});
  }
  double* in64 = (double*)b.cvt_in;
  for (int i = 0; i <= h->L; ++i) {
    const size_t off = (size_t)h->off[i], m = (size_t)(h->off[i + 1] - h->off[i]);
    if (cudaMemcpyAsync(in64 + off, u + off, 8 * m, cudaMemcpyHostToDevice, h->host_c) != cudaSuccess)
      return fail(h, {SGDG_ECUDA, "host-to-device copy"});
    cudaError_t e = cudaSuccess;
    if (prec == SGDG_MIXED_FP32)
      e = vec_convert<double, float>(in64 + off, (float*)h->b32.cvt_in + off, (long long)m, h->host_c);
    else if (prec == SGDG_BF16_STORE)
      e = vec_convert<double, __nv_bfloat16>(in64 + off, (__nv_bfloat16*)h->b16.cvt_in + off, (long long)m,
                                             h->host_c);
    if (e != cudaSuccess) return fail(h, {SGDG_ECUDA, "host apply: conversion"});
    if (cudaEventRecord(h->ev_in[i], h->host_c) != cudaSuccess) return fail(h, {SGDG_ECUDA, "host apply: event"});
  }
  HostApply ctx;
  ctx.h = h;
  ctx.prec = prec;
  ctx.y = y;
  ApplyHooks hooks;
  hooks.ready = h->ev_in.data();
  hooks.done = host_apply_done;
  hooks.ctx = &ctx;
  Status st;
  if (prec == SGDG_MIXED_FP32)
    st = apply_plan<float>(*h, h->op, (const float*)h->b32.cvt_in, (float*)h->b32.cvt_out, h->host_s, &hooks);
  else if (prec == SGDG_BF16_STORE)
    st = apply_plan<Bf16>(*h, h->op, (const __nv_bfloat16*)h->b16.cvt_in, (__nv_bfloat16*)h->b16.cvt_out,
                          h->host_s, &hooks);
  else
    st = apply_plan<double>(*h, h->op, (const double*)b.cvt_in, (double*)b.cvt_out, h->host_s, &hooks);
  if (st.code) {
    cudaStreamSynchronize(h->host_c);
    cudaStreamSynchronize(h->host_s);
    return fail(h, st);
  }
  if (cudaStreamSynchronize(h->host_s) != cudaSuccess || cudaStreamSynchronize(h->host_c) != cudaSuccess)
    return fail(h, {SGDG_ECUDA, "device-to-host copy"});
  return SGDG_OK;
}

sgdg_status sgdg_apply_diag(void* hp, int l1, int l2, const void* u, void* y, int prec, void* stream) {
  if (!hp || !u || !y) return fail((Handle*)hp, {SGDG_EINVAL, "null argument"});
  Handle* h = (Handle*)hp;
  if (l1 < 0 || l2 < 0 || l1 > h->L || l2 > h->L || (l1 + l2 != h->L && l1 + l2 != h->L - 1))
    return fail(h, {SGDG_EINVAL, "grid levels must satisfy l1 + l2 in {L-1, L}"});
  cudaStream_t s = (cudaStream_t)stream;
  Status st;
  if (prec == SGDG_FP64) {
    const double* ui[1] = {(const double*)u};
    double* yo[1] = {(double*)y};
    st = apply_diag_grids<double>(*h, 1, &l1, &l2, ui, yo, s);
  } else if (prec == SGDG_MIXED_FP32) {
    const float* ui[1] = {(const float*)u};
    float* yo[1] = {(float*)y};
    st = apply_diag_grids<float>(*h, 1, &l1, &l2, ui, yo, s);
  } else if (prec == SGDG_BF16_STORE) {
    const __nv_bfloat16* ui[1] = {(const __nv_bfloat16*)u};
    __nv_bfloat16* yo[1] = {(__nv_bfloat16*)y};
    st = apply_diag_grids<Bf16>(*h, 1, &l1, &l2, ui, yo, s);
  } else {
    st = {SGDG_EINVAL, "unknown precision"};
  }
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_ct_precondition(void* hp, const double* r, double* z, void* stream) {
  if (!hp || !r || !z) return fail((Handle*)hp, {SGDG_EINVAL, "null argument"});
  Handle* h = (Handle*)hp;
  int its = 0;
  Status st = ct_precondition(*h, r, z, (cudaStream_t)stream, &its);
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_set_initial(void* hp) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  // b_1 = eta(t_0^+) (x) (u0, phi_{l,k}) = (1, -1) (x) sum_p fx_p (x) fv_p per grid
  const int np = (int)h->u0x.size();
  if (np == 0) {
    if (cudaMemset(h->rhs, 0, sizeof(double) * h->n_coeffs) != cudaSuccess)
      return fail(h, {SGDG_ECUDA, "set_initial: clearing the right-hand side"});
  } else {
    for (int l = 0; l <= h->L; ++l) {
      const int n1 = h->n1[l], n2 = h->n2[l];
      std::vector<double> fx((size_t)np * n1), fv((size_t)np * n2);
      for (int p = 0; p < np; ++p) {
        for (int i = 0; i < n1; ++i) fx[(size_t)p * n1 + i] = h->u0coef[p] * h->u0x[p][l][i];
        for (int i = 0; i < n2; ++i) fv[(size_t)p * n2 + i] = h->u0v[p][h->L - l][i];
      }
      double *dfx = nullptr, *dfv = nullptr;
      Status st;
      if (cudaMalloc(&dfx, 8 * fx.size()) != cudaSuccess || cudaMalloc(&dfv, 8 * fv.size()) != cudaSuccess)
        st = {SGDG_ENOMEM, "initial load vectors"};
      else if (cudaMemcpy(dfx, fx.data(), 8 * fx.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemcpy(dfv, fv.data(), 8 * fv.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        st = {SGDG_ECUDA, "set_initial: uploading the initial load vectors"};
      else if (outer_init(h->rhs + h->off[l], n1, n2, np, dfx, dfv, 1.0, -1.0, nullptr) != cudaSuccess ||
               cudaDeviceSynchronize() != cudaSuccess)
        st = {SGDG_ECUDA, "set_initial: forming the first right-hand side"};
      if (dfx) cudaFree(dfx);
      if (dfv) cudaFree(dfv);
      if (st.code) return fail(h, st);
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(h, {SGDG_ECUDA, "set_initial"});
  h->have_initial = true;
  h->first_strip = true;
  h->t_now = 0.0;
  h->solved = false;
  h->nsolved = 0;
  {
    Status st = set_strip_time(*h, 0.0);
    if (st.code) return fail(h, st);
  }
  return SGDG_OK;
}

sgdg_status sgdg_advance_strip(void* hp, void* stream, sgdg_strip_stats* stats) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  Status st = advance_strip(*h, (cudaStream_t)stream, stats);
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_get_solution(const void* hp, double* dst, int on_device) {
  if (!hp || !dst) return SGDG_EINVAL;
  const Handle* h = (const Handle*)hp;
  cudaError_t e = cudaMemcpy(dst, h->u_sol, sizeof(double) * h->n_coeffs,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SGDG_OK : SGDG_ECUDA;
}

sgdg_status sgdg_get_end_value(const void* hp, double* dst, int on_device) {
  if (!hp || !dst) return SGDG_EINVAL;
  const Handle* h = (const Handle*)hp;
  cudaError_t e = cudaMemcpy(dst, h->U_end, sizeof(double) * h->n_spatial,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SGDG_OK : SGDG_ECUDA;
}

int sgdg_struct_sizes(int* out, int n) {
  const int sz[10] = {(int)sizeof(sgdg_mesh),   (int)sizeof(sgdg_product), (int)sizeof(sgdg_source),
                      (int)sizeof(sgdg_coeffs), (int)sizeof(sgdg_config),  (int)sizeof(sgdg_info),
                      (int)sizeof(sgdg_strip_stats), (int)sizeof(sgdg_kernel_stat),
                      (int)sizeof(sgdg_checkpoint_info), (int)sizeof(sgdg_factor_spec)};
  for (int i = 0; out && i < n && i < 10; ++i) out[i] = sz[i];
  return 10;
}

sgdg_status sgdg_set_launch_shape(void* hp, int code) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (code < 0 || code > 255 || (code > 0 && (code & 15) == 0))
    return fail(h, {SGDG_EINVAL, "launch shape code: rows per thread 1..15, flags in bits 4..7"});
  h->force_ch = code;
  return SGDG_OK;
}

sgdg_status sgdg_autotune(void* hp, const void* u, void* y, int prec, void* stream) {
  if (!hp || !u || !y) return fail((Handle*)hp, {SGDG_EINVAL, "null argument"});
  Handle* h = (Handle*)hp;
  Status st;
  if (prec == SGDG_FP64) st = autotune<double>(*h, (const double*)u, (double*)y, (cudaStream_t)stream);
  else if (prec == SGDG_MIXED_FP32) st = autotune<float>(*h, (const float*)u, (float*)y, (cudaStream_t)stream);
  else if (prec == SGDG_BF16_STORE)
    st = autotune<Bf16>(*h, (const __nv_bfloat16*)u, (__nv_bfloat16*)y, (cudaStream_t)stream);
  else st = {SGDG_EINVAL, "unknown precision"};
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_fused_plan_info(void* hp, int grid, int pair_bytes, int* iout, double* dout) {
  if (!hp || !iout || !dout) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (grid < 0 || grid > h->L || (pair_bytes != 4 && pair_bytes != 8 && pair_bytes != 16))
    return fail(h, {SGDG_EINVAL, "fused plan info: grid or pair size out of range"});
  int nterms = 0;
  for (const Chain& c : h->op.A) nterms += (int)c.terms.size();
  const Handle::FusedGrid* fg = nullptr;
  Status st = fused_plan(*h, grid, pair_bytes, (int)h->op.A.size(), nterms, &fg);
  if (st.code) return fail(h, st);
  for (int k = 0; k < 4; ++k) iout[k] = 0;
  dout[0] = dout[1] = 0.0;
  if (!fg) return SGDG_OK;
  iout[0] = fg->ntiles;
  iout[1] = fg->G;
  iout[2] = fg->W;
  iout[3] = (int)fg->smem;
  dout[0] = fg->s_points;
  dout[1] = fg->q_points;
  return SGDG_OK;
}

sgdg_status sgdg_set_sweep_variant(void* hp, int variant) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (variant < 0 || variant > 2) return fail(h, {SGDG_EINVAL, "sweep variant must be 0, 1 or 2"});
  h->sweep_variant = variant;
  return SGDG_OK;
}

sgdg_status sgdg_copy_tuning(void* dst, const void* src) {
  if (!dst || !src) return SGDG_EINVAL;
  Handle* d = (Handle*)dst;
  const Handle* sh = (const Handle*)src;
  for (const auto& kv : sh->tuned_ch) d->tuned_ch[kv.first] = kv.second;
  d->force_ch = 0;
  return SGDG_OK;
}

namespace {
struct Batch {
  std::vector<Handle*> m;
  struct Graph {
    std::vector<const void*> u;
    std::vector<void*> y;
    int prec;
    std::vector<long long> tau_version;   // members' time couplings when captured
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap = nullptr;
  // one stream and two events per member: the captured graph forks into one
  // branch per member (the members share no buffers), so instances whose
  // launches do not fill the GPU run side by side
  std::vector<cudaStream_t> ms;
  std::vector<cudaEvent_t> fork, join;
  ~Batch() {
    for (cudaStream_t x : ms) if (x) cudaStreamDestroy(x);
    for (cudaEvent_t e : fork) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : join) if (e) cudaEventDestroy(e);
  }
};
}  // namespace

sgdg_status sgdg_batch_create(int n, void* const* members, void** out) {
  if (n < 1 || !members || !out) return fail(nullptr, {SGDG_EINVAL, "bad batch arguments"});
  Batch* b = new Batch();
  for (int k = 0; k < n; ++k) {
    if (!members[k]) {
      delete b;
      return fail(nullptr, {SGDG_EINVAL, "null batch member"});
    }
    b->m.push_back((Handle*)members[k]);
  }
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return fail(nullptr, {SGDG_ECUDA, "batch stream"});
  }
  b->ms.assign(n, nullptr);
  b->fork.assign(n, nullptr);
  b->join.assign(n, nullptr);
  for (int k = 0; k < n; ++k)
    if (cudaStreamCreateWithFlags(&b->ms[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) != cudaSuccess) {
      delete b;
      return fail(nullptr, {SGDG_ECUDA, "batch member streams"});
    }
  *out = b;
  return SGDG_OK;
}

void sgdg_batch_destroy(void* bp) {
  if (!bp) return;
  Batch* b = (Batch*)bp;
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

sgdg_status sgdg_batch_apply(void* bp, const void* const* u, void* const* y, int prec, void* stream) {
  if (!bp || !u || !y) return fail(nullptr, {SGDG_EINVAL, "null argument"});
  if (prec != SGDG_FP64 && prec != SGDG_MIXED_FP32 && prec != SGDG_BF16_STORE)
    return fail(nullptr, {SGDG_EINVAL, "unknown precision"});
  Batch* b = (Batch*)bp;
  const size_t n = b->m.size();
  for (size_t gi = 0; gi < b->graphs.size(); ++gi) {
    Batch::Graph& g = b->graphs[gi];
    bool same = g.prec == prec;
    for (size_t k = 0; same && k < n; ++k) same = g.u[k] == u[k] && g.y[k] == y[k];
    if (!same) continue;
    bool fresh = true;
    for (size_t k = 0; k < n; ++k) fresh = fresh && g.tau_version[k] == b->m[k]->tau_version;
    if (!fresh) {   // time couplings changed since the capture (time factors): capture again
      cudaGraphExecDestroy(g.exec);
      b->graphs.erase(b->graphs.begin() + gi);
      break;
    }
    if (cudaGraphLaunch(g.exec, (cudaStream_t)stream) != cudaSuccess)
      return fail(nullptr, {SGDG_ECUDA, "batch graph launch"});
    return SGDG_OK;
  }
  // eager pass: allocates every lazily created buffer before the capture.
  // Both passes fork from stream s into one stream per member (members
  // whose device differs from the batch's stay on s) and join back into s.
  auto run_all = [&](cudaStream_t s) -> Status {
    int dev = 0;
    cudaGetDevice(&dev);
    for (size_t k = 0; k < n; ++k) {
      Handle& m = *b->m[k];
      const bool own = m.cfg.device == dev;
      cudaStream_t ks = own ? b->ms[k] : s;
      if (own) {
        SG_CU(cudaEventRecord(b->fork[k], s));
        SG_CU(cudaStreamWaitEvent(ks, b->fork[k], 0));
      }
      Status st =
          prec == SGDG_FP64        ? apply_plan<double>(m, m.op, (const double*)u[k], (double*)y[k], ks)
          : prec == SGDG_BF16_STORE ? apply_plan<Bf16>(m, m.op, (const __nv_bfloat16*)u[k], (__nv_bfloat16*)y[k], ks)
                                    : apply_plan<float>(m, m.op, (const float*)u[k], (float*)y[k], ks);
      if (st.code) return st;
      if (own) {
        SG_CU(cudaEventRecord(b->join[k], ks));
        SG_CU(cudaStreamWaitEvent(s, b->join[k], 0));
      }
    }
    return {};
  };
  {
    // the eager pass runs on the batch's own (non-blocking) stream: order it
    // after the caller's work, which may still use the members' buffers
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, (cudaStream_t)stream) != cudaSuccess || cudaStreamWaitEvent(b->cap, ev, 0) != cudaSuccess) {
      if (ev) cudaEventDestroy(ev);
      return fail(nullptr, {SGDG_ECUDA, "batch: ordering after the caller's stream"});
    }
    cudaEventDestroy(ev);
  }
  Status st = run_all(b->cap);
  if (st.code) return fail(nullptr, st);
  if (cudaStreamSynchronize(b->cap) != cudaSuccess) return fail(nullptr, {SGDG_ECUDA, "batch eager apply"});
  bool prof[64] = {};
  for (size_t k = 0; k < n && k < 64; ++k) { prof[k] = b->m[k]->prof; b->m[k]->prof = false; }
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(nullptr, {SGDG_ECUDA, "begin capture"});
  st = run_all(b->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
  for (size_t k = 0; k < n && k < 64; ++k) b->m[k]->prof = prof[k];
  if (st.code || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(nullptr, st.code ? st : Status{SGDG_ECUDA, "end capture"});
  }
  Batch::Graph g;
  g.u.assign(u, u + n);
  g.y.assign(y, y + n);
  g.prec = prec;
  for (size_t k = 0; k < n; ++k) g.tau_version.push_back(b->m[k]->tau_version);
  ce = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return fail(nullptr, {SGDG_ECUDA, "graph instantiate"});
  b->graphs.push_back(g);
  if (cudaGraphLaunch(g.exec, (cudaStream_t)stream) != cudaSuccess)
    return fail(nullptr, {SGDG_ECUDA, "batch graph launch"});
  return SGDG_OK;
}

sgdg_status sgdg_batch_advance(void* bp, sgdg_strip_stats* per_member) {
  if (!bp) return fail(nullptr, {SGDG_EINVAL, "null batch"});
  Batch* b = (Batch*)bp;
  const size_t n = b->m.size();
  std::vector<Status> res(n);
  std::vector<sgdg_strip_stats> st(n);
  std::vector<std::thread> th;
  // the members run on streams of their own: finish the callers' work first
  {
    int cur = 0;
    cudaGetDevice(&cur);
    std::vector<int> devs;
    for (size_t k = 0; k < n; ++k)
      if (std::find(devs.begin(), devs.end(), b->m[k]->cfg.device) == devs.end()) devs.push_back(b->m[k]->cfg.device);
    for (int d : devs)
      if (cudaSetDevice(d) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return fail(nullptr, {SGDG_ECUDA, "batch advance: synchronising a member's device"});
    cudaSetDevice(cur);
  }
  for (size_t k = 0; k < n; ++k) {
    th.emplace_back([&, k]() {
      Handle& h = *b->m[k];
      cudaSetDevice(h.cfg.device);
      cudaStream_t s;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        res[k] = {SGDG_ECUDA, "member stream"};
        return;
      }
      res[k] = advance_strip(h, s, &st[k]);
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    });
  }
  for (auto& t : th) t.join();
  sgdg_status first = SGDG_OK;
  for (size_t k = 0; k < n; ++k) {
    if (per_member) per_member[k] = st[k];
    if (res[k].code && first == SGDG_OK) {
      first = res[k].code;
      fail(b->m[k], res[k]);
    }
  }
  return first;
}

static void drop_events(Handle* h) {
  for (auto& k : h->kev) {
    cudaEventDestroy(k.e0);
    cudaEventDestroy(k.e1);
  }
  h->kev.clear();
}

sgdg_status sgdg_profile(void* hp, int enable) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  cudaDeviceSynchronize();
  drop_events(h);
  h->prof = enable != 0;
  return SGDG_OK;
}

sgdg_status sgdg_kernel_stats(void* hp, sgdg_kernel_stat* out, int n_kinds) {
  if (!hp || !out || n_kinds < KIND_COUNT) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(h, {SGDG_ECUDA, "synchronize"});
  for (int k = 0; k < n_kinds; ++k) out[k] = sgdg_kernel_stat{0, 0.0, 0.0, 0.0};
  for (auto& k : h->kev) {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, k.e0, k.e1);
    out[k.kind].launches++;
    out[k.kind].ms += ms;
    out[k.kind].bytes += k.bytes;
    out[k.kind].flops += k.flops;
  }
  drop_events(h);
  return SGDG_OK;
}

long long sgdg_launch_count(const void* hp) { return hp ? ((const Handle*)hp)->launches : 0; }

sgdg_status sgdg_field_update(void* hp, int source, double* energy) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  Status st = field_update(*h, source, energy);
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_set_field(void* hp, const double* E, int n_cells) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  Status st = field_set(*h, E, n_cells);
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_get_field(const void* hp, double* E, int n_cells) {
  if (!hp) return SGDG_EINVAL;
  const Handle* h = (const Handle*)hp;
  Status st = field_get(*h, E, n_cells);
  return st.code ? fail(const_cast<Handle*>(h), st) : SGDG_OK;
}

sgdg_status sgdg_coarse_values(void* hp, const double* u, int R, int lx, int lv, double* out, void* stream) {
  if (!hp || !u || !out) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  Status st = coarse_values(*h, u, R, lx, lv, out, (cudaStream_t)stream);
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_coarse_diff(void* hp, const double* a, const double* b, int R, int lx, int lv, double* out,
                             void* stream) {
  if (!hp || !a || !b || !out) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  Status st = coarse_diff(*h, a, b, R, lx, lv, out, (cudaStream_t)stream);
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_add_coarse(void* hp, const double* c, int lx, int lv, double* u, void* stream) {
  if (!hp || !c || !u) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  Status st = add_coarse(*h, c, lx, lv, u, (cudaStream_t)stream);
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_resolve_strip(void* hp, void* stream, sgdg_strip_stats* stats) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  Status st = advance_strip(*h, (cudaStream_t)stream, stats, true);
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_advance_strip_vp(void* hp, void* stream, double tol, int max_fp, sgdg_strip_stats* stats,
                                  int* fp_steps, double* phi_change) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (!h->field) return fail(h, {SGDG_EINVAL, "the handle was not created with vlasov_poisson = 1"});
  if (!(tol >= 0.0) || max_fp < 0) return fail(h, {SGDG_EINVAL, "tol and max_fp must be >= 0"});
  cudaStream_t s = (cudaStream_t)stream;
  double energy = 0.0;
  const bool paper = h->vp_stop == 1;
  if (paper && !h->vp_prev &&
      (dev_alloc(*h, (void**)&h->vp_prev, sizeof(double) * h->n_coeffs) != cudaSuccess ||
       dev_alloc(*h, (void**)&h->vp_tmp, sizeof(double) * h->n_coeffs) != cudaSuccess))
    return fail(h, {SGDG_ENOMEM, "fixed-point buffers"});
  Status st = field_update(*h, 0, &energy);
  // f^(0) = U^-_{j-1}, constant in time on the strip
  if (!st.code && paper) st = constant_in_time(*h, h->U_end, h->vp_prev, s);
  if (!st.code) st = advance_strip(*h, s, stats, false);
  int k = 0;
  double change = 0.0;
  std::vector<double> prev = h->field->phi;
  std::vector<std::vector<double>> E_prev = h->field->E;
  while (!st.code && k < max_fp) {
    st = field_update(*h, 1, &energy);
    if (st.code) break;
    if (paper) {
      // Sect. 5.3: ||E^(k+1) - E^(k)||_inf (E is constant in time on the strip)
      // + ||f^(k+1) - f^(k)||_{H^1(I_j x Omega)}
      double einf = 0.0;
      for (size_t c = 0; c < E_prev.size(); ++c)
        for (size_t e = 0; e < E_prev[c].size(); ++e)
          einf = std::max(einf, std::fabs(h->field->E[c][e] - E_prev[c][e]));
      if (vec_axpby<double>(h->n_coeffs, 1.0, h->u_sol, -1.0, h->vp_prev, s) != cudaSuccess) {
        st = {SGDG_ECUDA, "fixed-point difference"};
        break;
      }
      double fn = 0.0;
      st = h1_norm(*h, h->vp_prev, h->vp_tmp, &fn, s);
      if (st.code) break;
      change = einf + fn;
    } else {
      const std::vector<double>& phi = h->field->phi;
      double dn = 0.0, pn = 0.0;
      for (size_t i = 0; i < phi.size(); ++i) {
        dn += (phi[i] - prev[i]) * (phi[i] - prev[i]);
        pn += phi[i] * phi[i];
      }
      change = pn > 0.0 ? std::sqrt(dn / pn) : std::sqrt(dn);
    }
    if (change <= tol) break;
    prev = h->field->phi;
    E_prev = h->field->E;
    if (paper && cudaMemcpyAsync(h->vp_prev, h->u_sol, sizeof(double) * h->n_coeffs, cudaMemcpyDeviceToDevice, s) !=
                     cudaSuccess) {
      st = {SGDG_ECUDA, "fixed-point copy"};
      break;
    }
    st = advance_strip(*h, s, stats, true);
    ++k;
  }
  if (fp_steps) *fp_steps = k;
  if (phi_change) *phi_change = change;
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_set_vp_stop(void* hp, int criterion) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (criterion != 0 && criterion != 1) return fail(h, {SGDG_EINVAL, "fixed-point stop must be 0 or 1"});
  h->vp_stop = criterion;
  return SGDG_OK;
}

sgdg_status sgdg_h1_norm(void* hp, const double* u, double* out, void* stream) {
  if (!hp || !u || !out) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (!h->vp_tmp && dev_alloc(*h, (void**)&h->vp_tmp, sizeof(double) * h->n_coeffs) != cudaSuccess)
    return fail(h, {SGDG_ENOMEM, "H1 norm buffer"});
  Status st = h1_norm(*h, u, h->vp_tmp, out, (cudaStream_t)stream);
  return st.code ? fail(h, st) : SGDG_OK;
}

sgdg_status sgdg_set_warm_start(void* hp, int mode) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (mode < 0 || mode > 3) return fail(h, {SGDG_EINVAL, "warm start mode must be 0, 1, 2 or 3"});
  h->warm = mode;
  return SGDG_OK;
}

sgdg_status sgdg_extrapolated_guess(const void* hp, double* dst) {
  if (!hp || !dst) return SGDG_EINVAL;
  const Handle* h = (const Handle*)hp;
  if (!h->solved) return SGDG_EINVAL;
  const size_t bytes = sizeof(double) * h->n_coeffs;
  if (cudaMemcpy(dst, h->u_sol, bytes, cudaMemcpyDeviceToDevice) != cudaSuccess) return SGDG_ECUDA;
  if (h->nsolved >= 2 && h->u_prev2) {
    if (vec_axpby<double>(h->n_coeffs, -1.0, h->u_prev2, 2.0, dst, nullptr) != cudaSuccess) return SGDG_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return SGDG_ECUDA;
  }
  return SGDG_OK;
}

sgdg_status sgdg_set_guess(void* hp, const double* u) {
  if (!hp || !u) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (!h->guess && dev_alloc(*h, (void**)&h->guess, sizeof(double) * h->n_coeffs) != cudaSuccess)
    return fail(h, {SGDG_ENOMEM, "guess buffer"});
  if (cudaMemcpy(h->guess, u, sizeof(double) * h->n_coeffs, cudaMemcpyDeviceToDevice) != cudaSuccess)
    return fail(h, {SGDG_ECUDA, "guess copy"});
  return SGDG_OK;
}

sgdg_status sgdg_finest_x(const void* hp, int* nv, int* nc) {
  if (!hp) return SGDG_EINVAL;
  const Handle* h = (const Handle*)hp;
  if (!h->field) return SGDG_EINVAL;
  const MeshLevel& lv = h->field->hx.lev[h->L];
  if (nv) *nv = lv.n;
  if (nc) *nc = lv.ncells(h->d);
  return SGDG_OK;
}

sgdg_status sgdg_get_density_potential(const void* hp, double* rho, double* phi) {
  if (!hp) return SGDG_EINVAL;
  const Handle* h = (const Handle*)hp;
  if (!h->field || h->field->rho.empty()) return SGDG_EINVAL;
  if (rho) std::copy(h->field->rho.begin(), h->field->rho.end(), rho);
  if (phi) std::copy(h->field->phi.begin(), h->field->phi.end(), phi);
  return SGDG_OK;
}

sgdg_status sgdg_eval_nodal(void* hp, const double* u, double* out, void* stream) {
  if (!hp || !u || !out) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  Status st = nodal_eval(*h, u, out, (cudaStream_t)stream);
  return st.code ? fail(h, st) : SGDG_OK;
}

}  // extern "C"
