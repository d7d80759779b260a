// Vlasov-Poisson field update (Sect. 5.3).
//
// Vlasov: d_t f + v . grad_x f - E . grad_v f = 0, so beta = (v, -E(x)); the
// field comes from -Delta phi = 1 - int f dv, E = -grad phi, on the periodic
// Omega_x.  Once per strip (from U^-_{j-1}, the first iterate of the paper's
// fixed point, midpoint rule in time):
//   rho  = sum_l P_{L<-l} (U^-_l m_v),  m_v[k] = int phi^(2)_k dv     (GPU row sums, host prolongation)
//   K phi = M (1 - rho) with the source's mean removed; phi of zero mean   (FP64 CG, host)
//   E    = -grad phi on every finest cell                              (piecewise constant)
// then every x factor whose weight or inflow split uses E is re-assembled on
// the finest level, projected to all levels and uploaded in place.
#include <cmath>

#include "handle.h"

namespace sgdg {

namespace {

#define SG_CU(x)                                                              \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) return {SGDG_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// out[k1] = sum_k2 U[(k1 n2 + k2) stride] w[k2]: one warp per row, fixed-order
// reduction (stride 2 reads the first time coefficient of a strip vector).
__global__ void k_rowdot(const double* U, const double* w, int n1, int n2, int stride, double* out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n1) return;
  const double* row = U + (size_t)warp * n2 * stride;
  double s = 0.0;
  for (int k = lane; k < n2; k += 32) s += row[(size_t)k * stride] * w[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) out[warp] = s;
}

void spmv(const Csr& A, const std::vector<double>& x, std::vector<double>& y) {
  y.assign(A.nrows, 0.0);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < A.nrows; ++i) {
    double s = 0.0;
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) s += A.val[p] * x[A.col[p]];
    y[i] = s;
  }
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

// CG on the singular, consistent periodic Poisson system K phi = b (b has zero sum).
Status poisson_cg(const Csr& K, const std::vector<double>& b, std::vector<double>& x) {
  const int n = K.nrows;
  if ((int)x.size() != n) x.assign(n, 0.0);
  std::vector<double> r, p, Ap;
  spmv(K, x, Ap);
  r.resize(n);
  for (int i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
  p = r;
  double rr = dot(r, r);
  const double bn = std::sqrt(dot(b, b));
  if (bn == 0.0) {
    x.assign(n, 0.0);
    return {};
  }
  for (int it = 0; it < 20 * n + 100 && std::sqrt(rr) > 1e-13 * bn; ++it) {
    spmv(K, p, Ap);
    const double pAp = dot(p, Ap);
    if (!(pAp > 0.0)) break;
    const double a = rr / pAp;
    for (int i = 0; i < n; ++i) {
      x[i] += a * p[i];
      r[i] -= a * Ap[i];
    }
    const double rn = dot(r, r);
    const double beta = rn / rr;
    rr = rn;
    for (int i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
  }
  if (!std::isfinite(rr)) return {SGDG_ENAN, "NaN in the Poisson solve"};
  return {};
}

}  // namespace

Status field_setup(Handle& h, const sgdg_coeffs& c, const Hierarchy& hx, const Hierarchy& hv, const SideFns& fx) {
  const int d = h.d, L = h.L;
  const sgdg_mesh& mx = h.cfg.mesh_x;
  for (int k = 0; k < d; ++k)
    if (!mx.periodic || !mx.periodic[k]) return {SGDG_EINVAL, "vlasov_poisson needs a periodic Omega_x"};
  for (int i = 0; i < d; ++i)
    if (!c.beta[d + i].fx || c.beta[d + i].fv || c.beta[d + i].coef == 0.0)
      return {SGDG_EINVAL, "vlasov_poisson: beta[d+i] must be coef * E_i(x) with fv = NULL"};
  h.field.reset(new Handle::Field());
  Handle::Field& F = *h.field;
  F.hx = hx;
  F.fx = fx;
  F.fx.fn.assign(fx.fn.size(), nullptr);   // callbacks are valid during sgdg_create only
  F.fx.cell.assign(fx.fn.size(), nullptr);
  const MeshLevel& lv = hx.lev[L];
  const int nc = lv.ncells(d);
  F.E.assign(d, std::vector<double>(nc, 0.0));
  for (int i = 0; i < d; ++i) F.fx.cell[d + i] = &F.E[i];
  // int phi^(2) dv per v level, and on the device
  std::vector<std::vector<double>> one;
  Status st = load_vectors(hv, nullptr, nullptr, one);
  if (st.code) return st;
  F.mv = one;
  F.d_mv.resize(L + 1);
  for (int l = 0; l <= L; ++l) {
    if (dev_alloc(h, (void**)&F.d_mv[l], sizeof(double) * one[l].size()) != cudaSuccess)
      return {SGDG_ENOMEM, "density weights"};
    SG_CU(cudaMemcpy(F.d_mv[l], one[l].data(), sizeof(double) * one[l].size(), cudaMemcpyHostToDevice));
  }
  long long nsum = 0;
  for (int l = 0; l <= L; ++l) nsum += h.X.n[l];
  if (dev_alloc(h, (void**)&F.d_rowsum, sizeof(double) * nsum) != cudaSuccess) return {SGDG_ENOMEM, "row sums"};
  // density of u0 at the finest x vertices: sum_k coef_k u0x_k(x) int u0v_k dv
  F.rho0.assign(lv.n, 0.0);
  for (int k = 0; k < c.n_u0; ++k) {
    std::vector<double> vals(lv.n, 1.0);
    if (c.u0[k].fx) c.u0[k].fx(lv.n, lv.coords.data(), vals.data(), c.u0[k].ux);
    std::vector<std::vector<double>> lvv;
    st = load_vectors(hv, c.u0[k].fv, c.u0[k].uv, lvv);
    if (st.code) return st;
    double integ = 0.0;
    for (double x : lvv[0]) integ += x;
    for (int i = 0; i < lv.n; ++i) F.rho0[i] += c.u0[k].coef * vals[i] * integ;
  }
  // finest-level stiffness and mass
  SideFns none;
  none.fn.assign(5, nullptr);
  FactorSpec ms;
  std::vector<Csr> X;
  st = assemble_factor(hx, none, ms, X);
  if (st.code) return st;
  F.M = X[L];
  for (int i = 1; i <= d; ++i) {
    FactorSpec ks;
    ks.test = ks.trial = i;
    st = assemble_factor(hx, none, ks, X);
    if (st.code) return st;
    if (i == 1) F.K = X[L];
    else
      for (size_t p = 0; p < F.K.val.size(); ++p) F.K.val[p] += X[L].val[p];
  }
  return {};
}

Status field_update(Handle& h, int source, double* energy) {
  if (!h.field) return {SGDG_EINVAL, "the handle was not created with vlasov_poisson = 1"};
  Handle::Field& F = *h.field;
  const int d = h.d, L = h.L;
  const MeshLevel& lv = F.hx.lev[L];
  // density: of u0, of the end value U^-, or of the strip solution at the
  // strip midpoint (sum_s eta_s(1/2) u_s = u_0 for the Legendre basis)
  if (source != 0 && source != 1) return {SGDG_EINVAL, "field source must be 0 or 1"};
  if (source == 1 && !h.solved) return {SGDG_EINVAL, "no strip solution for the midpoint density"};
  if (source == 0 && h.first_strip) {
    F.rho = F.rho0;
  } else {
    long long o = 0;
    std::vector<long long> ro(L + 2, 0);
    for (int l = 0; l <= L; ++l) {
      const int n1 = h.n1[l], n2 = h.n2[l];
      if (source == 0) k_rowdot<<<(n1 + 7) / 8, 256>>>(h.U_end + h.soff[l], F.d_mv[L - l], n1, n2, 1, F.d_rowsum + o);
      else k_rowdot<<<(n1 + 7) / 8, 256>>>(h.u_sol + h.off[l], F.d_mv[L - l], n1, n2, 2, F.d_rowsum + o);
      SG_CU(cudaGetLastError());
      ro[l] = o;
      o += n1;
    }
    std::vector<double> rs(o);
    SG_CU(cudaMemcpy(rs.data(), F.d_rowsum, sizeof(double) * o, cudaMemcpyDeviceToHost));
    std::vector<double> acc(rs.begin() + ro[0], rs.begin() + ro[0] + h.n1[0]);
    for (int l = 1; l <= L; ++l) {
      const Csr& E = F.hx.E[l - 1];
      std::vector<double> nx(E.nrows, 0.0);
      for (int i = 0; i < E.nrows; ++i)
        for (int p = E.rowptr[i]; p < E.rowptr[i + 1]; ++p) nx[i] += E.val[p] * acc[E.col[p]];
      for (int i = 0; i < h.n1[l]; ++i) nx[i] += rs[ro[l] + i];
      acc.swap(nx);
    }
    F.rho = acc;
  }
  // Poisson: K phi = M (1 - rho), mean of the source removed
  const int n = lv.n;
  std::vector<double> src(n), b, m;
  for (int i = 0; i < n; ++i) src[i] = 1.0 - F.rho[i];
  spmv(F.M, src, b);
  spmv(F.M, std::vector<double>(n, 1.0), m);
  double sb = 0.0, sm = 0.0;
  for (int i = 0; i < n; ++i) { sb += b[i]; sm += m[i]; }
  for (int i = 0; i < n; ++i) b[i] -= m[i] * (sb / sm);
  Status st = poisson_cg(F.K, b, F.phi);
  if (st.code) return st;
  double pm = 0.0;
  for (int i = 0; i < n; ++i) pm += m[i] * F.phi[i];
  for (int i = 0; i < n; ++i) F.phi[i] -= pm / sm;
  // E = -grad phi per finest cell (geometric, unwrapped cell coordinates)
  const int nc = lv.ncells(d), d1 = d + 1;
  double en = 0.0;
  for (int e = 0; e < nc; ++e) {
    const double* v0 = &lv.cell_coords[(size_t)e * d1 * d];
    const int* cv = &lv.cells[(size_t)e * d1];
    double J[2][2] = {{0, 0}, {0, 0}}, Ji[2][2], det;
    for (int k = 0; k < d; ++k)
      for (int a = 0; a < d; ++a) J[k][a] = v0[(a + 1) * d + k] - v0[k];
    if (d == 1) { det = J[0][0]; Ji[0][0] = 1.0 / det; }
    else {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
      Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
    }
    // grad phi = J^{-T} (phi_a - phi_0)_a
    double dphi[2] = {0, 0};
    for (int a = 0; a < d; ++a) dphi[a] = F.phi[cv[a + 1]] - F.phi[cv[0]];
    double area = std::fabs(det) / (d == 1 ? 1.0 : 2.0);
    double e2 = 0.0;
    for (int k = 0; k < d; ++k) {
      double g = 0.0;
      for (int a = 0; a < d; ++a) g += Ji[a][k] * dphi[a];
      F.E[k][e] = -g;
      e2 += g * g;
    }
    en += 0.5 * e2 * area;
  }
  if (energy) *energy = en;
  F.updated = true;
  return field_reassemble(h);
}

Status field_set(Handle& h, const double* E, int n_cells) {
  if (!h.field) return {SGDG_EINVAL, "the handle was not created with vlasov_poisson = 1"};
  Handle::Field& F = *h.field;
  const int d = h.d, nc = F.hx.lev[h.L].ncells(d);
  if (!E || n_cells != nc) return {SGDG_EINVAL, "set_field: n_cells differs from the finest x cell count"};
  for (int k = 0; k < d; ++k)
    for (int e = 0; e < nc; ++e)
      if (!std::isfinite(E[(size_t)k * nc + e])) return {SGDG_EINVAL, "set_field: NaN or Inf in the field"};
  for (int k = 0; k < d; ++k) F.E[k].assign(E + (size_t)k * nc, E + (size_t)(k + 1) * nc);
  F.updated = true;
  return field_reassemble(h);
}

Status field_get(const Handle& h, double* E, int n_cells) {
  if (!h.field) return {SGDG_EINVAL, "the handle was not created with vlasov_poisson = 1"};
  const Handle::Field& F = *h.field;
  const int d = h.d, nc = F.hx.lev[h.L].ncells(d);
  if (!E || n_cells != nc) return {SGDG_EINVAL, "get_field: n_cells differs from the finest x cell count"};
  for (int k = 0; k < d; ++k) std::copy(F.E[k].begin(), F.E[k].end(), E + (size_t)k * nc);
  return {};
}

// Re-assemble and upload every x factor whose weight or inflow split uses E,
// from the current cell field F.E.
Status field_reassemble(Handle& h) {
  if (!h.field) return {SGDG_EINVAL, "the handle was not created with vlasov_poisson = 1"};
  Handle::Field& F = *h.field;
  const int d = h.d, L = h.L;
  Status st;
  for (size_t f = 0; f < h.tt.xf.size(); ++f) {
    const FactorSpec& fs = h.tt.xf[f];
    bool uses = false;
    for (int id : fs.wfn) uses = uses || (id >= d && id < 2 * d);
    for (auto& rs : fs.restrict_) uses = uses || (rs.first >= d && rs.first < 2 * d);
    if (!uses) continue;
    std::vector<Csr> X;
    st = assemble_factor(F.hx, F.fx, fs, X);
    if (st.code) return st;
    for (int l = 0; l <= L; ++l) {
      st = upload_pattern_vals(h, h.X, F.hx.lev[l].pattern, l, X[l].val, &h.X.v64.ell_fac[f][l],
                           &h.X.v32.ell_fac[f][l]);
      if (st.code) return st;
    }
    st = upload_factor_products(h, F.hx, h.X, (int)f, X);
    if (st.code) return st;
  }
  return {};
}

}  // namespace sgdg
