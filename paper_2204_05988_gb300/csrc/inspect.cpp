// Host-only views of the discrete spaces, factors and Kronecker terms the
// library builds (sgdg_inspect_level, sgdg_inspect_embedding,
// sgdg_inspect_factor, sgdg_inspect_product, sgdg_inspect_load,
// sgdg_inspect_terms).
//
// They run the same host code as sgdg_create - the mesh checks, the
// refinement into nested levels with their canonical vertex order, the FP64
// assembly on the finest level and the Galerkin projection of Sect. 4.2 - on
// one mesh, without a handle or a device, and copy the result out.  They let
// a caller (or a test on a machine without a GPU) compare what the library
// assembles with an independent implementation.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace sgdg {
namespace {

sgdg_status fail_host(const Status& st) {
  set_last_error(st.msg);
  return st.code;
}

Status hierarchy_of(const sgdg_mesh* m, int L, int level, Hierarchy& h) {
  if (!m) return {SGDG_EINVAL, "null mesh"};
  if (L < 0 || L >= kMaxLevels) return {SGDG_EINVAL, "L out of range 0..11"};
  if (level < 0 || level > L) return {SGDG_EINVAL, "level out of range 0..L"};
  Status st = validate_mesh(*m);
  if (st.code) return st;
  return build_hierarchy(*m, L, h);
}

// CSR out: sizes always; arrays when all three are given
void copy_csr(const Csr& A, int* nrows, int* nnz, int* rowptr, int* col, double* val) {
  if (nrows) *nrows = A.nrows;
  if (nnz) *nnz = A.nnz();
  if (rowptr && col && val) {
    std::memcpy(rowptr, A.rowptr.data(), sizeof(int) * A.rowptr.size());
    std::memcpy(col, A.col.data(), sizeof(int) * A.col.size());
    std::memcpy(val, A.val.data(), sizeof(double) * A.val.size());
  }
}

Status spec_out(const FactorSpec& f, sgdg_factor_spec& o) {
  if (f.wfn.size() > 4 || f.restrict_.size() > 2) return {SGDG_EINVAL, "a factor spec does not fit sgdg_factor_spec"};
  std::memset(&o, 0, sizeof(o));
  o.kind = f.kind;
  o.test = f.test;
  o.trial = f.trial;
  o.n_weight = (int)f.wfn.size();
  for (size_t i = 0; i < f.wfn.size(); ++i) o.weight[i] = f.wfn[i];
  o.n_restrict = (int)f.restrict_.size();
  for (size_t i = 0; i < f.restrict_.size(); ++i) {
    o.restrict_fn[i] = f.restrict_[i].first;
    o.restrict_sign[i] = f.restrict_[i].second;
  }
  o.face_axis = f.face_axis;
  o.face_side = f.face_side;
  return {};
}

// one factor on every level of the hierarchy refined to L (the code of
// sgdg_create: the side's coefficient functions numbered as there, beta
// components 0 .. 2 kMaxDim - 1, then sigma)
Status factor_levels(const sgdg_mesh* mesh, const sgdg_coeffs* coeffs, int side, int L, int level,
                     const sgdg_factor_spec* spec, Hierarchy& h, std::vector<Csr>& per_level) {
  if (!coeffs || !spec) return {SGDG_EINVAL, "null coefficients or factor spec"};
  if (side != 0 && side != 1) return {SGDG_EINVAL, "side must be 0 (x) or 1 (v)"};
  Status st = hierarchy_of(mesh, L, level, h);
  if (st.code) return st;
  const int d = mesh->dim;
  SideFns fns;
  for (int p = 0; p < 2 * kMaxDim; ++p) {
    const sgdg_product& b = coeffs->beta[p];
    fns.fn.push_back(p < 2 * d ? (side == 0 ? b.fx : b.fv) : nullptr);
    fns.user.push_back(side == 0 ? b.ux : b.uv);
  }
  fns.fn.push_back(side == 0 ? coeffs->sigma.fx : coeffs->sigma.fv);
  fns.user.push_back(side == 0 ? coeffs->sigma.ux : coeffs->sigma.uv);
  const int nfn = (int)fns.fn.size();
  FactorSpec f;
  f.kind = spec->kind;
  f.test = spec->test;
  f.trial = spec->trial;
  if (f.kind != 0 && f.kind != 1) return {SGDG_EINVAL, "factor kind must be 0 (volume) or 1 (faces)"};
  if (f.test < 0 || f.test > d || f.trial < 0 || f.trial > d)
    return {SGDG_EINVAL, "derivative index out of range 0..dim"};
  if (spec->n_weight < 0 || spec->n_weight > 4 || spec->n_restrict < 0 || spec->n_restrict > 2)
    return {SGDG_EINVAL, "at most 4 weight functions and 2 restrictions"};
  for (int i = 0; i < spec->n_weight; ++i) {
    if (spec->weight[i] < 0 || spec->weight[i] >= nfn || !fns.fn[spec->weight[i]])
      return {SGDG_EINVAL, "weight function id names no function of this side"};
    f.wfn.push_back(spec->weight[i]);
  }
  for (int i = 0; i < spec->n_restrict; ++i) {
    const int id = spec->restrict_fn[i], sg = spec->restrict_sign[i];
    if (id < 0 || id >= nfn || !fns.fn[id] || (sg != 1 && sg != -1))
      return {SGDG_EINVAL, "restriction: a function of this side and a sign of +-1"};
    f.restrict_.push_back({id, sg});
  }
  std::sort(f.wfn.begin(), f.wfn.end());
  std::sort(f.restrict_.begin(), f.restrict_.end());
  if (f.kind == 1) {
    if (spec->face_axis < 0 || spec->face_axis >= d || (spec->face_side != 1 && spec->face_side != -1))
      return {SGDG_EINVAL, "face: an axis of the mesh and a side of +-1"};
    f.face_axis = spec->face_axis;
    f.face_side = spec->face_side;
  }
  return assemble_factor(h, fns, f, per_level);
}

}  // namespace
}  // namespace sgdg

using namespace sgdg;

extern "C" {

sgdg_status sgdg_inspect_level(const sgdg_mesh* mesh, int L, int level, int* n_vertices, double* coords) {
  Hierarchy h;
  Status st = hierarchy_of(mesh, L, level, h);
  if (st.code) return fail_host(st);
  const MeshLevel& lv = h.lev[level];
  if (n_vertices) *n_vertices = lv.n;
  if (coords) std::memcpy(coords, lv.coords.data(), sizeof(double) * lv.coords.size());
  return SGDG_OK;
}

sgdg_status sgdg_inspect_embedding(const sgdg_mesh* mesh, int L, int level, int* nrows, int* nnz, int* rowptr,
                                   int* col, double* val) {
  Hierarchy h;
  Status st = hierarchy_of(mesh, L, level, h);
  if (st.code) return fail_host(st);
  if (level >= L) return fail_host({SGDG_EINVAL, "the embedding of level l needs l < L"});
  copy_csr(h.E[level], nrows, nnz, rowptr, col, val);
  return SGDG_OK;
}

sgdg_status sgdg_inspect_factor(const sgdg_mesh* mesh, const sgdg_coeffs* coeffs, int side, int L, int level,
                                const sgdg_factor_spec* spec, int* nrows, int* nnz, int* rowptr, int* col,
                                double* val) {
  Hierarchy h;
  std::vector<Csr> per_level;
  Status st = factor_levels(mesh, coeffs, side, L, level, spec, h, per_level);
  if (st.code) return fail_host(st);
  copy_csr(per_level[level], nrows, nnz, rowptr, col, val);
  return SGDG_OK;
}

sgdg_status sgdg_inspect_product(const sgdg_mesh* mesh, const sgdg_coeffs* coeffs, int side, int L, int level,
                                 const sgdg_factor_spec* spec, int which, int* nrows, int* nnz, int* rowptr,
                                 int* col, double* val) {
  if (which == 0 ? level >= L : (which == 1 ? level < 1 : true))
    return fail_host({SGDG_EINVAL, "which 0 needs level < L, which 1 needs level >= 1"});
  Hierarchy h;
  std::vector<Csr> X;
  Status st = factor_levels(mesh, coeffs, side, L, level, spec, h, X);
  if (st.code) return fail_host(st);
  // the products as sgdg_create forms them for the sweep (Sect. 4.2: the
  // restriction of a factor and a factor with the prolongation)
  Csr C;
  if (which == 0) {
    C = product_pattern(h.Rt[level], h.lev[level + 1].pattern);
    product_values(h.Rt[level], h.Rt[level].val, X[level + 1], X[level + 1].val, C, C.val);
  } else {
    C = product_pattern(h.lev[level].pattern, h.E[level - 1]);
    product_values(X[level], X[level].val, h.E[level - 1], h.E[level - 1].val, C, C.val);
  }
  copy_csr(C, nrows, nnz, rowptr, col, val);
  return SGDG_OK;
}

sgdg_status sgdg_inspect_load(const sgdg_mesh* mesh, int L, int level, int n_fn, const sgdg_fn* fns,
                              void* const* users, int deriv, double* out) {
  if (n_fn < 0 || n_fn > 4 || (n_fn > 0 && !fns)) return fail_host({SGDG_EINVAL, "0..4 weight functions"});
  Hierarchy h;
  Status st = hierarchy_of(mesh, L, level, h);
  if (st.code) return fail_host(st);
  std::vector<std::pair<sgdg_fn, void*>> w;
  for (int i = 0; i < n_fn; ++i) w.push_back({fns[i], users ? users[i] : nullptr});
  std::vector<std::vector<double>> per_level;
  st = load_vectors_w(h, w, deriv, per_level);
  if (st.code) return fail_host(st);
  if (out) std::memcpy(out, per_level[level].data(), sizeof(double) * per_level[level].size());
  return SGDG_OK;
}

sgdg_status sgdg_inspect_terms(const sgdg_mesh* mesh_x, const sgdg_mesh* mesh_v, const sgdg_coeffs* coeffs,
                               double dt, double delta, double t0, int capacity, int* n_terms, double* tau,
                               sgdg_factor_spec* xspec, sgdg_factor_spec* vspec) {
  if (!mesh_x || !mesh_v || !coeffs || !n_terms) return fail_host({SGDG_EINVAL, "null argument"});
  if (mesh_x->dim != mesh_v->dim) return fail_host({SGDG_EINVAL, "mesh_x and mesh_v must have the same dimension"});
  if (!(dt > 0.0) || !(delta >= 0.0)) return fail_host({SGDG_EINVAL, "dt must be > 0 and delta >= 0"});
  if (coeffs->time_quad < 0 || coeffs->time_quad > 8) return fail_host({SGDG_EINVAL, "time_quad must be in 0..8"});
  Status st = validate_mesh(*mesh_x);
  if (!st.code) st = validate_mesh(*mesh_v);
  if (st.code) return fail_host(st);
  const int d = mesh_x->dim;
  TermTable tt;
  st = build_terms(*coeffs, d, *mesh_x, *mesh_v, dt, delta, tt);
  if (st.code) return fail_host(st);
  if (tt.time_dep) {
    // the couplings of the strip (t0, t0 + dt), as sgdg_create and every
    // strip compute them
    std::vector<std::pair<sgdg_tfn, void*>> ft;
    for (int p = 0; p < 2 * kMaxDim; ++p) ft.push_back({p < 2 * d ? coeffs->beta_t[p] : nullptr, coeffs->beta_ut[p]});
    ft.push_back({coeffs->sigma_t, coeffs->sigma_ut});
    st = strip_time_couplings(tt, t0, dt, coeffs->time_quad > 0 ? coeffs->time_quad : 3, ft);
    if (st.code) return fail_host(st);
  }
  const int n = (int)tt.terms.size();
  *n_terms = n;
  if (!tau && !xspec && !vspec) return SGDG_OK;
  if (!tau || !xspec || !vspec || capacity < n) return fail_host({SGDG_EINVAL, "output arrays missing or too short"});
  for (int k = 0; k < n; ++k) {
    const Term& t = tt.terms[k];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) tau[4 * k + 2 * a + b] = t.tau[a][b];
    st = spec_out(tt.xf[t.x], xspec[k]);
    if (!st.code) st = spec_out(tt.vf[t.v], vspec[k]);
    if (st.code) return fail_host(st);
  }
  return SGDG_OK;
}

}  // extern "C"
