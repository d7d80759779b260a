// FP64 assembly of the d-dimensional factor matrices on the finest level and
// their Galerkin projection to every coarser level (Sect. 4.2):
//     X_l = E_{l+1<-l}^T X_{l+1} E_{l+1<-l}   (=> X_l = E_{L<-l}^T X_L E_{L<-l}).
//
// Quadrature: q = 4 Gauss-Legendre points per direction on [0,1] (nodes by
// Newton's method on P_q), collapsed onto the triangle (Duffy map
// (a, b) -> (a, b (1 - a)), Jacobian 1 - a).  Sign restrictions (inflow
// splitting, Sect. 5.2) test the sign of one coefficient function at the cell
// or face centroid.
#include <algorithm>
#include <cmath>
#include <map>

#include "internal.h"

namespace sgdg {

namespace {

constexpr int kQ = 4;

void gauss_legendre01(int q, std::vector<double>& x, std::vector<double>& w) {
  x.resize(q);
  w.resize(q);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);   // 2/((1-z^2) P'^2) on [-1,1], halved
  }
}

// Reference simplex rule of dimension k (0: a point).
void simplex_rule(int k, std::vector<double>& pts, std::vector<double>& wts) {
  std::vector<double> g, w;
  gauss_legendre01(kQ, g, w);
  pts.clear();
  wts.clear();
  if (k == 0) { wts.push_back(1.0); return; }
  if (k == 1) { pts = g; wts = w; return; }
  for (int a = 0; a < kQ; ++a)
    for (int b = 0; b < kQ; ++b) {
      pts.push_back(g[a]);
      pts.push_back(g[b] * (1.0 - g[a]));
      wts.push_back(w[a] * w[b] * (1.0 - g[a]));
    }
}

int find_pos(const Csr& P, int i, int j) {
  auto b = P.col.begin() + P.rowptr[i], e = P.col.begin() + P.rowptr[i + 1];
  auto it = std::lower_bound(b, e, j);
  if (it == e || *it != j) return -1;
  return (int)(it - P.col.begin());
}

void eval_fn(const SideFns& fns, int id, const std::vector<double>& pts, int d, std::vector<double>& out) {
  int n = (int)(pts.size() / d);
  out.assign(n, 0.0);
  const int chunk = 1 << 22;
  for (int s = 0; s < n; s += chunk) {
    int m = std::min(chunk, n - s);
    fns.fn[id](m, pts.data() + (size_t)s * d, out.data() + s, fns.user[id]);
  }
}

}  // namespace

bool FactorSpec::operator<(const FactorSpec& o) const {
  if (kind != o.kind) return kind < o.kind;
  if (wfn != o.wfn) return wfn < o.wfn;
  if (test != o.test) return test < o.test;
  if (trial != o.trial) return trial < o.trial;
  if (restrict_ != o.restrict_) return restrict_ < o.restrict_;
  if (face_axis != o.face_axis) return face_axis < o.face_axis;
  return face_side < o.face_side;
}
bool FactorSpec::operator==(const FactorSpec& o) const { return !(*this < o) && !(o < *this); }

static void project_down(const Hierarchy& h, std::vector<Csr>& X) {
  for (int l = h.L - 1; l >= 0; --l) {
    const Csr& P = h.lev[l].pattern;
    const Csr& Rt = h.Rt[l];
    const Csr& E = h.E[l];
    const Csr& F = X[l + 1];
    Csr& C = X[l];
    C.nrows = C.ncols = P.nrows;
    C.rowptr = P.rowptr;
    C.col = P.col;
    C.val.assign(P.col.size(), 0.0);
#pragma omp parallel for schedule(dynamic, 256)
    for (int i = 0; i < P.nrows; ++i) {
      for (int p = Rt.rowptr[i]; p < Rt.rowptr[i + 1]; ++p) {
        int k = Rt.col[p];
        double r = Rt.val[p];
        for (int q = F.rowptr[k]; q < F.rowptr[k + 1]; ++q) {
          int m = F.col[q];
          double rx = r * F.val[q];
          if (rx == 0.0) continue;
          for (int e = E.rowptr[m]; e < E.rowptr[m + 1]; ++e) {
            int pos = find_pos(P, i, E.col[e]);
            if (pos >= 0) C.val[pos] += rx * E.val[e];
          }
        }
      }
    }
  }
}

Status prefill_cache(const Hierarchy& h, const SideFns& fns, const std::vector<FactorSpec>& specs, QuadCache& cache) {
  // one serial assembly of a plain volume factor fills the points and positions
  FactorSpec plain;
  std::vector<Csr> X;
  Status st = assemble_factor(h, fns, plain, X, &cache);
  if (st.code) return st;
  const int d = h.d, d1 = d + 1;
  const MeshLevel& lv = h.lev[h.L];
  const int nc = lv.ncells(d);
  std::vector<double> cen;
  for (const FactorSpec& f : specs) {
    if (f.kind != 0) continue;
    for (int id : f.wfn) {
      if (fns.cell_field(id) || cache.fn_vals.count(id)) continue;
      if (!fns.fn[id]) return {SGDG_EINVAL, "factor needs a coefficient function that is no longer available"};
      eval_fn(fns, id, cache.pts, d, cache.fn_vals[id]);
    }
    for (auto& rs : f.restrict_) {
      if (fns.cell_field(rs.first) || cache.cen_vals.count(rs.first)) continue;
      if (cen.empty()) {
        cen.assign((size_t)nc * d, 0.0);
        for (int e = 0; e < nc; ++e)
          for (int a = 0; a < d1; ++a)
            for (int k = 0; k < d; ++k) cen[(size_t)e * d + k] += lv.cell_coords[((size_t)e * d1 + a) * d + k] / d1;
      }
      eval_fn(fns, rs.first, cen, d, cache.cen_vals[rs.first]);
    }
  }
  return {};
}

Status assemble_factor(const Hierarchy& h, const SideFns& fns, const FactorSpec& f, std::vector<Csr>& X,
                       QuadCache* cache) {
  const int d = h.d, d1 = d + 1, L = h.L;
  const MeshLevel& lv = h.lev[L];
  const Csr& P = lv.pattern;
  X.assign(L + 1, Csr());
  Csr& A = X[L];
  A.nrows = A.ncols = lv.n;
  A.rowptr = P.rowptr;
  A.col = P.col;
  A.val.assign(P.col.size(), 0.0);

  if (f.kind == 0) {
    const int nc = lv.ncells(d);
    std::vector<double> rp, rw;
    simplex_rule(d, rp, rw);
    const int nq = (int)rw.size();
    // centroids for the sign restriction
    std::vector<char> keep(nc, 1);
    if (!f.restrict_.empty()) {
      std::vector<double> cen((size_t)nc * d, 0.0), val;
      for (int e = 0; e < nc; ++e)
        for (int a = 0; a < d1; ++a)
          for (int k = 0; k < d; ++k) cen[(size_t)e * d + k] += lv.cell_coords[((size_t)e * d1 + a) * d + k] / d1;
      for (auto& rs : f.restrict_) {
        if (const std::vector<double>* cf = fns.cell_field(rs.first)) {
          if ((int)cf->size() != nc) return {SGDG_EINVAL, "cell field size differs from the finest cell count"};
          val = *cf;
        } else if (cache && cache->cen_vals.count(rs.first)) {
          val = cache->cen_vals.at(rs.first);
        } else {
          eval_fn(fns, rs.first, cen, d, val);
          if (cache) cache->cen_vals[rs.first] = val;
        }
        for (int e = 0; e < nc; ++e)
          if (!(rs.second * val[e] > 0.0)) keep[e] = 0;
      }
    }
    // quadrature points of all cells and the weight product there
    std::vector<double> own_pts;
    std::vector<double>& pts = cache ? cache->pts : own_pts;
    if (pts.size() != (size_t)nc * nq * d) {
      pts.assign((size_t)nc * nq * d, 0.0);
#pragma omp parallel for schedule(static)
      for (int e = 0; e < nc; ++e) {
        const double* v0 = &lv.cell_coords[(size_t)e * d1 * d];
        for (int q = 0; q < nq; ++q)
          for (int k = 0; k < d; ++k) {
            double x = v0[k];
            for (int a = 1; a < d1; ++a) x += (v0[a * d + k] - v0[k]) * rp[q * d + (a - 1)];
            pts[((size_t)e * nq + q) * d + k] = x;
          }
      }
    }
    std::vector<double> wprod((size_t)nc * nq, 1.0), tmp;
    for (int id : f.wfn) {
      if (const std::vector<double>* cf = fns.cell_field(id)) {
        if ((int)cf->size() != nc) return {SGDG_EINVAL, "cell field size differs from the finest cell count"};
        for (int e = 0; e < nc; ++e)
          for (int q = 0; q < nq; ++q) wprod[(size_t)e * nq + q] *= (*cf)[e];
        continue;
      }
      if (!fns.fn[id]) return {SGDG_EINVAL, "factor needs a coefficient function that is no longer available"};
      const std::vector<double>* vals = nullptr;
      if (cache) {
        auto it = cache->fn_vals.find(id);
        if (it == cache->fn_vals.end()) {
          eval_fn(fns, id, pts, d, tmp);
          it = cache->fn_vals.emplace(id, std::move(tmp)).first;
        }
        vals = &it->second;
      } else {
        eval_fn(fns, id, pts, d, tmp);
        vals = &tmp;
      }
      for (size_t i = 0; i < wprod.size(); ++i) wprod[i] *= (*vals)[i];
    }
    // element matrices in parallel, then one ordered scatter: the assembled
    // values do not depend on the thread count (bit-reproducible set-up)
    std::vector<double> Kall((size_t)nc * d1 * d1, 0.0);
#pragma omp parallel for schedule(static)
    for (int e = 0; e < nc; ++e) {
      if (!keep[e]) continue;
      const double* v0 = &lv.cell_coords[(size_t)e * d1 * d];
      double J[2][2] = {{0, 0}, {0, 0}}, Ji[2][2], det;
      for (int k = 0; k < d; ++k)
        for (int a = 0; a < d; ++a) J[k][a] = v0[(a + 1) * d + k] - v0[k];
      if (d == 1) { det = J[0][0]; Ji[0][0] = 1.0 / det; }
      else {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
      }
      // physical gradients of the barycentric functions: grad lam_a = Ji^T gref_a
      double grad[3][2];
      for (int a = 0; a < d1; ++a)
        for (int k = 0; k < d; ++k) {
          double g = 0.0;
          for (int m = 0; m < d; ++m) {
            double gr = (a == 0) ? -1.0 : (m == a - 1 ? 1.0 : 0.0);
            g += Ji[m][k] * gr;
          }
          grad[a][k] = g;
        }
      double Ke[3][3] = {{0}};
      for (int q = 0; q < nq; ++q) {
        double lam[3];
        lam[0] = 1.0;
        for (int a = 1; a < d1; ++a) { lam[a] = rp[q * d + a - 1]; lam[0] -= lam[a]; }
        double wq = rw[q] * std::fabs(det) * wprod[(size_t)e * nq + q];
        for (int i = 0; i < d1; ++i) {
          double ti = f.test == 0 ? lam[i] : grad[i][f.test - 1];
          for (int j = 0; j < d1; ++j) {
            double tj = f.trial == 0 ? lam[j] : grad[j][f.trial - 1];
            Ke[i][j] += wq * ti * tj;
          }
        }
      }
      for (int i = 0; i < d1; ++i)
        for (int j = 0; j < d1; ++j) Kall[((size_t)e * d1 + i) * d1 + j] = Ke[i][j];
    }
    std::vector<int> own_pos;
    std::vector<int>& pos = cache ? cache->pos : own_pos;
    if (pos.size() != (size_t)nc * d1 * d1) {
      pos.assign((size_t)nc * d1 * d1, 0);
#pragma omp parallel for schedule(static)
      for (int e = 0; e < nc; ++e) {
        const int* cv = &lv.cells[(size_t)e * d1];
        for (int i = 0; i < d1; ++i)
          for (int j = 0; j < d1; ++j) pos[((size_t)e * d1 + i) * d1 + j] = find_pos(P, cv[i], cv[j]);
      }
    }
    for (int e = 0; e < nc; ++e) {
      if (!keep[e]) continue;
      for (int i = 0; i < d1; ++i)
        for (int j = 0; j < d1; ++j) A.val[pos[((size_t)e * d1 + i) * d1 + j]] += Kall[((size_t)e * d1 + i) * d1 + j];
    }
  } else {
    // boundary faces on one side
    std::vector<int> sel;
    const int nf = lv.nbfaces(d);
    for (int i = 0; i < nf; ++i)
      if (lv.bface_axis[i] == f.face_axis && lv.bface_side[i] == f.face_side) sel.push_back(i);
    const int dv = d;  // vertices per face
    std::vector<double> rp, rw;
    simplex_rule(dv - 1, rp, rw);
    const int nq = (int)rw.size();
    std::vector<char> keep(sel.size(), 1);
    for (auto& rs : f.restrict_)
      if (fns.cell_field(rs.first)) return {SGDG_EINVAL, "cell fields are not supported on boundary faces"};
    for (int id : f.wfn)
      if (fns.cell_field(id)) return {SGDG_EINVAL, "cell fields are not supported on boundary faces"};
    if (!f.restrict_.empty() && !sel.empty()) {
      std::vector<double> cen(sel.size() * d, 0.0), val;
      for (size_t s = 0; s < sel.size(); ++s)
        for (int a = 0; a < dv; ++a)
          for (int k = 0; k < d; ++k) cen[s * d + k] += lv.bface_coords[((size_t)sel[s] * dv + a) * d + k] / dv;
      for (auto& rs : f.restrict_) {
        eval_fn(fns, rs.first, cen, d, val);
        for (size_t s = 0; s < sel.size(); ++s)
          if (!(rs.second * val[s] > 0.0)) keep[s] = 0;
      }
    }
    std::vector<double> pts(sel.size() * nq * d);
    std::vector<double> meas(sel.size());
    for (size_t s = 0; s < sel.size(); ++s) {
      const double* f0 = &lv.bface_coords[(size_t)sel[s] * dv * d];
      if (dv == 1) meas[s] = 1.0;
      else {
        double l2 = 0.0;
        for (int k = 0; k < d; ++k) l2 += (f0[d + k] - f0[k]) * (f0[d + k] - f0[k]);
        meas[s] = std::sqrt(l2);
      }
      for (int q = 0; q < nq; ++q)
        for (int k = 0; k < d; ++k) {
          double x = f0[k];
          for (int a = 1; a < dv; ++a) x += (f0[a * d + k] - f0[k]) * rp[q * (dv - 1) + a - 1];
          pts[(s * nq + q) * d + k] = x;
        }
    }
    std::vector<double> wprod(sel.size() * nq, 1.0), tmp;
    for (int id : f.wfn) {
      if (sel.empty()) break;
      eval_fn(fns, id, pts, d, tmp);
      for (size_t i = 0; i < wprod.size(); ++i) wprod[i] *= tmp[i];
    }
    for (size_t s = 0; s < sel.size(); ++s) {
      if (!keep[s]) continue;
      const int* fv = &lv.bfaces[(size_t)sel[s] * dv];
      for (int q = 0; q < nq; ++q) {
        double lam[2];
        lam[0] = 1.0;
        for (int a = 1; a < dv; ++a) { lam[a] = rp[q * (dv - 1) + a - 1]; lam[0] -= lam[a]; }
        double wq = rw[q] * meas[s] * wprod[s * nq + q];
        for (int i = 0; i < dv; ++i)
          for (int j = 0; j < dv; ++j) A.val[find_pos(P, fv[i], fv[j])] += wq * lam[i] * lam[j];
      }
    }
  }
  project_down(h, X);
  return {};
}

Status load_vectors(const Hierarchy& h, sgdg_fn fn, void* user, std::vector<std::vector<double>>& out) {
  return load_vectors_w(h, {{fn, user}}, 0, out);
}

Status load_vectors_w(const Hierarchy& h, const std::vector<std::pair<sgdg_fn, void*>>& fns, int deriv,
                      std::vector<std::vector<double>>& out) {
  const int d = h.d, d1 = d + 1, L = h.L;
  if (deriv < 0 || deriv > d) return {SGDG_EINVAL, "load vector: derivative direction out of range"};
  const MeshLevel& lv = h.lev[L];
  const int nc = lv.ncells(d);
  std::vector<double> rp, rw;
  simplex_rule(d, rp, rw);
  const int nq = (int)rw.size();
  std::vector<double> pts((size_t)nc * nq * d), val((size_t)nc * nq, 1.0), tmp;
  for (int e = 0; e < nc; ++e) {
    const double* v0 = &lv.cell_coords[(size_t)e * d1 * d];
    for (int q = 0; q < nq; ++q)
      for (int k = 0; k < d; ++k) {
        double x = v0[k];
        for (int a = 1; a < d1; ++a) x += (v0[a * d + k] - v0[k]) * rp[q * d + (a - 1)];
        pts[((size_t)e * nq + q) * d + k] = x;
      }
  }
  for (const auto& f : fns) {
    if (!f.first) continue;
    SideFns t;
    t.fn.push_back(f.first);
    t.user.push_back(f.second);
    eval_fn(t, 0, pts, d, tmp);
    for (size_t i = 0; i < val.size(); ++i) val[i] *= tmp[i];
  }
  out.assign(L + 1, {});
  out[L].assign(lv.n, 0.0);
  for (int e = 0; e < nc; ++e) {
    const double* v0 = &lv.cell_coords[(size_t)e * d1 * d];
    double J[2][2] = {{0, 0}, {0, 0}}, Ji[2][2], det;
    for (int k = 0; k < d; ++k)
      for (int a = 0; a < d; ++a) J[k][a] = v0[(a + 1) * d + k] - v0[k];
    if (d == 1) { det = J[0][0]; Ji[0][0] = 1.0 / det; }
    else {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
      Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
    }
    // physical gradient component of the barycentric functions (constant per cell)
    double grad[3] = {0.0, 0.0, 0.0};
    if (deriv > 0)
      for (int a = 0; a < d1; ++a) {
        double g = 0.0;
        for (int m = 0; m < d; ++m) {
          const double gr = (a == 0) ? -1.0 : (m == a - 1 ? 1.0 : 0.0);
          g += Ji[m][deriv - 1] * gr;
        }
        grad[a] = g;
      }
    det = std::fabs(det);
    for (int q = 0; q < nq; ++q) {
      double lam[3];
      lam[0] = 1.0;
      for (int a = 1; a < d1; ++a) { lam[a] = rp[q * d + a - 1]; lam[0] -= lam[a]; }
      const double wq = rw[q] * det * val[(size_t)e * nq + q];
      for (int a = 0; a < d1; ++a)
        out[L][lv.cells[(size_t)e * d1 + a]] += wq * (deriv > 0 ? grad[a] : lam[a]);
    }
  }
  for (int l = L - 1; l >= 0; --l) {
    const Csr& Rt = h.Rt[l];
    out[l].assign(h.lev[l].n, 0.0);
    for (int i = 0; i < Rt.nrows; ++i)
      for (int p = Rt.rowptr[i]; p < Rt.rowptr[i + 1]; ++p) out[l][i] += Rt.val[p] * out[l + 1][Rt.col[p]];
  }
  return {};
}

}  // namespace sgdg
