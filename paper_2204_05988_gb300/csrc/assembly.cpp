// FP64 assembly of the d-dimensional factor matrices on the finest level and
// their Galerkin projection to every coarser level (Sect. 4.2):
//     X_l = E_{l+1<-l}^T X_{l+1} E_{l+1<-l}   (=> X_l = E_{L<-l}^T X_L E_{L<-l}).
//
// Quadrature: q = 4 Gauss-Legendre points per direction on [0,1] (nodes by
// Newton's method on P_q), collapsed onto the triangle (Duffy map
// (a, b) -> (a, b (1 - a)), Jacobian 1 - a) and the tetrahedron
// ((a, b, c) -> (a, b (1 - a), c (1 - a)(1 - b)), Jacobian (1 - a)^2 (1 - b)).  Sign restrictions (inflow
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
  if (k == 2) {
    for (int a = 0; a < kQ; ++a)
      for (int b = 0; b < kQ; ++b) {
        pts.push_back(g[a]);
        pts.push_back(g[b] * (1.0 - g[a]));
        wts.push_back(w[a] * w[b] * (1.0 - g[a]));
      }
    return;
  }
  // tetrahedron: (a, b, c) -> (a, b (1 - a), c (1 - a)(1 - b)), Jacobian (1 - a)^2 (1 - b)
  for (int a = 0; a < kQ; ++a)
    for (int b = 0; b < kQ; ++b)
      for (int c = 0; c < kQ; ++c) {
        pts.push_back(g[a]);
        pts.push_back(g[b] * (1.0 - g[a]));
        pts.push_back(g[c] * (1.0 - g[a]) * (1.0 - g[b]));
        wts.push_back(w[a] * w[b] * w[c] * (1.0 - g[a]) * (1.0 - g[a]) * (1.0 - g[b]));
      }
}

int find_pos(const Csr& P, int i, int j) {
  auto b = P.col.begin() + P.rowptr[i], e = P.col.begin() + P.rowptr[i + 1];
  auto it = std::lower_bound(b, e, j);
  if (it == e || *it != j) return -1;
  return (int)(it - P.col.begin());
}

// The coefficient function id at every point.  With `finite` a NaN or Inf
// value (a bad coefficient of a factor - beta, sigma, the inflow data g -
// or a callback that failed and reported NaN) is refused; the load vectors
// of u0 and the sources pass it on, so that NaN data reach the solver and
// its NaN check (SGDG_ENAN).
Status eval_fn(const SideFns& fns, int id, const std::vector<double>& pts, int d, std::vector<double>& out,
               bool finite = true) {
  int n = (int)(pts.size() / d);
  out.assign(n, 0.0);
  const int chunk = 1 << 22;
  for (int s = 0; s < n; s += chunk) {
    int m = std::min(chunk, n - s);
    fns.fn[id](m, pts.data() + (size_t)s * d, out.data() + s, fns.user[id]);
  }
  if (finite)
    for (double v : out)
      if (!std::isfinite(v)) return {SGDG_EINVAL, "a coefficient function returned NaN or Inf"};
  return {};
}

}  // namespace

void gauss_rule01(int q, std::vector<double>& x, std::vector<double>& w) { gauss_legendre01(q, x, w); }

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

namespace {

// Affine map of a simplex (vertices v0 .. vd): the inverse Jacobian Ji and
// det J, for d = 1, 2, 3.
void simplex_jacobian(int d, const double* v0, double (&Ji)[3][3], double& det) {
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int k = 0; k < d; ++k)
    for (int a = 0; a < d; ++a) J[k][a] = v0[(a + 1) * d + k] - v0[k];
  if (d == 1) {
    det = J[0][0];
    Ji[0][0] = 1.0 / det;
  } else if (d == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
  } else {
    // cofactors: Ji = adj(J) / det
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    Ji[0][0] = c00 / det;
    Ji[1][0] = c01 / det;
    Ji[2][0] = c02 / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  }
}

// physical gradients of the barycentric functions: grad lam_a = Ji^T gref_a
void barycentric_gradients(int d, const double (&Ji)[3][3], double (&grad)[4][3]) {
  for (int a = 0; a <= d; ++a)
    for (int k = 0; k < d; ++k) {
      double g = 0.0;
      for (int m = 0; m < d; ++m) {
        const double gr = (a == 0) ? -1.0 : (m == a - 1 ? 1.0 : 0.0);
        g += Ji[m][k] * gr;
      }
      grad[a][k] = g;
    }
}

constexpr int kCellChunk = 1 << 15;   // cells per pass of the volume assembly

}  // namespace

Status assemble_volume(const Hierarchy& h, const SideFns& fns, const std::vector<FactorSpec>& specs,
                       std::vector<std::vector<Csr>>& X) {
  const int d = h.d, d1 = d + 1, L = h.L;
  const MeshLevel& lv = h.lev[L];
  const Csr& P = lv.pattern;
  const int nc = lv.ncells(d);
  const int nf = (int)specs.size();
  X.assign(nf, std::vector<Csr>());
  // the functions the factors read (weights at the quadrature points, signs
  // at the cell centroids); cell fields are read per cell
  std::vector<int> wids, rids;
  for (const FactorSpec& f : specs) {
    if (f.kind != 0) return {SGDG_EINVAL, "assemble_volume: boundary-face factor"};
    for (int id : f.wfn) {
      if (const std::vector<double>* cf = fns.cell_field(id)) {
        if ((int)cf->size() != nc) return {SGDG_EINVAL, "cell field size differs from the finest cell count"};
      } else if (id < 0 || id >= (int)fns.fn.size() || !fns.fn[id]) {
        return {SGDG_EINVAL, "factor needs a coefficient function that is no longer available"};
      } else if (std::find(wids.begin(), wids.end(), id) == wids.end()) {
        wids.push_back(id);
      }
    }
    for (auto& rs : f.restrict_) {
      if (const std::vector<double>* cf = fns.cell_field(rs.first)) {
        if ((int)cf->size() != nc) return {SGDG_EINVAL, "cell field size differs from the finest cell count"};
      } else if (rs.first < 0 || rs.first >= (int)fns.fn.size() || !fns.fn[rs.first]) {
        return {SGDG_EINVAL, "factor needs a coefficient function that is no longer available"};
      } else if (std::find(rids.begin(), rids.end(), rs.first) == rids.end()) {
        rids.push_back(rs.first);
      }
    }
  }
  for (int f = 0; f < nf; ++f) {
    X[f].assign(L + 1, Csr());
    Csr& A = X[f][L];
    A.nrows = A.ncols = lv.n;
    A.rowptr = P.rowptr;
    A.col = P.col;
    A.val.assign(P.col.size(), 0.0);
  }
  std::vector<double> rp, rw;
  simplex_rule(d, rp, rw);
  const int nq = (int)rw.size();
  // per chunk: quadrature points, centroids, function values, element scatter
  // positions; then every factor's element matrices, scattered in cell order
  // (the values do not depend on the chunk size or the thread count)
  std::vector<double> pts, cen;
  std::map<int, std::vector<double>> wv, rv;
  std::vector<int> pos;
  for (int e0 = 0; e0 < nc; e0 += kCellChunk) {
    const int ne = std::min(kCellChunk, nc - e0);
    pts.assign((size_t)ne * nq * d, 0.0);
    cen.assign((size_t)ne * d, 0.0);
    pos.assign((size_t)ne * d1 * d1, 0);
#pragma omp parallel for schedule(static)
    for (int c = 0; c < ne; ++c) {
      const size_t e = (size_t)e0 + c;
      const double* v0 = &lv.cell_coords[e * d1 * d];
      for (int q = 0; q < nq; ++q)
        for (int k = 0; k < d; ++k) {
          double x = v0[k];
          for (int a = 1; a < d1; ++a) x += (v0[a * d + k] - v0[k]) * rp[q * d + (a - 1)];
          pts[((size_t)c * nq + q) * d + k] = x;
        }
      for (int a = 0; a < d1; ++a)
        for (int k = 0; k < d; ++k) cen[(size_t)c * d + k] += v0[a * d + k] / d1;
      const int* cv = &lv.cells[e * d1];
      for (int i = 0; i < d1; ++i)
        for (int j = 0; j < d1; ++j) pos[((size_t)c * d1 + i) * d1 + j] = find_pos(P, cv[i], cv[j]);
    }
    for (int id : wids) {
      Status se = eval_fn(fns, id, pts, d, wv[id]);
      if (se.code) return se;
    }
    for (int id : rids) {
      Status se = eval_fn(fns, id, cen, d, rv[id]);
      if (se.code) return se;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int fi = 0; fi < nf; ++fi) {
      const FactorSpec& f = specs[fi];
      std::vector<double>& val = X[fi][L].val;
      std::vector<double> wq((size_t)nq);
      for (int c = 0; c < ne; ++c) {
        const size_t e = (size_t)e0 + c;
        bool keep = true;
        for (auto& rs : f.restrict_) {
          const std::vector<double>* cf = fns.cell_field(rs.first);
          const double sv = cf ? (*cf)[e] : rv.at(rs.first)[c];
          if (!(rs.second * sv > 0.0)) keep = false;
        }
        if (!keep) continue;
        const double* v0 = &lv.cell_coords[e * d1 * d];
        double Ji[3][3], det, grad[4][3];
        simplex_jacobian(d, v0, Ji, det);
        barycentric_gradients(d, Ji, grad);
        for (int q = 0; q < nq; ++q) wq[q] = 1.0;
        for (int id : f.wfn) {
          if (const std::vector<double>* cf = fns.cell_field(id)) {
            for (int q = 0; q < nq; ++q) wq[q] *= (*cf)[e];
          } else {
            const double* fv = &wv.at(id)[(size_t)c * nq];
            for (int q = 0; q < nq; ++q) wq[q] *= fv[q];
          }
        }
        double Ke[4][4] = {{0}};
        for (int q = 0; q < nq; ++q) {
          double lam[4];
          lam[0] = 1.0;
          for (int a = 1; a < d1; ++a) { lam[a] = rp[q * d + a - 1]; lam[0] -= lam[a]; }
          const double w = rw[q] * std::fabs(det) * wq[q];
          for (int i = 0; i < d1; ++i) {
            const double ti = f.test == 0 ? lam[i] : grad[i][f.test - 1];
            for (int j = 0; j < d1; ++j) {
              const double tj = f.trial == 0 ? lam[j] : grad[j][f.trial - 1];
              Ke[i][j] += w * ti * tj;
            }
          }
        }
        for (int i = 0; i < d1; ++i)
          for (int j = 0; j < d1; ++j) val[pos[((size_t)c * d1 + i) * d1 + j]] += Ke[i][j];
      }
    }
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int fi = 0; fi < nf; ++fi) project_down(h, X[fi]);
  return {};
}

Status assemble_factor(const Hierarchy& h, const SideFns& fns, const FactorSpec& f, std::vector<Csr>& X) {
  const int d = h.d, L = h.L;
  const MeshLevel& lv = h.lev[L];
  const Csr& P = lv.pattern;
  if (f.kind == 0) {
    std::vector<std::vector<Csr>> one;
    Status st = assemble_volume(h, fns, {f}, one);
    if (st.code) return st;
    X = std::move(one[0]);
    return {};
  }
  X.assign(L + 1, Csr());
  Csr& A = X[L];
  A.nrows = A.ncols = lv.n;
  A.rowptr = P.rowptr;
  A.col = P.col;
  A.val.assign(P.col.size(), 0.0);
  {
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
    for (auto& rs : f.restrict_) {
      if (fns.cell_field(rs.first)) return {SGDG_EINVAL, "cell fields are not supported on boundary faces"};
      if (rs.first < 0 || rs.first >= (int)fns.fn.size() || !fns.fn[rs.first])
        return {SGDG_EINVAL, "boundary-face factor restricted by a missing coefficient function"};
    }
    for (int id : f.wfn) {
      if (fns.cell_field(id)) return {SGDG_EINVAL, "cell fields are not supported on boundary faces"};
      if (id < 0 || id >= (int)fns.fn.size() || !fns.fn[id])
        return {SGDG_EINVAL, "boundary-face factor needs a missing coefficient function"};
    }
    if (!f.restrict_.empty() && !sel.empty()) {
      std::vector<double> cen(sel.size() * d, 0.0), val;
      for (size_t s = 0; s < sel.size(); ++s)
        for (int a = 0; a < dv; ++a)
          for (int k = 0; k < d; ++k) cen[s * d + k] += lv.bface_coords[((size_t)sel[s] * dv + a) * d + k] / dv;
      for (auto& rs : f.restrict_) {
        Status se = eval_fn(fns, rs.first, cen, d, val);
        if (se.code) return se;
        for (size_t s = 0; s < sel.size(); ++s)
          if (!(rs.second * val[s] > 0.0)) keep[s] = 0;
      }
    }
    std::vector<double> pts(sel.size() * nq * d);
    std::vector<double> meas(sel.size());
    for (size_t s = 0; s < sel.size(); ++s) {
      const double* f0 = &lv.bface_coords[(size_t)sel[s] * dv * d];
      // |det| of the map from the reference face: 1 (a point), the edge
      // length, or twice the triangle area |(f1 - f0) x (f2 - f0)|
      if (dv == 1) meas[s] = 1.0;
      else if (dv == 2) {
        double l2 = 0.0;
        for (int k = 0; k < d; ++k) l2 += (f0[d + k] - f0[k]) * (f0[d + k] - f0[k]);
        meas[s] = std::sqrt(l2);
      } else {
        double a[3], b[3];
        for (int k = 0; k < 3; ++k) { a[k] = f0[3 + k] - f0[k]; b[k] = f0[6 + k] - f0[k]; }
        const double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
        meas[s] = std::sqrt(cx * cx + cy * cy + cz * cz);
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
      Status se = eval_fn(fns, id, pts, d, tmp);
      if (se.code) return se;
      for (size_t i = 0; i < wprod.size(); ++i) wprod[i] *= tmp[i];
    }
    for (size_t s = 0; s < sel.size(); ++s) {
      if (!keep[s]) continue;
      const int* fv = &lv.bfaces[(size_t)sel[s] * dv];
      for (int q = 0; q < nq; ++q) {
        double lam[3];
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
  out.assign(L + 1, {});
  out[L].assign(lv.n, 0.0);
  // cells in chunks (points, function values), accumulated in cell order
  std::vector<double> pts, val, tmp;
  for (int e0 = 0; e0 < nc; e0 += kCellChunk) {
    const int ne = std::min(kCellChunk, nc - e0);
    pts.assign((size_t)ne * nq * d, 0.0);
    val.assign((size_t)ne * nq, 1.0);
#pragma omp parallel for schedule(static)
    for (int c = 0; c < ne; ++c) {
      const double* v0 = &lv.cell_coords[((size_t)e0 + c) * d1 * d];
      for (int q = 0; q < nq; ++q)
        for (int k = 0; k < d; ++k) {
          double x = v0[k];
          for (int a = 1; a < d1; ++a) x += (v0[a * d + k] - v0[k]) * rp[q * d + (a - 1)];
          pts[((size_t)c * nq + q) * d + k] = x;
        }
    }
    for (const auto& f : fns) {
      if (!f.first) continue;
      SideFns t;
      t.fn.push_back(f.first);
      t.user.push_back(f.second);
      eval_fn(t, 0, pts, d, tmp, false);   // data: NaN is the solver's to report
      for (size_t i = 0; i < val.size(); ++i) val[i] *= tmp[i];
    }
    for (int c = 0; c < ne; ++c) {
      const size_t e = (size_t)e0 + c;
      const double* v0 = &lv.cell_coords[e * d1 * d];
      double Ji[3][3], det, grad[4][3];
      simplex_jacobian(d, v0, Ji, det);
      // physical gradient component of the barycentric functions (constant per cell)
      if (deriv > 0) barycentric_gradients(d, Ji, grad);
      det = std::fabs(det);
      for (int q = 0; q < nq; ++q) {
        double lam[4];
        lam[0] = 1.0;
        for (int a = 1; a < d1; ++a) { lam[a] = rp[q * d + a - 1]; lam[0] -= lam[a]; }
        const double wq = rw[q] * det * val[(size_t)c * nq + q];
        for (int a = 0; a < d1; ++a)
          out[L][lv.cells[e * d1 + a]] += wq * (deriv > 0 ? grad[a][deriv - 1] : lam[a]);
      }
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
