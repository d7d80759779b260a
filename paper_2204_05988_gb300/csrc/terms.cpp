// Kronecker term table of the strip operator (Sect. 2, Eq. 5; Sect. 4.2).
//
// Expanding the strip form
//   a(v,w) = int_I (d_t v + d_beta v + sigma v, w + delta (d_t w + d_beta w))
//            - <v, w>_{Gamma^-} dt + (v(t_{j-1}^+), w(t_{j-1}^+))
// on the product basis eta_s phi^(1) phi^(2) with time-constant coefficients
// in the tensor form beta_p = c_p fx_p(x) fv_p(v), sigma = c_s sx(x) sv(v)
// gives a short sum of terms tau (x) X (x) V, tau the 2x2 time coupling.
// For the Legendre basis on a strip of length dt (derived from the
// definitions of Sect. 4.2, Eq. 10):
//   M_t = dt diag(1, 1/3), T_t = [[0, 2], [0, 0]], C_t = [[0, 0], [0, 4/dt]],
//   G_t = [[1, -1], [-1, 1]]
// Contributions (row s = test, column s' = trial):
//   (d_t v, w) + (d_t v, d d_t w) + (v^+, w^+)  -> (T_t + d C_t + G_t) (x) M (x) M
//   (d_t v, d d_beta w)                          -> d T_t   (x) [phi_j, c_q fx_q D_q phi_i]
//   (d_beta v, w) + (d_beta v, d d_t w)          -> (M_t + d T_t^T) (x) [c_p fx_p D_p phi_j, phi_i]
//   (d_beta v, d d_beta w)                       -> d M_t  (x) [c_p c_q D_p phi_j, D_q phi_i]
//   (sigma v, w) + (sigma v, d d_t w)            -> (M_t + d T_t^T) (x) [sigma phi_j, phi_i]
//   (sigma v, d d_beta w)                        -> d M_t  (x) [sigma phi_j, c_q D_q phi_i]
//   -<v, w>_{Gamma^-}                            -> -M_t (x) G, G split by box side and by
//                                                   the signs of the beta factors (Sect. 5.2)
// Scalar coefficients go into tau; terms with identical factor pairs merge.
#include <algorithm>
#include <cmath>
#include <map>

#include "internal.h"

namespace sgdg {

std::vector<InflowPart> inflow_parts(const sgdg_coeffs& c, int d, const sgdg_mesh& mx, const sgdg_mesh& mv) {
  // beta_p = cp b_p(x) c_p(v); on the face y_ax = side of Omega_x (p < d) or
  // Omega_v (p >= d), beta . n = side cp b_p c_p < 0 where the signs s1 of
  // cp b_p and s2 of c_p satisfy side s1 s2 < 0; each sign pair is one
  // Kronecker pair with the sign restricted at cell or face centroids
  std::vector<InflowPart> out;
  for (int p = 0; p < 2 * d; ++p) {
    if (c.beta[p].coef == 0.0) continue;
    const bool xface = p < d;
    const int ax = xface ? p : p - d;
    const sgdg_mesh& m = xface ? mx : mv;
    if (m.periodic && m.periodic[ax]) continue;
    const double cp = c.beta[p].coef;
    const int sc = cp > 0 ? 1 : -1;
    const bool hx = c.beta[p].fx != nullptr, hv = c.beta[p].fv != nullptr;
    for (int side = -1; side <= 1; side += 2)
      for (int s1 = 1; s1 >= -1; s1 -= 2) {
        const int s2 = -side * s1;
        InflowPart ip;
        ip.x.kind = xface ? 1 : 0;
        ip.v.kind = xface ? 0 : 1;
        if (hx) { ip.x.wfn = {p}; ip.x.restrict_ = {{p, s1 * sc}}; }
        else if (s1 != sc) continue;
        if (hv) { ip.v.wfn = {p}; ip.v.restrict_ = {{p, s2}}; }
        else if (s2 != 1) continue;
        FactorSpec& F = xface ? ip.x : ip.v;
        F.face_axis = ax;
        F.face_side = side;
        ip.scale = side * cp;
        out.push_back(ip);
      }
  }
  return out;
}

Status build_terms(const sgdg_coeffs& c, int d, const sgdg_mesh& mx, const sgdg_mesh& mv,
                   double dt, double delta, TermTable& out) {
  const double Mt[2][2] = {{dt, 0.0}, {0.0, dt / 3.0}};
  const double Tt[2][2] = {{0.0, 2.0}, {0.0, 0.0}};
  const double Ct[2][2] = {{0.0, 0.0}, {0.0, 4.0 / dt}};
  const double Gt[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
  // function ids: beta components 0..2d-1, sigma kSigmaFn
  const int SIG = kSigmaFn;
  auto has_x = [&](int p) { return (p == SIG ? c.sigma.fx : c.beta[p].fx) != nullptr; };
  auto has_v = [&](int p) { return (p == SIG ? c.sigma.fv : c.beta[p].fv) != nullptr; };
  auto Dx = [&](int p) { return p < d ? p + 1 : 0; };
  auto Dv = [&](int p) { return p >= d ? p - d + 1 : 0; };

  struct Raw { double tau[2][2]; FactorSpec x, v; };
  std::vector<Raw> raw;
  auto add = [&](const double t[2][2], double scale, FactorSpec x, FactorSpec v) {
    std::sort(x.wfn.begin(), x.wfn.end());
    std::sort(v.wfn.begin(), v.wfn.end());
    std::sort(x.restrict_.begin(), x.restrict_.end());
    std::sort(v.restrict_.begin(), v.restrict_.end());
    Raw r;
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < 2; ++q) r.tau[s][q] = scale * t[s][q];
    r.x = x;
    r.v = v;
    raw.push_back(r);
  };
  auto vol = [](std::vector<int> w, int test, int trial) {
    FactorSpec f;
    f.kind = 0;
    f.wfn = w;
    f.test = test;
    f.trial = trial;
    return f;
  };
  auto wx = [&](std::initializer_list<int> ps) {
    std::vector<int> w;
    for (int p : ps) if (has_x(p)) w.push_back(p);
    return w;
  };
  auto wv = [&](std::initializer_list<int> ps) {
    std::vector<int> w;
    for (int p : ps) if (has_v(p)) w.push_back(p);
    return w;
  };
  std::vector<int> act;
  for (int p = 0; p < 2 * d; ++p)
    if (c.beta[p].coef != 0.0) act.push_back(p);

  double t1[2][2], t2[2][2], t3[2][2];
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 2; ++q) {
      t1[s][q] = Tt[s][q] + delta * Ct[s][q] + Gt[s][q];
      t2[s][q] = Mt[s][q] + delta * Tt[q][s];
      t3[s][q] = delta * Mt[s][q];
    }
  double dTt[2][2];
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 2; ++q) dTt[s][q] = delta * Tt[s][q];

  add(t1, 1.0, vol({}, 0, 0), vol({}, 0, 0));
  for (int q : act) add(dTt, c.beta[q].coef, vol(wx({q}), Dx(q), 0), vol(wv({q}), Dv(q), 0));
  for (int p : act) add(t2, c.beta[p].coef, vol(wx({p}), 0, Dx(p)), vol(wv({p}), 0, Dv(p)));
  for (int p : act)
    for (int q : act)
      add(t3, c.beta[p].coef * c.beta[q].coef, vol(wx({p, q}), Dx(q), Dx(p)), vol(wv({p, q}), Dv(q), Dv(p)));
  if (c.sigma.coef != 0.0) {
    add(t2, c.sigma.coef, vol(wx({SIG}), 0, 0), vol(wv({SIG}), 0, 0));
    for (int q : act)
      add(t3, c.sigma.coef * c.beta[q].coef, vol(wx({SIG, q}), Dx(q), 0), vol(wv({SIG, q}), Dv(q), 0));
  }
  // inflow boundary
  double mMt[2][2];
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 2; ++q) mMt[s][q] = -Mt[s][q];
  for (const InflowPart& ip : inflow_parts(c, d, mx, mv)) add(mMt, ip.scale, ip.x, ip.v);
  // merge equal factor pairs; index the distinct factors
  std::map<FactorSpec, int> xid, vid;
  std::map<std::pair<int, int>, int> tid;
  out = TermTable();
  for (const Raw& r : raw) {
    auto ix = xid.find(r.x);
    if (ix == xid.end()) { ix = xid.emplace(r.x, (int)out.xf.size()).first; out.xf.push_back(r.x); }
    auto iv = vid.find(r.v);
    if (iv == vid.end()) { iv = vid.emplace(r.v, (int)out.vf.size()).first; out.vf.push_back(r.v); }
    auto key = std::make_pair(ix->second, iv->second);
    auto it = tid.find(key);
    if (it == tid.end()) {
      Term t;
      for (int s = 0; s < 2; ++s)
        for (int q = 0; q < 2; ++q) t.tau[s][q] = r.tau[s][q];
      t.x = key.first;
      t.v = key.second;
      tid.emplace(key, (int)out.terms.size());
      out.terms.push_back(t);
    } else {
      for (int s = 0; s < 2; ++s)
        for (int q = 0; q < 2; ++q) out.terms[it->second].tau[s][q] += r.tau[s][q];
    }
  }
  // drop terms whose time coupling cancelled
  std::vector<Term> kept;
  for (const Term& t : out.terms) {
    double mx_ = 0.0;
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < 2; ++q) mx_ = std::max(mx_, std::fabs(t.tau[s][q]));
    if (mx_ > 0.0) kept.push_back(t);
  }
  out.terms = kept;
  return {};
}

}  // namespace sgdg
