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
// Coefficients with a time factor (beta_p = c_p t_p(t) ..., Sect. 4.2) keep
// the same Kronecker factors; their time couplings become Gauss sums over
// the strip (TauPart), recomputed per strip by strip_time_couplings.
#include <algorithm>
#include <cmath>
#include <map>

#include "internal.h"

namespace sgdg {

std::vector<InflowPart> inflow_parts(const sgdg_coeffs& c, int d, const sgdg_mesh& mx, const sgdg_mesh& mv,
                                     bool with_time) {
  // beta_p = cp tp(t) b_p(x) c_p(v); on the face y_ax = side of Omega_x
  // (p < d) or Omega_v (p >= d), beta . n = side cp tp b_p c_p < 0 where the
  // signs sc of cp tp, s1 of sc b_p and s2 of c_p satisfy side s1 s2 < 0;
  // each sign pair is one Kronecker pair with the sign restricted at cell or
  // face centroids.  Without a time factor sc = sign(cp); with one, both
  // values of sc give parts, each active at the times where it holds.
  std::vector<InflowPart> out;
  for (int p = 0; p < 2 * d; ++p) {
    if (c.beta[p].coef == 0.0) continue;
    const bool xface = p < d;
    const int ax = xface ? p : p - d;
    const sgdg_mesh& m = xface ? mx : mv;
    if (m.periodic && m.periodic[ax]) continue;
    const double cp = c.beta[p].coef;
    const bool timed = with_time && c.beta_t[p] != nullptr;
    const bool hx = c.beta[p].fx != nullptr, hv = c.beta[p].fv != nullptr;
    for (int sc : {1, -1}) {
      if (!timed && sc != (cp > 0 ? 1 : -1)) continue;
      for (int side = -1; side <= 1; side += 2)
        for (int s1 = 1; s1 >= -1; s1 -= 2) {
          const int s2 = -side * s1;
          InflowPart ip;
          ip.x.kind = xface ? 1 : 0;
          ip.v.kind = xface ? 0 : 1;
          // (cp tp) b_p has sign s1 where b_p has sign s1 sc
          const int sb = s1 * sc;
          if (hx) { ip.x.wfn = {p}; ip.x.restrict_ = {{p, sb}}; }
          else if (sb != 1) continue;
          if (hv) { ip.v.wfn = {p}; ip.v.restrict_ = {{p, s2}}; }
          else if (s2 != 1) continue;
          FactorSpec& F = xface ? ip.x : ip.v;
          F.face_axis = ax;
          F.face_side = side;
          ip.scale = side * cp;
          if (timed) { ip.gate_fn = p; ip.gate_sign = sc; }
          out.push_back(ip);
        }
    }
  }
  return out;
}

namespace {

// Exact time matrices of the Legendre basis on a strip of length dt
// (Eq. 10): M_t = dt diag(1, 1/3), T_t = [[0, 2], [0, 0]],
// C_t = [[0, 0], [0, 4/dt]], G_t = [[1, -1], [-1, 1]]; T^T is base TT.
void exact_base(int base, double dt, double (&B)[2][2]) {
  const double Mt[2][2] = {{dt, 0.0}, {0.0, dt / 3.0}};
  const double Tt[2][2] = {{0.0, 2.0}, {0.0, 0.0}};
  const double Ct[2][2] = {{0.0, 0.0}, {0.0, 4.0 / dt}};
  const double Gt[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 2; ++q)
      B[s][q] = base == TauPart::M ? Mt[s][q] : base == TauPart::T ? Tt[s][q] : base == TauPart::TT ? Tt[q][s]
              : base == TauPart::C ? Ct[s][q] : Gt[s][q];
}

}  // namespace

Status strip_time_couplings(TermTable& tt, double t0, double dt, int m,
                            const std::vector<std::pair<sgdg_tfn, void*>>& ft) {
  const bool timed = tt.time_dep;
  std::vector<double> x, w;
  if (timed) {
    if (m < 1 || m > 8) return {SGDG_EINVAL, "time_quad must be in 1..8"};
    gauss_rule01(m, x, w);
  }
  // time factors at the Gauss points of the strip
  std::vector<std::vector<double>> fv(ft.size());
  std::vector<double> tq(x.size());
  for (size_t q = 0; q < x.size(); ++q) tq[q] = t0 + x[q] * dt;
  for (size_t id = 0; id < ft.size() && timed; ++id) {
    fv[id].assign(x.size(), 1.0);
    if (ft[id].first) ft[id].first((int)x.size(), tq.data(), fv[id].data(), ft[id].second);
    for (double v : fv[id])
      if (!std::isfinite(v)) return {SGDG_EINVAL, "a time factor returned NaN or Inf"};
  }
  auto fval = [&](int id, size_t q) { return id < 0 || id >= (int)fv.size() ? 1.0 : fv[id][q]; };
  for (size_t k = 0; k < tt.terms.size(); ++k) {
    double tau[2][2] = {{0, 0}, {0, 0}};
    for (const TauPart& pt : tt.parts[k]) {
      double B[2][2];
      if (!timed || pt.base == TauPart::G) {
        exact_base(pt.base, dt, B);
      } else {
        B[0][0] = B[0][1] = B[1][0] = B[1][1] = 0.0;
        for (size_t q = 0; q < x.size(); ++q) {
          double g = w[q] * dt * fval(pt.f1, q) * fval(pt.f2, q);
          if (pt.gate_fn >= 0 && !(pt.gate_sign * pt.gate_coef * fval(pt.gate_fn, q) > 0.0)) g = 0.0;
          // Legendre basis at the point: eta = (1, 2x - 1), eta' = (0, 2/dt)
          const double e[2] = {1.0, 2.0 * x[q] - 1.0}, de[2] = {0.0, 2.0 / dt};
          for (int s = 0; s < 2; ++s)
            for (int r = 0; r < 2; ++r) {
              const double b = pt.base == TauPart::M ? e[s] * e[r] : pt.base == TauPart::T ? e[s] * de[r]
                             : pt.base == TauPart::TT ? de[s] * e[r] : de[s] * de[r];
              B[s][r] += g * b;
            }
        }
      }
      for (int s = 0; s < 2; ++s)
        for (int r = 0; r < 2; ++r) tau[s][r] += pt.scale * B[s][r];
    }
    for (int s = 0; s < 2; ++s)
      for (int r = 0; r < 2; ++r) tt.terms[k].tau[s][r] = tau[s][r];
  }
  return {};
}

Status build_terms(const sgdg_coeffs& c, int d, const sgdg_mesh& mx, const sgdg_mesh& mv,
                   double dt, double delta, TermTable& out) {
  // function ids: beta components 0..2d-1, sigma kSigmaFn
  const int SIG = kSigmaFn;
  bool timed = c.sigma_t != nullptr;
  for (int p = 0; p < 2 * d; ++p) timed = timed || c.beta_t[p] != nullptr;
  auto has_x = [&](int p) { return (p == SIG ? c.sigma.fx : c.beta[p].fx) != nullptr; };
  auto has_v = [&](int p) { return (p == SIG ? c.sigma.fv : c.beta[p].fv) != nullptr; };
  auto Dx = [&](int p) { return p < d ? p + 1 : 0; };
  auto Dv = [&](int p) { return p >= d ? p - d + 1 : 0; };

  struct Raw { std::vector<TauPart> parts; FactorSpec x, v; };
  std::vector<Raw> raw;
  auto part = [](int base, double scale, int f1 = -1, int f2 = -1) {
    TauPart t;
    t.base = base;
    t.scale = scale;
    t.f1 = f1;
    t.f2 = f2;
    return t;
  };
  auto add = [&](std::vector<TauPart> parts, FactorSpec x, FactorSpec v) {
    std::sort(x.wfn.begin(), x.wfn.end());
    std::sort(v.wfn.begin(), v.wfn.end());
    std::sort(x.restrict_.begin(), x.restrict_.end());
    std::sort(v.restrict_.begin(), v.restrict_.end());
    raw.push_back({parts, x, v});
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
  using TP = TauPart;
  // (T_t + d C_t + G_t) (x) M (x) M
  add({part(TP::T, 1.0), part(TP::C, delta), part(TP::G, 1.0)}, vol({}, 0, 0), vol({}, 0, 0));
  // d T_t (x) [phi_j, c_q fx_q D_q phi_i]
  for (int q : act) add({part(TP::T, delta * c.beta[q].coef, q)}, vol(wx({q}), Dx(q), 0), vol(wv({q}), Dv(q), 0));
  // (M_t + d T_t^T) (x) [c_p fx_p D_p phi_j, phi_i]
  for (int p : act)
    add({part(TP::M, c.beta[p].coef, p), part(TP::TT, delta * c.beta[p].coef, p)}, vol(wx({p}), 0, Dx(p)),
        vol(wv({p}), 0, Dv(p)));
  // d M_t (x) [c_p c_q D_p phi_j, D_q phi_i]
  for (int p : act)
    for (int q : act)
      add({part(TP::M, delta * c.beta[p].coef * c.beta[q].coef, p, q)}, vol(wx({p, q}), Dx(q), Dx(p)),
          vol(wv({p, q}), Dv(q), Dv(p)));
  if (c.sigma.coef != 0.0) {
    // (M_t + d T_t^T) (x) [sigma phi_j, phi_i];  d M_t (x) [sigma phi_j, c_q D_q phi_i]
    add({part(TP::M, c.sigma.coef, SIG), part(TP::TT, delta * c.sigma.coef, SIG)}, vol(wx({SIG}), 0, 0),
        vol(wv({SIG}), 0, 0));
    for (int q : act)
      add({part(TP::M, delta * c.sigma.coef * c.beta[q].coef, SIG, q)}, vol(wx({SIG, q}), Dx(q), 0),
          vol(wv({SIG, q}), Dv(q), 0));
  }
  // inflow boundary: -M_t (x) G per part, its time factor and sign gate
  for (const InflowPart& ip : inflow_parts(c, d, mx, mv, timed)) {
    TauPart t = part(TP::M, -ip.scale, ip.gate_fn >= 0 ? ip.gate_fn : -1);
    if (ip.gate_fn >= 0) {
      t.gate_fn = ip.gate_fn;
      t.gate_sign = ip.gate_sign;
      t.gate_coef = c.beta[ip.gate_fn].coef;
    }
    add({t}, ip.x, ip.v);
  }
  // merge equal factor pairs; index the distinct factors
  std::map<FactorSpec, int> xid, vid;
  std::map<std::pair<int, int>, int> tid;
  out = TermTable();
  out.time_dep = timed;
  for (const Raw& r : raw) {
    auto ix = xid.find(r.x);
    if (ix == xid.end()) { ix = xid.emplace(r.x, (int)out.xf.size()).first; out.xf.push_back(r.x); }
    auto iv = vid.find(r.v);
    if (iv == vid.end()) { iv = vid.emplace(r.v, (int)out.vf.size()).first; out.vf.push_back(r.v); }
    auto key = std::make_pair(ix->second, iv->second);
    auto it = tid.find(key);
    if (it == tid.end()) {
      Term t{};
      t.x = key.first;
      t.v = key.second;
      tid.emplace(key, (int)out.terms.size());
      out.terms.push_back(t);
      out.parts.push_back(r.parts);
    } else {
      auto& ps = out.parts[it->second];
      ps.insert(ps.end(), r.parts.begin(), r.parts.end());
    }
  }
  // the time couplings of the first strip (exact time matrices without time
  // factors); time-constant terms whose coupling cancelled are dropped
  Status st = strip_time_couplings(out, 0.0, dt, 3, {});
  if (st.code) return st;
  if (!timed) {
    std::vector<Term> kept;
    std::vector<std::vector<TauPart>> kparts;
    for (size_t k = 0; k < out.terms.size(); ++k) {
      double mx_ = 0.0;
      for (int s = 0; s < 2; ++s)
        for (int q = 0; q < 2; ++q) mx_ = std::max(mx_, std::fabs(out.terms[k].tau[s][q]));
      if (mx_ > 0.0) { kept.push_back(out.terms[k]); kparts.push_back(out.parts[k]); }
    }
    out.terms = kept;
    out.parts = kparts;
  }
  return {};
}

}  // namespace sgdg
