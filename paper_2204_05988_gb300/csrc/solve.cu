// Strip solve on the GPU (Sect. 4.3): right-preconditioned FGMRES on the
// sparse-grid system A^(delta) u = b (Eq. 21) with the combination technique
// of Algorithm 1 as the preconditioner.  Each component system A_{l,l} (Eq. 22)
// is solved by GMRES preconditioned with the inverse of
// (T_t + delta C_t + G_t) (x) M^(1)_{l1} (x) M^(2)_{l2}; the mass inverses are
// applied by a fixed number of Chebyshev-Jacobi steps (a fixed linear
// operator, using the element bounds of D^{-1} M for P1 elements:
// [1/2, 3/2] on intervals, [1/2, 2] on triangles).
//
// Krylov scalars (dot products, norms, Givens rotations) are FP64.  In mixed
// mode the applies and component solves run in FP32 and every restart of the
// outer FGMRES recomputes the true residual b - A u with the FP64 apply, i.e.
// restarted FGMRES is iterative refinement with an FP32 correction solver.
#include <chrono>
#include <cmath>

#include "handle.h"

namespace sgdg {

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

namespace {

constexpr int kThreads = 256;
constexpr int kMaxKrylov = 64;

template <typename T>
__global__ void k_cheb_init(long long npts, int n2, int dim, const T* dinv, const T* f, T* r, T* d, T* x, double c) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    long long k1 = i / n2, k2 = i - k1 * n2;
    double di = (double)dinv[dim == 1 ? k1 : k2];
    for (int s = 0; s < 2; ++s) {
      double fr = (double)f[2 * i + s];
      double dd = c * di * fr;
      r[2 * i + s] = (T)fr;
      d[2 * i + s] = (T)dd;
      x[2 * i + s] = (T)dd;
    }
  }
}

template <typename T>
__global__ void k_cheb_step(long long npts, int n2, int dim, const T* dinv, const T* Md, T* r, T* d, T* x, double c1,
                            double c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    long long k1 = i / n2, k2 = i - k1 * n2;
    double di = (double)dinv[dim == 1 ? k1 : k2];
    for (int s = 0; s < 2; ++s) {
      double rr = (double)r[2 * i + s] - (double)Md[2 * i + s];
      double dd = c1 * (double)d[2 * i + s] + c2 * di * rr;
      r[2 * i + s] = (T)rr;
      d[2 * i + s] = (T)dd;
      x[2 * i + s] = (T)((double)x[2 * i + s] + dd);
    }
  }
}

__global__ void k_expand(long long npts, const double* U, double* v, double e0, double e1) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
    v[2 * i] = e0 * U[i];
    v[2 * i + 1] = e1 * U[i];
  }
}
__global__ void k_endpoint(long long npts, const double* u, double* U, double e0, double e1) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x)
    U[i] = e0 * u[2 * i] + e1 * u[2 * i + 1];
}

int gridsz(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  long long cap = (long long)num_sms() * 8;
  return (int)std::max(1LL, std::min(b, cap));
}

}  // namespace

// Krylov workspace for one storage type.
template <typename T>
struct KrylovWs {
  int m = 0;
  long long n = 0;
  T* V = nullptr;     // (m+1) x n
  T* Z = nullptr;     // m x n (flexible only)
  T* t0 = nullptr;    // n
  T* t1 = nullptr;
  T* ch[4] = {nullptr, nullptr, nullptr, nullptr};   // Chebyshev x, r, d, Md
};

struct Workspace {
  int nb = 0;                 // blocks of the multi-dot
  double* part = nullptr;     // kMaxKrylov+2 x nb
  double* dev_dots = nullptr; // 3 * (kMaxKrylov + 2)
  double* host = nullptr;     // pinned
  KrylovWs<double> outer;
  KrylovWs<double> in64;
  KrylovWs<float> in32;
  // CT buffers
  void* ct_x = nullptr;       // solutions of all CT grids (both precisions: max bytes)
  void* ct_b = nullptr;       // restricted rhs of a lower grid
  float* r32 = nullptr;       // mixed: residual / direction in FP32
  float* z32 = nullptr;
  long long nmax_grid = 0;    // largest CT grid (elements with time index)
  std::vector<int> cl1, cl2;  // CT grids: upper l = 0..L then lower l = 0..L-1
  std::vector<long long> coff;
};

namespace {

template <typename T>
KrylovWs<T>& inner_ws(Workspace& w);
template <> KrylovWs<double>& inner_ws<double>(Workspace& w) { return w.in64; }
template <> KrylovWs<float>& inner_ws<float>(Workspace& w) { return w.in32; }

// dots[0..k-1] = V_i . w (device), via deterministic block partials
template <typename T>
Status mdot(Handle& h, int k, const T* V, long long ldv, const T* w, long long n, double* out, cudaStream_t s) {
  Workspace& ws = *h.ws;
  SG_CU(vec_multidot<T>(k, V, ldv, w, n, ws.part, ws.nb, s));
  SG_CU(reduce_parts(k, ws.part, ws.nb, out, s));
  return {};
}

// Arnoldi step: orthogonalise w against V_0..V_j (CGS2), normalise into V_{j+1}.
// Returns the new Hessenberg column hcol[0..j+1] on the host.
template <typename T>
Status arnoldi(Handle& h, T* V, long long n, int j, T* w, double* hcol, cudaStream_t s) {
  Workspace& ws = *h.ws;
  double* d = ws.dev_dots;
  SG_ST(mdot<T>(h, j + 1, V, n, w, n, d, s));
  SG_CU(vec_multiaxpy<T>(j + 1, V, n, d, w, n, s));
  SG_ST(mdot<T>(h, j + 1, V, n, w, n, d + kMaxKrylov, s));
  SG_CU(vec_multiaxpy<T>(j + 1, V, n, d + kMaxKrylov, w, n, s));
  SG_ST(mdot<T>(h, 1, w, n, w, n, d + 2 * kMaxKrylov, s));
  SG_CU(cudaMemcpyAsync(ws.host, d, sizeof(double) * 3 * kMaxKrylov, cudaMemcpyDeviceToHost, s));
  SG_CU(cudaStreamSynchronize(s));
  for (int i = 0; i <= j; ++i) hcol[i] = ws.host[i] + ws.host[kMaxKrylov + i];
  double nrm = std::sqrt(std::max(0.0, ws.host[2 * kMaxKrylov]));
  hcol[j + 1] = nrm;
  if (!std::isfinite(nrm)) return {SGDG_ENAN, "NaN/Inf in Krylov vector"};
  if (nrm > 0.0) SG_CU(vec_axpby<T>(n, 1.0 / nrm, w, 0.0, w, s));
  return {};
}

template <typename T>
Status vnorm(Handle& h, const T* x, long long n, double* out, cudaStream_t s) {
  Workspace& ws = *h.ws;
  SG_ST(mdot<T>(h, 1, x, n, x, n, ws.dev_dots, s));
  SG_CU(cudaMemcpyAsync(ws.host, ws.dev_dots, sizeof(double), cudaMemcpyDeviceToHost, s));
  SG_CU(cudaStreamSynchronize(s));
  *out = std::sqrt(std::max(0.0, ws.host[0]));
  if (!std::isfinite(*out)) return {SGDG_ENAN, "NaN/Inf in a residual"};
  return {};
}

// Givens QR of the Hessenberg matrix, column by column.
struct Givens {
  double H[kMaxKrylov + 1][kMaxKrylov];
  double cs[kMaxKrylov], sn[kMaxKrylov], g[kMaxKrylov + 1];
  void start(double beta) {
    for (int i = 0; i <= kMaxKrylov; ++i) g[i] = 0.0;
    g[0] = beta;
  }
  // returns |residual estimate|
  double add(int j, const double* hcol) {
    for (int i = 0; i <= j + 1; ++i) H[i][j] = hcol[i];
    for (int i = 0; i < j; ++i) {
      double t = cs[i] * H[i][j] + sn[i] * H[i + 1][j];
      H[i + 1][j] = -sn[i] * H[i][j] + cs[i] * H[i + 1][j];
      H[i][j] = t;
    }
    double rho = std::hypot(H[j][j], H[j + 1][j]);
    if (rho == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
    else { cs[j] = H[j][j] / rho; sn[j] = H[j + 1][j] / rho; }
    H[j][j] = rho;
    H[j + 1][j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    return std::fabs(g[j + 1]);
  }
  void solve(int k, double* y) {
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < k; ++q) s -= H[i][q] * y[q];
      y[i] = H[i][i] != 0.0 ? s / H[i][i] : 0.0;
    }
  }
};

// Chebyshev-Jacobi approximation of M^{-1} along one dimension, in place on x.
template <typename T>
Status cheb_dim(Handle& h, int dim, int lev, int n1, int n2, const T* f, T* out, cudaStream_t s) {
  KrylovWs<T>& W = inner_ws<T>(*h.ws);
  const int K = std::max(1, h.cfg.cheb_steps);
  const double a = 0.5, b = (h.d == 1) ? 1.5 : 2.0;
  const double theta = 0.5 * (a + b), del = 0.5 * (b - a), sigma1 = theta / del;
  SideDev& sd = dim == 1 ? h.X : h.V;
  const T* dinv = sd.vals<T>().dinv[lev];
  const long long npts = (long long)n1 * n2;
  T *x = out, *r = W.ch[1], *d = W.ch[2], *Md = W.ch[3];
  k_cheb_init<T><<<gridsz(npts), kThreads, 0, s>>>(npts, n2, dim, dinv, f, r, d, x, 1.0 / theta);
  SG_CU(cudaGetLastError());
  double rho = 1.0 / sigma1;
  for (int k = 1; k < K; ++k) {
    SpmmLaunch<T> A;
    A.ngrids = 1;
    A.nterms = 1;
    A.identity = 1;
    A.accumulate = 0;
    SpmmGrid<T>& G = A.g[0];
    G.in = d; G.in2 = nullptr; G.out = Md;
    G.n1_in = G.n1_out = n1; G.n2_in = G.n2_out = n2;
    G.rowptr = sd.rowptr[lev]; G.col = sd.col[lev]; G.val[0] = sd.vals<T>().fac[sd.mass][lev];
    if (dim == 1) SG_CU(launch_left(A, s)); else SG_CU(launch_right(A, s));
    double rhon = 1.0 / (2.0 * sigma1 - rho);
    k_cheb_step<T><<<gridsz(npts), kThreads, 0, s>>>(npts, n2, dim, dinv, Md, r, d, x, rhon * rho, 2.0 * rhon / del);
    SG_CU(cudaGetLastError());
    rho = rhon;
  }
  return {};
}

// out = ((T_t + delta C_t + G_t)^{-1} (x) M1^{-1} (x) M2^{-1}) v on grid (l1, l2); v intact.
template <typename T>
Status precond_grid(Handle& h, int l1, int l2, const T* v, T* out, cudaStream_t s) {
  KrylovWs<T>& W = inner_ws<T>(*h.ws);
  const int n1 = h.X.n[l1], n2 = h.V.n[l2];
  const long long npts = (long long)n1 * n2;
  const double dt = h.cfg.dt, dl = h.cfg.delta;
  // P_t = [[1, 1], [-1, 1 + 4 delta / dt]]
  const double p00 = 1.0, p01 = 1.0, p10 = -1.0, p11 = 1.0 + 4.0 * dl / dt;
  const double det = p00 * p11 - p01 * p10;
  const double inv[4] = {p11 / det, -p01 / det, -p10 / det, p00 / det};
  T* t = W.ch[0];
  SG_CU(vec_time2x2<T>(npts, inv, v, out, s));
  SG_ST(cheb_dim<T>(h, 1, l1, n1, n2, out, t, s));
  SG_ST(cheb_dim<T>(h, 2, l2, n1, n2, t, out, s));
  return {};
}

// GMRES(m) on A_{l,l} x = b (one restart cycle, x0 = 0), right preconditioned.
template <typename T>
Status component_solve(Handle& h, int l1, int l2, const T* b, T* x, cudaStream_t s, int* its) {
  KrylovWs<T>& W = inner_ws<T>(*h.ws);
  const long long n = 2LL * h.X.n[l1] * h.V.n[l2];
  const int m = std::min(h.cfg.inner_its, W.m);
  double beta;
  SG_ST(vnorm<T>(h, b, n, &beta, s));
  if (beta == 0.0) {
    SG_CU(vec_fill<T>(x, n, (T)0, s));
    return {};
  }
  static thread_local Givens G;
  G.start(beta);
  SG_CU(vec_axpby<T>(n, 1.0 / beta, b, 0.0, W.V, s));
  double hcol[kMaxKrylov + 1];
  int k = 0;
  for (int j = 0; j < m; ++j) {
    T* Vj = W.V + (long long)j * n;
    T* Vn = W.V + (long long)(j + 1) * n;
    SG_ST(precond_grid<T>(h, l1, l2, Vj, W.t0, s));
    const T* uin[1] = {W.t0};
    T* yout[1] = {Vn};
    SG_ST(apply_diag_grids<T>(h, 1, &l1, &l2, uin, yout, s));
    SG_ST(arnoldi<T>(h, W.V, n, j, Vn, hcol, s));
    double res = G.add(j, hcol);
    k = j + 1;
    if (res <= h.cfg.inner_rtol * beta || hcol[j + 1] == 0.0) break;
  }
  double y[kMaxKrylov];
  G.solve(k, y);
  double* dy = h.ws->dev_dots;
  SG_CU(cudaMemcpyAsync(dy, y, sizeof(double) * k, cudaMemcpyHostToDevice, s));
  SG_CU(vec_combine<T>(k, W.V, n, dy, 0.0, W.t1, n, s));
  SG_ST(precond_grid<T>(h, l1, l2, W.t1, x, s));
  SG_CU(cudaStreamSynchronize(s));   // dy (pageable source) must stay valid
  if (its) *its += k;
  return {};
}

template <typename T>
Status ct_apply(Handle& h, const T* r, T* z, cudaStream_t s, int* its) {
  Workspace& ws = *h.ws;
  const int L = h.L;
  T* X = (T*)ws.ct_x;
  T* B = (T*)ws.ct_b;
  // upper grids (l, L-l)
  for (int l = 0; l <= L; ++l) SG_ST(component_solve<T>(h, l, L - l, r + h.off[l], X + ws.coff[l], s, its));
  // lower grids (l, L-1-l): residual restricted in dim 1 from grid (l+1, L-1-l)
  for (int l = 0; l < L; ++l) {
    SpmmLaunch<T> a;
    a.ngrids = 1; a.nterms = 1; a.identity = 1; a.accumulate = 0;
    SpmmGrid<T>& G = a.g[0];
    G.in = r + h.off[l + 1]; G.in2 = nullptr; G.out = B;
    G.n1_in = h.n1[l + 1]; G.n2_in = G.n2_out = h.n2[l + 1]; G.n1_out = h.X.n[l];
    G.rowptr = h.X.R_rowptr[l]; G.col = h.X.R_col[l]; G.val[0] = h.X.vals<T>().R[l];
    SG_CU(launch_left(a, s));
    SG_ST(component_solve<T>(h, l, L - 1 - l, B, X + ws.coff[L + 1 + l], s, its));
  }
  // combination: z_l = dhat_l - (E^(1) (x) Id) dhat_(l-1, L-l)
  SG_CU(cudaMemcpyAsync(z, X, sizeof(T) * h.n_coeffs, cudaMemcpyDeviceToDevice, s));
  for (int l = 1; l <= L; ++l) {
    SpmmLaunch<T> a;
    a.ngrids = 1; a.nterms = 1; a.identity = 0; a.accumulate = 1;
    a.tau[0][0] = (T)-1; a.tau[0][1] = 0; a.tau[0][2] = 0; a.tau[0][3] = (T)-1;
    SpmmGrid<T>& G = a.g[0];
    G.in = X + ws.coff[L + 1 + (l - 1)]; G.in2 = nullptr; G.out = z + h.off[l];
    G.n1_in = h.X.n[l - 1]; G.n2_in = G.n2_out = h.n2[l]; G.n1_out = h.n1[l];
    G.rowptr = h.X.E_rowptr[l - 1]; G.col = h.X.E_col[l - 1]; G.val[0] = h.X.vals<T>().E[l - 1];
    SG_CU(launch_left(a, s));
  }
  return {};
}

template <typename T>
Status alloc_krylov(Handle& h, KrylovWs<T>& W, int m, long long n, bool flexible, bool cheb) {
  W.m = m;
  W.n = n;
  if (dev_alloc(h, (void**)&W.V, sizeof(T) * (size_t)(m + 1) * n) != cudaSuccess) return {SGDG_ENOMEM, "Krylov basis"};
  if (flexible && dev_alloc(h, (void**)&W.Z, sizeof(T) * (size_t)m * n) != cudaSuccess)
    return {SGDG_ENOMEM, "Krylov basis"};
  if (dev_alloc(h, (void**)&W.t0, sizeof(T) * n) != cudaSuccess ||
      dev_alloc(h, (void**)&W.t1, sizeof(T) * n) != cudaSuccess)
    return {SGDG_ENOMEM, "Krylov temporaries"};
  if (cheb)
    for (int i = 0; i < 4; ++i)
      if (dev_alloc(h, (void**)&W.ch[i], sizeof(T) * n) != cudaSuccess) return {SGDG_ENOMEM, "Chebyshev temporaries"};
  return {};
}

}  // namespace

Status solver_init(Handle& h) {
  if (h.ws) return {};
  h.ws = new Workspace();
  Workspace& ws = *h.ws;
  const int L = h.L;
  ws.nb = num_sms() * 2;
  if (dev_alloc(h, (void**)&ws.part, sizeof(double) * (kMaxKrylov + 2) * ws.nb) != cudaSuccess ||
      dev_alloc(h, (void**)&ws.dev_dots, sizeof(double) * 3 * (kMaxKrylov + 2)) != cudaSuccess)
    return {SGDG_ENOMEM, "Krylov scalars"};
  if (cudaMallocHost((void**)&ws.host, sizeof(double) * 3 * (kMaxKrylov + 2)) != cudaSuccess)
    return {SGDG_ENOMEM, "pinned host scalars"};
  // CT grids
  long long tot = 0;
  for (int l = 0; l <= L; ++l) { ws.cl1.push_back(l); ws.cl2.push_back(L - l); }
  for (int l = 0; l < L; ++l) { ws.cl1.push_back(l); ws.cl2.push_back(L - 1 - l); }
  for (size_t g = 0; g < ws.cl1.size(); ++g) {
    long long n = 2LL * h.X.n[ws.cl1[g]] * h.V.n[ws.cl2[g]];
    ws.coff.push_back(tot);
    tot += n;
    ws.nmax_grid = std::max(ws.nmax_grid, n);
  }
  const bool mixed = h.cfg.precision == SGDG_MIXED_FP32;
  size_t esz = mixed ? sizeof(float) : sizeof(double);
  if (dev_alloc(h, &ws.ct_x, esz * (size_t)tot) != cudaSuccess ||
      dev_alloc(h, &ws.ct_b, esz * (size_t)ws.nmax_grid) != cudaSuccess)
    return {SGDG_ENOMEM, "CT buffers"};
  const int mi = std::max(1, std::min(h.cfg.inner_its, kMaxKrylov - 1));
  if (mixed) {
    SG_ST(alloc_krylov<float>(h, ws.in32, mi, ws.nmax_grid, false, true));
    if (dev_alloc(h, (void**)&ws.r32, sizeof(float) * h.n_coeffs) != cudaSuccess ||
        dev_alloc(h, (void**)&ws.z32, sizeof(float) * h.n_coeffs) != cudaSuccess)
      return {SGDG_ENOMEM, "mixed-precision buffers"};
  } else {
    SG_ST(alloc_krylov<double>(h, ws.in64, mi, ws.nmax_grid, false, true));
  }
  const int mo = std::max(1, std::min(h.cfg.restart, kMaxKrylov - 1));
  SG_ST(alloc_krylov<double>(h, ws.outer, mo, h.n_coeffs, true, false));
  return {};
}

Status ct_precondition(Handle& h, const double* r, double* z, cudaStream_t s, int* its) {
  SG_ST(solver_init(h));
  Workspace& ws = *h.ws;
  if (h.cfg.precision == SGDG_MIXED_FP32) {
    SG_CU((vec_convert<double, float>(r, ws.r32, h.n_coeffs, s)));
    SG_ST(ct_apply<float>(h, ws.r32, ws.z32, s, its));
    SG_CU((vec_convert<float, double>(ws.z32, z, h.n_coeffs, s)));
    return {};
  }
  return ct_apply<double>(h, r, z, s, its);
}

// w = A z in the configured precision (FP64 storage in and out).
static Status apply_mixed(Handle& h, const double* z, double* w, bool force64, cudaStream_t s) {
  if (force64 || h.cfg.precision == SGDG_FP64) return apply_plan<double>(h, h.op, z, w, s);
  Workspace& ws = *h.ws;
  SG_CU((vec_convert<double, float>(z, ws.r32, h.n_coeffs, s)));
  SG_ST(apply_plan<float>(h, h.op, ws.r32, ws.z32, s));
  SG_CU((vec_convert<float, double>(ws.z32, w, h.n_coeffs, s)));
  return {};
}

Status advance_strip(Handle& h, cudaStream_t s, sgdg_strip_stats* st, bool resolve) {
  auto t0 = std::chrono::steady_clock::now();
  SG_ST(solver_init(h));
  Workspace& ws = *h.ws;
  KrylovWs<double>& O = ws.outer;
  const long long n = h.n_coeffs;
  if (!h.have_initial) return {SGDG_EINVAL, "sgdg_set_initial was not called"};
  if (resolve && !h.solved) return {SGDG_EINVAL, "no strip has been solved yet"};
  // right-hand side: eta(t_{j-1}^+) (x) M_sg U^-_{j-1}; the first strip uses (u0, phi);
  // a re-solve keeps the right-hand side of the strip
  if (!resolve && !h.first_strip) {
    k_expand<<<gridsz(h.n_spatial), kThreads, 0, s>>>(h.n_spatial, h.U_end, O.t0, 1.0, -1.0);
    SG_CU(cudaGetLastError());
    SG_ST(apply_plan<double>(h, h.mass, O.t0, h.rhs, s));
  }
  sgdg_strip_stats S{};
  double bnorm;
  SG_ST(vnorm<double>(h, h.rhs, n, &bnorm, s));
  double* x = h.u_sol;
  double* r = O.t1;
  // initial guess: the last solution (re-solve, warm start 1), a given guess
  // (2), the linear extrapolation 2 u_{j-1} - u_{j-2} of the last two strip
  // solutions (3) or zero; u_prev2 keeps u_{j-1} for the next extrapolation
  const int mode = resolve ? 1 : h.warm;
  double beta = bnorm;
  if (mode == 2 && !h.guess) return {SGDG_EINVAL, "warm start 2 needs sgdg_set_guess"};
  if (!resolve && h.solved) {
    if (!h.u_prev2 && dev_alloc(h, (void**)&h.u_prev2, sizeof(double) * n) != cudaSuccess)
      return {SGDG_ENOMEM, "previous solution buffer"};
    SG_CU(cudaMemcpyAsync(O.t0, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (mode == 3 && h.nsolved >= 2) SG_CU(vec_axpby<double>(n, -1.0, h.u_prev2, 2.0, x, s));
    SG_CU(cudaMemcpyAsync(h.u_prev2, O.t0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  if (mode == 2) SG_CU(cudaMemcpyAsync(x, h.guess, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if (((mode == 1 || mode == 3) && h.solved) || mode == 2) {
    SG_ST(apply_plan<double>(h, h.op, x, r, s));
    S.applies++;
    SG_CU(vec_axpby<double>(n, 1.0, h.rhs, -1.0, r, s));
    SG_ST(vnorm<double>(h, r, n, &beta, s));
  } else {
    SG_CU(vec_fill<double>(x, n, 0.0, s));
    SG_CU(cudaMemcpyAsync(r, h.rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  S.initial_rel_residual = bnorm > 0.0 ? beta / bnorm : 0.0;
  const double tol = h.cfg.rtol * bnorm;
  static thread_local Givens G;
  double hcol[kMaxKrylov + 1], y[kMaxKrylov];
  int total = 0;
  Status res{};
  // mixed mode: one restart cycle is one refinement step; it stops once its
  // FP32-level Krylov estimate has gained kRefineGain (the FP32 apply bounds
  // what one cycle can resolve), then the FP64 residual restarts it
  const bool mixed = h.cfg.precision == SGDG_MIXED_FP32;
  const double kRefineGain = 1e-4;
  while (beta > tol && total < h.cfg.max_outer && bnorm > 0.0) {
    G.start(beta);
    SG_CU(vec_axpby<double>(n, 1.0 / beta, r, 0.0, O.V, s));
    const double cycle_tol = mixed ? std::max(tol, kRefineGain * beta) : tol;
    int k = 0;
    for (int j = 0; j < O.m && total < h.cfg.max_outer; ++j) {
      double* Vj = O.V + (long long)j * n;
      double* Zj = O.Z + (long long)j * n;
      double* Vn = O.V + (long long)(j + 1) * n;
      SG_ST(ct_precondition(h, Vj, Zj, s, &S.inner_its_total));
      SG_ST(apply_mixed(h, Zj, Vn, false, s));
      S.applies++;
      SG_ST(arnoldi<double>(h, O.V, n, j, Vn, hcol, s));
      double est = G.add(j, hcol);
      k = j + 1;
      total++;
      if (est <= cycle_tol || hcol[j + 1] == 0.0) break;
    }
    G.solve(k, y);
    SG_CU(cudaMemcpyAsync(ws.dev_dots, y, sizeof(double) * k, cudaMemcpyHostToDevice, s));
    SG_CU(vec_combine<double>(k, O.Z, n, ws.dev_dots, 1.0, x, n, s));
    // true residual in FP64 (iterative refinement in mixed mode)
    SG_ST(apply_plan<double>(h, h.op, x, r, s));
    S.applies++;
    SG_CU(vec_axpby<double>(n, 1.0, h.rhs, -1.0, r, s));
    SG_ST(vnorm<double>(h, r, n, &beta, s));
  }
  S.outer_its = total;
  S.rel_residual = bnorm > 0.0 ? beta / bnorm : 0.0;
  if (beta > tol && bnorm > 0.0) S.status = SGDG_ENOCONV;
  // end value U^-_j = sum_s eta_s(t_j^-) u_s = u_0 + u_1
  k_endpoint<<<gridsz(h.n_spatial), kThreads, 0, s>>>(h.n_spatial, x, h.U_end, 1.0, 1.0);
  SG_CU(cudaGetLastError());
  SG_CU(cudaStreamSynchronize(s));
  h.first_strip = false;
  h.solved = true;
  if (!resolve) h.nsolved++;
  S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = S;
  if (S.status == SGDG_ENOCONV) return {SGDG_ENOCONV, "outer FGMRES reached max_outer"};
  return res;
}

Handle::~Handle() {}

void solver_free(Handle& h) {
  if (!h.ws) return;
  if (h.ws->host) cudaFreeHost(h.ws->host);
  delete h.ws;
  h.ws = nullptr;
}

}  // namespace sgdg
