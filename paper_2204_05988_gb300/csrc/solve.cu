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

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };

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

// Workspace of the lockstep component solves: per CT grid g a Krylov basis
// (m+1 vectors), the preconditioner output t0, the combined correction t1
// and four Chebyshev vectors, slices of one arena.
template <typename T>
struct CtBatch {
  int m = 0;
  T* arena = nullptr;
  std::vector<T*> V, t0, t1, cx, cr, cd, cm;
  double* part = nullptr;   // grouped partial sums: grid x (kMaxKrylov + 2) x nbg
  double* dots = nullptr;   // grid x 3 x kMaxKrylov (device)
  double* host = nullptr;   // pinned mirror of dots
  double* y = nullptr;      // grid x kMaxKrylov (device), Givens solutions
  double* yh = nullptr;     // pinned staging of y
};

struct Workspace {
  int nb = 0;                 // blocks of the multi-dot
  double* part = nullptr;     // kMaxKrylov+2 x nb
  double* dev_dots = nullptr; // 3 * (kMaxKrylov + 2)
  double* host = nullptr;     // pinned
  KrylovWs<double> outer;
  CtBatch<double> ct64;       // batched component solves (the configured inner precision)
  CtBatch<float> ct32;
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
CtBatch<T>& ct_ws(Workspace& w);
template <> CtBatch<double>& ct_ws<double>(Workspace& w) { return w.ct64; }
template <> CtBatch<float>& ct_ws<float>(Workspace& w) { return w.ct32; }

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
// sqrt of a reduced squared norm; NaN stays NaN (std::max(0.0, NaN) would
// return 0.0 and hide it from the finiteness checks)
inline double norm_of(double sq) { return std::isnan(sq) ? sq : std::sqrt(std::max(0.0, sq)); }

template <typename T>
Status arnoldi(Handle& h, T* V, long long n, int j, T* w, double* hcol, cudaStream_t s) {
  NvtxRange range("sgdg.orth");
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
  double nrm = norm_of(ws.host[2 * kMaxKrylov]);
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
  *out = norm_of(ws.host[0]);
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

// ---------------------------------------------------------------------------
// Lockstep component solves (Algorithm 1): the 2L+1 CT systems are
// independent, so their GMRES iterations advance together.  Every vector
// operation of one inner step is one grouped launch over the active grids
// (blockIdx.y = grid); the diagonal-block applies are queued grid by grid
// without host synchronisation; the Hessenberg columns of all grids come
// back in one copy per step.
// ---------------------------------------------------------------------------

constexpr int kGroupBlocks = 64;   // blocks per grid of the grouped reductions

// Pointers and sizes of up to kMaxGrids grids for the grouped kernels.
template <typename T>
struct GVec {
  int ng = 0;
  long long n[kMaxGrids];        // scalars of grid g (time index included)
  int n2[kMaxGrids];             // row length of grid g (pairs)
  int slot[kMaxGrids];           // the grid's index in the per-grid scalar arrays
  const T* a[kMaxGrids];
  T* b[kMaxGrids];
  T* c[kMaxGrids];
  T* d[kMaxGrids];
  T* e[kMaxGrids];
  const T* dinv[kMaxGrids];      // Chebyshev: inverse mass diagonal along the smoothed dimension
  long long ldv[kMaxGrids];      // stride of the Krylov basis
};

struct TimeInv {
  double m[4];
};

// Elementwise grouped kernels compute in the storage type T (FP32 in mixed
// mode: the component solves are FP32 there); only the dot products below
// accumulate in FP64.
template <typename T>
__global__ void k_gtime2x2(const __grid_constant__ GVec<T> p, TimeInv M) {
  using T2 = typename V2<T>::type;
  const int g = blockIdx.y;
  const unsigned npts = (unsigned)(p.n[g] / 2);
  const T2* x = reinterpret_cast<const T2*>(p.a[g]);
  T2* y = reinterpret_cast<T2*>(p.b[g]);
  const T m0 = (T)M.m[0], m1 = (T)M.m[1], m2 = (T)M.m[2], m3 = (T)M.m[3];
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += gridDim.x * blockDim.x) {
    const T2 v = x[i];
    T2 r;
    r.x = m0 * v.x + m1 * v.y;
    r.y = m2 * v.x + m3 * v.y;
    y[i] = r;
  }
}

// Chebyshev start on every grid: r = f, d = x = c D^{-1} f (a = f, b = r, c = d, d = x)
template <typename T>
__global__ void k_gcheb_init(const __grid_constant__ GVec<T> p, int dim, double c) {
  using T2 = typename V2<T>::type;
  const int g = blockIdx.y;
  const unsigned npts = (unsigned)(p.n[g] / 2);
  const unsigned n2 = (unsigned)p.n2[g];
  const T2* f = reinterpret_cast<const T2*>(p.a[g]);
  T2* r = reinterpret_cast<T2*>(p.b[g]);
  T2* d = reinterpret_cast<T2*>(p.c[g]);
  T2* x = reinterpret_cast<T2*>(p.d[g]);
  const T cc = (T)c;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += gridDim.x * blockDim.x) {
    const unsigned k1 = i / n2, k2 = i - k1 * n2;
    const T di = cc * p.dinv[g][dim == 1 ? k1 : k2];
    const T2 fr = f[i];
    T2 dd;
    dd.x = di * fr.x;
    dd.y = di * fr.y;
    r[i] = fr;
    d[i] = dd;
    x[i] = dd;
  }
}

// Fused Chebyshev step on every grid, the mass apply included:
//   r -= M d_old;  d_new = c1 d_old + c2 D^{-1} r;  x += d_new
// with M along dim 1 (rows k1) or dim 2 (rows k2) from its ELL rows (width W,
// zero padding); d ping-pongs between two buffers because neighbouring
// elements still read d_old.
template <typename T>
struct GCheb {
  int ng = 0;
  int n1[kMaxGrids], n2[kMaxGrids];
  const int* col[kMaxGrids];
  const T* val[kMaxGrids];
  const T* dinv[kMaxGrids];
  const T* dold[kMaxGrids];
  T* dnew[kMaxGrids];
  T* r[kMaxGrids];
  T* x[kMaxGrids];
};

template <typename T, bool DIM2, int W>
__global__ void __launch_bounds__(kThreads) k_gcheb_fused(const __grid_constant__ GCheb<T> p, double c1, double c2) {
  using T2 = typename V2<T>::type;
  const int g = blockIdx.y;
  const unsigned n1 = (unsigned)p.n1[g], n2 = (unsigned)p.n2[g];
  const unsigned npts = n1 * n2;
  const T2* dold = reinterpret_cast<const T2*>(p.dold[g]);
  T2* dnew = reinterpret_cast<T2*>(p.dnew[g]);
  T2* r = reinterpret_cast<T2*>(p.r[g]);
  T2* x = reinterpret_cast<T2*>(p.x[g]);
  const T a1 = (T)c1, a2 = (T)c2;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += gridDim.x * blockDim.x) {
    const unsigned k1 = i / n2, k2 = i - k1 * n2;
    const unsigned row = DIM2 ? k2 : k1;
    const int4* cq = reinterpret_cast<const int4*>(p.col[g] + (size_t)row * W);
    const T* vq = p.val[g] + (size_t)row * W;
    T2 m;
    m.x = m.y = 0;
#pragma unroll
    for (int q = 0; q < W / 4; ++q) {
      const int4 c = __ldg(cq + q);
      const int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const T v = __ldg(vq + 4 * q + e);
        const T2 dv = DIM2 ? dold[k1 * n2 + (unsigned)cc[e]] : dold[(unsigned)cc[e] * n2 + k2];
        m.x += v * dv.x;
        m.y += v * dv.y;
      }
    }
    const T di = a2 * p.dinv[g][row];
    T2 rr = r[i], dd = dold[i], xx = x[i];
    rr.x -= m.x;
    rr.y -= m.y;
    dd.x = a1 * dd.x + di * rr.x;
    dd.y = a1 * dd.y + di * rr.y;
    xx.x += dd.x;
    xx.y += dd.y;
    r[i] = rr;
    dnew[i] = dd;
    x[i] = xx;
  }
}

// part[(slot * (kMaxKrylov + 2) + i) * kGroupBlocks + block] = partial sum of
// V_i . w over the block's share (a = V base, b = w), for i < k; fixed order.
// The two time coefficients of a node are multiplied and added in T, the
// node sums accumulate in FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_gmultidot(const __grid_constant__ GVec<T> p, int k, double* part) {
  using T2 = typename V2<T>::type;
  const int g = blockIdx.y;
  const long long n = p.n[g] / 2;   // nodes (pairs)
  const T2* V = reinterpret_cast<const T2*>(p.a[g]);
  const T2* w = reinterpret_cast<const T2*>(p.b[g]);
  __shared__ double red[kThreads / 32];
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * per, hi = min(n, lo + per);
  for (int i = 0; i < k; ++i) {
    const T2* Vi = V + (long long)i * (p.ldv[g] / 2);
    double acc = 0.0;
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) {
      const T2 a = Vi[t], b = w[t];
      acc += (double)(a.x * b.x + a.y * b.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int q = 0; q < kThreads / 32; ++q) sum += red[q];
      part[((long long)p.slot[g] * (kMaxKrylov + 2) + i) * gridDim.x + blockIdx.x] = sum;
    }
    __syncthreads();
  }
}

// dots[slot * ld + off + i] = sum over blocks of part (fixed order), i < k
__global__ void k_greduce2(const __grid_constant__ GVec<double> p, int k, const double* part, int nbg, double* dots,
                           int ld, int off) {
  const int g = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const int slot = p.slot[g];
  const double* src = part + ((long long)slot * (kMaxKrylov + 2) + i) * nbg;
  double sum = 0.0;
  for (int b = 0; b < nbg; ++b) sum += src[b];
  dots[(long long)slot * ld + off + i] = sum;
}

// w -= sum_i h[slot * ld + off + i] V_i   (a = V base, b = w); coefficients
// rounded to T, accumulation in T
template <typename T>
__global__ void k_gmultiaxpy(const __grid_constant__ GVec<T> p, int k, const double* h, int ld, int off) {
  const int g = blockIdx.y;
  const long long n = p.n[g];
  const double* hg = h + (long long)p.slot[g] * ld + off;
  const T* V = p.a[g];
  const long long ldv = p.ldv[g];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    T acc = p.b[g][t];
    for (int i = 0; i < k; ++i) acc -= (T)hg[i] * V[(long long)i * ldv + t];
    p.b[g][t] = acc;
  }
}

// w *= 1 / sqrt(h[slot * ld + off]) when positive   (b = w)
template <typename T>
__global__ void k_gnormalize(const __grid_constant__ GVec<T> p, const double* h, int ld, int off) {
  const int g = blockIdx.y;
  const double nn = h[(long long)p.slot[g] * ld + off];
  if (!(nn > 0.0)) return;
  const T sc = (T)(1.0 / sqrt(nn));
  const long long n = p.n[g];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    p.b[g][t] *= sc;
}

// c = sum_i y[slot * ld + i] V_i   (a = V base, c = output), i < k[g] (in n2 of the descriptor)
template <typename T>
__global__ void k_gcombine(const __grid_constant__ GVec<T> p, const double* y, int ld) {
  const int g = blockIdx.y;
  const long long n = p.n[g];
  const int k = p.n2[g];
  const double* yg = y + (long long)p.slot[g] * ld;
  const T* V = p.a[g];
  const long long ldv = p.ldv[g];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    T acc = 0;
    for (int i = 0; i < k; ++i) acc += (T)yg[i] * V[(long long)i * ldv + t];
    p.c[g][t] = acc;
  }
}

// grid of a grouped elementwise launch: enough blocks for the largest grid, capped
inline dim3 ggrid(const long long* n, int ng) {
  long long mx = 1;
  for (int g = 0; g < ng; ++g) mx = std::max(mx, n[g]);
  long long b = (mx + kThreads - 1) / kThreads;
  const long long cap = std::max(1LL, (long long)num_sms() * 8 / std::max(1, ng) + 1);
  return dim3((unsigned)std::max(1LL, std::min(b, cap)), (unsigned)ng);
}

// The active grids of one lockstep step.
struct Active {
  std::vector<int> g;   // CT grid indices
};

// out_g = ((T_t + delta C_t + G_t)^{-1} (x) M1^{-1} (x) M2^{-1}) in_g on every
// active grid.  Uses cx, cr, cd, cm and t1 of each grid: in_g may be t1 (it is
// consumed first), out_g must be none of them.
template <typename T>
Status precond_group(Handle& h, const Active& act, const std::vector<const T*>& in, const std::vector<T*>& out,
                     cudaStream_t s) {
  Workspace& ws = *h.ws;
  CtBatch<T>& B = ct_ws<T>(ws);
  const int ng = (int)act.g.size();
  if (ng == 0) return {};
  const double dt = h.cfg.dt, dl = h.cfg.delta;
  // P_t = [[1, 1], [-1, 1 + 4 delta / dt]]
  const double p00 = 1.0, p01 = 1.0, p10 = -1.0, p11 = 1.0 + 4.0 * dl / dt;
  const double det = p00 * p11 - p01 * p10;
  TimeInv Minv;
  Minv.m[0] = p11 / det; Minv.m[1] = -p01 / det; Minv.m[2] = -p10 / det; Minv.m[3] = p00 / det;
  GVec<T> t;
  t.ng = ng;
  for (int q = 0; q < ng; ++q) {
    const int g = act.g[q];
    t.n[q] = 2LL * h.X.n[ws.cl1[g]] * h.V.n[ws.cl2[g]];
    t.a[q] = in[q];
    t.b[q] = B.cx[g];   // time-inverted input, smoothed along dim 1 next
  }
  k_gtime2x2<T><<<ggrid(t.n, ng), kThreads, 0, s>>>(t, Minv);
  SG_CU(cudaGetLastError());
  // Chebyshev-Jacobi along dim 1 (f = cx -> x = t1), then along dim 2 (f = t1 -> x = out)
  const int K = std::max(1, h.cfg.cheb_steps);
  const double a = 0.5, b = (h.d == 1) ? 1.5 : (h.d == 2 ? 2.0 : 2.5);
  const double theta = 0.5 * (a + b), del = 0.5 * (b - a), sigma1 = theta / del;
  for (int dim = 1; dim <= 2; ++dim) {
    GVec<T> c;
    c.ng = ng;
    for (int q = 0; q < ng; ++q) {
      const int g = act.g[q];
      const int l1 = ws.cl1[g], l2 = ws.cl2[g];
      const SideDev& sd = dim == 1 ? h.X : h.V;
      const int lev = dim == 1 ? l1 : l2;
      c.n[q] = 2LL * h.X.n[l1] * h.V.n[l2];
      c.n2[q] = h.V.n[l2];
      c.dinv[q] = sd.vals<T>().dinv[lev];
      c.a[q] = dim == 1 ? B.cx[g] : B.t1[g];      // f
      c.b[q] = B.cr[g];                            // r
      c.c[q] = B.cd[g];                            // d
      c.d[q] = dim == 1 ? B.t1[g] : out[q];        // x
    }
    k_gcheb_init<T><<<ggrid(c.n, ng), kThreads, 0, s>>>(c, dim, 1.0 / theta);
    SG_CU(cudaGetLastError());
    double rho = 1.0 / sigma1;
    // steps: d ping-pongs between cd and cm
    GCheb<T> fz;
    fz.ng = ng;
    const SideDev& sdd = dim == 1 ? h.X : h.V;
    const int W = sdd.ell_w();
    for (int q = 0; q < ng; ++q) {
      const int g = act.g[q];
      const int lev = dim == 1 ? ws.cl1[g] : ws.cl2[g];
      fz.n1[q] = h.X.n[ws.cl1[g]];
      fz.n2[q] = h.V.n[ws.cl2[g]];
      fz.col[q] = sdd.ell_col[lev];
      fz.val[q] = sdd.vals<T>().ell_fac[sdd.mass][lev];
      fz.dinv[q] = sdd.vals<T>().dinv[lev];
      fz.dold[q] = B.cd[g];
      fz.dnew[q] = B.cm[g];
      fz.r[q] = B.cr[g];
      fz.x[q] = c.d[q];
    }
    for (int k = 1; k < K; ++k) {
      const double rhon = 1.0 / (2.0 * sigma1 - rho);
      const dim3 gg = ggrid(c.n, ng);
      if (dim == 1) {
        if (W == 4) k_gcheb_fused<T, false, 4><<<gg, kThreads, 0, s>>>(fz, rhon * rho, 2.0 * rhon / del);
        else if (W == 8) k_gcheb_fused<T, false, 8><<<gg, kThreads, 0, s>>>(fz, rhon * rho, 2.0 * rhon / del);
        else k_gcheb_fused<T, false, 16><<<gg, kThreads, 0, s>>>(fz, rhon * rho, 2.0 * rhon / del);
      } else {
        if (W == 4) k_gcheb_fused<T, true, 4><<<gg, kThreads, 0, s>>>(fz, rhon * rho, 2.0 * rhon / del);
        else if (W == 8) k_gcheb_fused<T, true, 8><<<gg, kThreads, 0, s>>>(fz, rhon * rho, 2.0 * rhon / del);
        else k_gcheb_fused<T, true, 16><<<gg, kThreads, 0, s>>>(fz, rhon * rho, 2.0 * rhon / del);
      }
      SG_CU(cudaGetLastError());
      for (int q = 0; q < ng; ++q) {
        T* t = const_cast<T*>(fz.dold[q]);
        fz.dold[q] = fz.dnew[q];
        fz.dnew[q] = t;
      }
      rho = rhon;
    }
  }
  return {};
}

// Grouped dots d[slot][off + i] = V_{g,i} . w_g (i < k) for the active grids.
template <typename T>
Status gdots(Handle& h, const Active& act, const std::vector<const T*>& V, const std::vector<long long>& ldv,
             const std::vector<const T*>& w, int k, double* dots, int ld, int off, cudaStream_t s) {
  Workspace& ws = *h.ws;
  CtBatch<T>& B = ct_ws<T>(ws);
  const int ng = (int)act.g.size();
  GVec<T> p;
  GVec<double> r;
  p.ng = r.ng = ng;
  for (int q = 0; q < ng; ++q) {
    const int g = act.g[q];
    p.n[q] = 2LL * h.X.n[ws.cl1[g]] * h.V.n[ws.cl2[g]];
    p.a[q] = V[q];
    p.b[q] = const_cast<T*>(w[q]);
    p.ldv[q] = ldv[q];
    p.slot[q] = r.slot[q] = g;
  }
  k_gmultidot<T><<<dim3(kGroupBlocks, ng), kThreads, 0, s>>>(p, k, B.part);
  SG_CU(cudaGetLastError());
  k_greduce2<<<dim3((k + 63) / 64, ng), 64, 0, s>>>(r, k, B.part, kGroupBlocks, dots, ld, off);
  SG_CU(cudaGetLastError());
  return {};
}

// z (+)= CT correction for the residual r: lockstep GMRES(m) on every
// component system A_{l,l} x_l = r_l (x0 = 0, one restart cycle, right
// preconditioned), then the combination of Algorithm 1.
template <typename T>
Status ct_apply(Handle& h, const T* r, T* z, cudaStream_t s, int* its) {
  Workspace& ws = *h.ws;
  CtBatch<T>& B = ct_ws<T>(ws);
  const int L = h.L;
  const int NG = (int)ws.cl1.size();
  const int m = B.m;
  constexpr int LD = 3 * kMaxKrylov;   // per-grid stride of the dot arrays
  T* X = (T*)ws.ct_x;
  auto gsize = [&](int g) { return 2LL * h.X.n[ws.cl1[g]] * h.V.n[ws.cl2[g]]; };
  // right-hand sides into V_{g,0}: upper grids (l, L-l) take r_l; lower grids
  // (l, L-1-l) the residual restricted in dim 1 from grid (l+1, L-1-l)
  for (int l = 0; l <= L; ++l)
    SG_CU(cudaMemcpyAsync(B.V[l], r + h.off[l], sizeof(T) * gsize(l), cudaMemcpyDeviceToDevice, s));
  if (L >= 1) {
    SpmmLaunch<T> a;
    a.ngrids = L; a.nterms = 1; a.identity = 1; a.accumulate = 0;
    for (int l = 0; l < L; ++l) {
      SpmmGrid<T>& G = a.g[l];
      G.in = r + h.off[l + 1]; G.in2 = nullptr; G.out = B.V[L + 1 + l];
      G.n1_in = h.n1[l + 1]; G.n2_in = G.n2_out = h.n2[l + 1]; G.n1_out = h.X.n[l];
      G.rowptr = h.X.R_rowptr[l]; G.col = h.X.R_col[l]; G.val[0] = h.X.vals<T>().R[l];
    }
    SG_CU(launch_left(a, s));
  }
  // beta_g and V_{g,0} = r_g / beta_g
  Active all;
  for (int g = 0; g < NG; ++g) all.g.push_back(g);
  std::vector<const T*> v0(NG), w0(NG);
  std::vector<long long> ldv(NG);
  for (int g = 0; g < NG; ++g) { v0[g] = B.V[g]; w0[g] = B.V[g]; ldv[g] = gsize(g); }
  SG_ST(gdots<T>(h, all, v0, ldv, w0, 1, B.dots, LD, 2 * kMaxKrylov, s));
  SG_CU(cudaMemcpyAsync(B.host, B.dots, sizeof(double) * NG * LD, cudaMemcpyDeviceToHost, s));
  SG_CU(cudaStreamSynchronize(s));
  std::vector<double> beta(NG);
  std::vector<int> kdone(NG, 0);
  static thread_local std::vector<Givens> Gv;
  Gv.resize(NG);
  Active act;
  for (int g = 0; g < NG; ++g) {
    beta[g] = norm_of(B.host[(long long)g * LD + 2 * kMaxKrylov]);
    if (!std::isfinite(beta[g])) return {SGDG_ENAN, "NaN/Inf in a component right-hand side"};
    if (beta[g] > 0.0) {
      act.g.push_back(g);
      Gv[g].start(beta[g]);
    }
  }
  {
    GVec<T> p;
    p.ng = (int)act.g.size();
    for (int q = 0; q < p.ng; ++q) {
      const int g = act.g[q];
      p.n[q] = gsize(g); p.b[q] = B.V[g]; p.slot[q] = g;
    }
    if (p.ng) {
      k_gnormalize<T><<<ggrid(p.n, p.ng), kThreads, 0, s>>>(p, B.dots, LD, 2 * kMaxKrylov);
      SG_CU(cudaGetLastError());
    }
  }
  Active live = act;
  for (int j = 0; j < m && !live.g.empty(); ++j) {
    NvtxRange step("sgdg.inner");
    const int na = (int)live.g.size();
    std::vector<const T*> vin(na), Vb(na), wv(na);
    std::vector<T*> pout(na);
    std::vector<long long> lv(na);
    for (int q = 0; q < na; ++q) {
      const int g = live.g[q];
      vin[q] = B.V[g] + (long long)j * gsize(g);
      pout[q] = B.t0[g];
    }
    SG_ST(precond_group<T>(h, live, vin, pout, s));
    for (int q = 0; q < na; ++q) {
      const int g = live.g[q];
      const int l1 = ws.cl1[g], l2 = ws.cl2[g];
      const T* uin[1] = {B.t0[g]};
      T* yout[1] = {B.V[g] + (long long)(j + 1) * gsize(g)};
      SG_ST(apply_diag_grids<T>(h, 1, &l1, &l2, uin, yout, s));
      Vb[q] = B.V[g];
      wv[q] = yout[0];
      lv[q] = gsize(g);
    }
    // CGS2 against V_{g,0..j}, then the norm; all grids at once
    SG_ST(gdots<T>(h, live, Vb, lv, wv, j + 1, B.dots, LD, 0, s));
    GVec<T> ax;
    ax.ng = na;
    for (int q = 0; q < na; ++q) {
      const int g = live.g[q];
      ax.n[q] = gsize(g); ax.a[q] = B.V[g]; ax.b[q] = const_cast<T*>(wv[q]); ax.ldv[q] = gsize(g); ax.slot[q] = g;
    }
    k_gmultiaxpy<T><<<ggrid(ax.n, na), kThreads, 0, s>>>(ax, j + 1, B.dots, LD, 0);
    SG_CU(cudaGetLastError());
    SG_ST(gdots<T>(h, live, Vb, lv, wv, j + 1, B.dots, LD, kMaxKrylov, s));
    k_gmultiaxpy<T><<<ggrid(ax.n, na), kThreads, 0, s>>>(ax, j + 1, B.dots, LD, kMaxKrylov);
    SG_CU(cudaGetLastError());
    SG_ST(gdots<T>(h, live, wv, lv, wv, 1, B.dots, LD, 2 * kMaxKrylov, s));
    k_gnormalize<T><<<ggrid(ax.n, na), kThreads, 0, s>>>(ax, B.dots, LD, 2 * kMaxKrylov);
    SG_CU(cudaGetLastError());
    SG_CU(cudaMemcpyAsync(B.host, B.dots, sizeof(double) * NG * LD, cudaMemcpyDeviceToHost, s));
    SG_CU(cudaStreamSynchronize(s));
    Active next;
    for (int q = 0; q < na; ++q) {
      const int g = live.g[q];
      const double* hd = B.host + (long long)g * LD;
      double hcol[kMaxKrylov + 1];
      for (int i = 0; i <= j; ++i) hcol[i] = hd[i] + hd[kMaxKrylov + i];
      const double nrm = norm_of(hd[2 * kMaxKrylov]);
      if (!std::isfinite(nrm)) return {SGDG_ENAN, "NaN/Inf in a component Krylov vector"};
      hcol[j + 1] = nrm;
      const double res = Gv[g].add(j, hcol);
      kdone[g] = j + 1;
      if (!(res <= h.cfg.inner_rtol * beta[g] || nrm == 0.0)) next.g.push_back(g);
    }
    live = next;
  }
  // x_g = P^{-1} sum_i y_i V_{g,i};  grids with beta = 0 get x = 0
  for (int g = 0; g < NG; ++g)
    if (beta[g] == 0.0) SG_CU(vec_fill<T>(X + ws.coff[g], gsize(g), (T)0, s));
  if (!act.g.empty()) {
    for (int g : act.g) {
      double y[kMaxKrylov];
      Gv[g].solve(kdone[g], y);
      for (int i = 0; i < kdone[g]; ++i) B.yh[(long long)g * kMaxKrylov + i] = y[i];
      if (its) *its += kdone[g];
    }
    SG_CU(cudaMemcpyAsync(B.y, B.yh, sizeof(double) * NG * kMaxKrylov, cudaMemcpyHostToDevice, s));
    GVec<T> cb;
    cb.ng = (int)act.g.size();
    std::vector<const T*> cin(cb.ng);
    std::vector<T*> xout(cb.ng);
    for (int q = 0; q < cb.ng; ++q) {
      const int g = act.g[q];
      cb.n[q] = gsize(g); cb.n2[q] = kdone[g]; cb.a[q] = B.V[g]; cb.c[q] = B.t1[g]; cb.ldv[q] = gsize(g);
      cb.slot[q] = g;
      cin[q] = B.t1[g];
      xout[q] = X + ws.coff[g];
    }
    k_gcombine<T><<<ggrid(cb.n, cb.ng), kThreads, 0, s>>>(cb, B.y, kMaxKrylov);
    SG_CU(cudaGetLastError());
    SG_ST(precond_group<T>(h, act, cin, xout, s));
    SG_CU(cudaStreamSynchronize(s));   // B.yh is reused by the next call
  }
  // combination: z_l = dhat_l - (E^(1) (x) Id) dhat_(l-1, L-l)
  SG_CU(cudaMemcpyAsync(z, X, sizeof(T) * h.n_coeffs, cudaMemcpyDeviceToDevice, s));
  if (L >= 1) {
    SpmmLaunch<T> a;
    a.ngrids = L; a.nterms = 1; a.identity = 0; a.accumulate = 1;
    a.tau[0][0] = (T)-1; a.tau[0][1] = 0; a.tau[0][2] = 0; a.tau[0][3] = (T)-1;
    for (int l = 1; l <= L; ++l) {
      SpmmGrid<T>& G = a.g[l - 1];
      G.in = X + ws.coff[L + 1 + (l - 1)]; G.in2 = nullptr; G.out = z + h.off[l];
      G.n1_in = h.X.n[l - 1]; G.n2_in = G.n2_out = h.n2[l]; G.n1_out = h.n1[l];
      G.rowptr = h.X.E_rowptr[l - 1]; G.col = h.X.E_col[l - 1]; G.val[0] = h.X.vals<T>().E[l - 1];
    }
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

template <typename T>
Status alloc_ct(Handle& h, CtBatch<T>& B, int m, long long tot) {
  Workspace& ws = *h.ws;
  const int NG = (int)ws.cl1.size();
  B.m = m;
  const long long per = (long long)(m + 1) + 6;   // basis + t0, t1, cx, cr, cd, cm
  if (dev_alloc(h, (void**)&B.arena, sizeof(T) * (size_t)(per * tot)) != cudaSuccess)
    return {SGDG_ENOMEM, "component-solve workspace"};
  T* p = B.arena;
  for (int g = 0; g < NG; ++g) {
    const long long n = 2LL * h.X.n[ws.cl1[g]] * h.V.n[ws.cl2[g]];
    B.V.push_back(p); p += (m + 1) * n;
    B.t0.push_back(p); p += n;
    B.t1.push_back(p); p += n;
    B.cx.push_back(p); p += n;
    B.cr.push_back(p); p += n;
    B.cd.push_back(p); p += n;
    B.cm.push_back(p); p += n;
  }
  if (dev_alloc(h, (void**)&B.part, sizeof(double) * (size_t)NG * (kMaxKrylov + 2) * kGroupBlocks) != cudaSuccess ||
      dev_alloc(h, (void**)&B.dots, sizeof(double) * (size_t)NG * 3 * kMaxKrylov) != cudaSuccess ||
      dev_alloc(h, (void**)&B.y, sizeof(double) * (size_t)NG * kMaxKrylov) != cudaSuccess)
    return {SGDG_ENOMEM, "component-solve scalars"};
  if (cudaMallocHost((void**)&B.host, sizeof(double) * (size_t)NG * 3 * kMaxKrylov) != cudaSuccess ||
      cudaMallocHost((void**)&B.yh, sizeof(double) * (size_t)NG * kMaxKrylov) != cudaSuccess)
    return {SGDG_ENOMEM, "pinned component-solve scalars"};
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
  if ((int)ws.cl1.size() > kMaxGrids) return {SGDG_EINVAL, "more CT grids than one grouped launch holds"};
  if (mixed) {
    SG_ST(alloc_ct<float>(h, ws.ct32, mi, tot));
    if (dev_alloc(h, (void**)&ws.r32, sizeof(float) * h.n_coeffs) != cudaSuccess ||
        dev_alloc(h, (void**)&ws.z32, sizeof(float) * h.n_coeffs) != cudaSuccess)
      return {SGDG_ENOMEM, "mixed-precision buffers"};
  } else {
    SG_ST(alloc_ct<double>(h, ws.ct64, mi, tot));
  }
  const int mo = std::max(1, std::min(h.cfg.restart, kMaxKrylov - 1));
  SG_ST(alloc_krylov<double>(h, ws.outer, mo, h.n_coeffs, true, false));
  return {};
}

Status ct_precondition(Handle& h, const double* r, double* z, cudaStream_t s, int* its) {
  NvtxRange range("sgdg.ct");
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

// rhs += the source and inflow parts of b_j (Sect. 2) on the strip
// [t_now, t_now + dt]: per Kronecker term the time weights
//   e1_s = int_I g eta_s dt,   e0_s = e1_s + delta int_I g eta_s' dt
// by 3-point Gauss-Legendre (exact for g of degree <= 4), g the source's
// (or inflow datum's) time factor times, for the SD and inflow terms, the
// time factor of the beta component they carry, with an inflow part's gate
// (Sect. 4.2); then every term on every grid.
static Status add_source(Handle& h, cudaStream_t s) {
  if (h.src_terms.empty()) return {};
  NvtxRange range("sgdg.rhs");
  const double dt = h.cfg.dt, ta = h.t_now, dl = h.cfg.delta;
  const double z[3] = {-std::sqrt(0.6), 0.0, std::sqrt(0.6)};
  const double wz[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  double tq[3];
  for (int q = 0; q < 3; ++q) tq[q] = ta + 0.5 * dt * (1.0 + z[q]);
  const size_t ns = h.src_t.size(), nc = h.coef_t.size();
  std::vector<double> fq(3 * ns, 1.0), cq(3 * nc, 1.0);
  for (size_t k = 0; k < ns; ++k)
    if (h.src_t[k].first) h.src_t[k].first(3, tq, &fq[3 * k], h.src_t[k].second);
  for (size_t k = 0; k < nc; ++k)
    if (h.coef_t[k].first) {
      h.coef_t[k].first(3, tq, &cq[3 * k], h.coef_t[k].second);
      for (int q = 0; q < 3; ++q)
        if (!std::isfinite(cq[3 * k + q])) return {SGDG_EINVAL, "a time factor returned NaN or Inf"};
    }
  for (const Handle::SourceTerm& t : h.src_terms) {
    double a0 = 0.0, a1 = 0.0, d1 = 0.0;   // int g eta_0, int g eta_1, int g eta_1'
    for (int q = 0; q < 3; ++q) {
      double g = fq[3 * t.src + q];
      if (t.tfn >= 0) g *= cq[3 * t.tfn + q];
      if (t.gate_fn >= 0 && !(t.gate_sign * t.gate_coef * cq[3 * t.gate_fn + q] > 0.0)) g = 0.0;
      const double w = 0.5 * dt * wz[q] * g;
      a0 += w;                 // eta_0 = 1
      a1 += w * z[q];          // eta_1 = 2 (t - t_a) / dt - 1 = z
      d1 += w * 2.0 / dt;      // eta_1' = 2 / dt  (eta_0' = 0)
    }
    const double e0 = a0, e1 = t.kind == 0 ? a1 + dl * d1 : a1;
    // kind 0: (f, w + delta d_t w); kind 1: delta (f, beta_c d_c w); kind 2: -<g, w>_{Gamma^-}
    const double sc = t.kind == 0 ? t.coef : (t.kind == 1 ? t.coef * dl : -t.coef);
    for (int l = 0; l <= h.L; ++l)
      SG_CU(outer_add(h.rhs + h.off[l], h.n1[l], h.n2[l], t.lx[l], t.lv[h.L - l], sc * e0, sc * e1, s));
  }
  return {};
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

Status set_strip_time(Handle& h, double t0) {
  if (!h.tt.time_dep) return {};
  SG_ST(strip_time_couplings(h.tt, t0, h.cfg.dt, h.time_quad, h.coef_t));
  for (size_t k = 0; k < h.tt.terms.size() && k < h.op.terms.size(); ++k)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) h.op.terms[k].tau[a][b] = h.tt.terms[k].tau[a][b];
  h.tau_version++;
  return {};
}

Status advance_strip(Handle& h, cudaStream_t s, sgdg_strip_stats* st, bool resolve) {
  NvtxRange range("sgdg.strip");
  auto t0 = std::chrono::steady_clock::now();
  SG_ST(solver_init(h));
  Workspace& ws = *h.ws;
  KrylovWs<double>& O = ws.outer;
  const long long n = h.n_coeffs;
  if (!h.have_initial) return {SGDG_EINVAL, "sgdg_set_initial was not called"};
  if (resolve && !h.solved) return {SGDG_EINVAL, "no strip has been solved yet"};
  // the strip's operator (time factors: couplings of (t_{j-1}, t_j))
  SG_ST(set_strip_time(h, resolve ? h.t_now - h.cfg.dt : h.t_now));
  // right-hand side: eta(t_{j-1}^+) (x) M_sg U^-_{j-1}; the first strip uses (u0, phi);
  // a re-solve keeps the right-hand side of the strip
  if (!resolve && !h.first_strip) {
    k_expand<<<gridsz(h.n_spatial), kThreads, 0, s>>>(h.n_spatial, h.U_end, O.t0, 1.0, -1.0);
    SG_CU(cudaGetLastError());
    SG_ST(apply_plan<double>(h, h.mass, O.t0, h.rhs, s));
  }
  if (!resolve) SG_ST(add_source(h, s));
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
  // Algorithm 1 (Sect. 4.3): Richardson on the CT-preconditioned system,
  // u <- u + P_CT(b - A u), with the true residual in FP64 after every step
  while (h.cfg.outer_method == SGDG_OUTER_RICHARDSON && beta > tol && total < h.cfg.max_outer && bnorm > 0.0) {
    SG_ST(ct_precondition(h, r, O.Z, s, &S.inner_its_total));
    SG_CU(vec_axpby<double>(n, 1.0, O.Z, 1.0, x, s));
    SG_ST(apply_plan<double>(h, h.op, x, r, s));
    S.applies++;
    SG_CU(vec_axpby<double>(n, 1.0, h.rhs, -1.0, r, s));
    SG_ST(vnorm<double>(h, r, n, &beta, s));
    total++;
  }
  while (h.cfg.outer_method == SGDG_OUTER_FGMRES && beta > tol && total < h.cfg.max_outer && bnorm > 0.0) {
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
  if (!resolve) {
    h.nsolved++;
    h.t_now += h.cfg.dt;
  }
  // applies between strips use the operator of the next strip
  SG_ST(set_strip_time(h, h.t_now));
  S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (st) *st = S;
  if (S.status == SGDG_ENOCONV) return {SGDG_ENOCONV, "outer iteration reached max_outer"};
  return res;
}

Status h1_norm(Handle& h, const double* u, double* tmp, double* out, cudaStream_t s) {
  SG_ST(solver_init(h));
  SG_ST(apply_plan<double>(h, h.h1, u, tmp, s));
  Workspace& ws = *h.ws;
  SG_ST(mdot<double>(h, 1, u, h.n_coeffs, tmp, h.n_coeffs, ws.dev_dots, s));
  SG_CU(cudaMemcpyAsync(ws.host, ws.dev_dots, sizeof(double), cudaMemcpyDeviceToHost, s));
  SG_CU(cudaStreamSynchronize(s));
  *out = norm_of(ws.host[0]);
  if (!std::isfinite(*out)) return {SGDG_ENAN, "NaN/Inf in an H1 norm"};
  return {};
}

Status constant_in_time(Handle& h, const double* U, double* dst, cudaStream_t s) {
  k_expand<<<gridsz(h.n_spatial), kThreads, 0, s>>>(h.n_spatial, U, dst, 1.0, 0.0);
  SG_CU(cudaGetLastError());
  return {};
}

Handle::~Handle() {}

void solver_free(Handle& h) {
  if (!h.ws) return;
  if (h.ws->host) cudaFreeHost(h.ws->host);
  for (double* p : {h.ws->ct32.host, h.ws->ct32.yh, h.ws->ct64.host, h.ws->ct64.yh})
    if (p) cudaFreeHost(p);
  delete h.ws;
  h.ws = nullptr;
}

}  // namespace sgdg
