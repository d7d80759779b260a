// Coarse full-grid views of sparse-grid functions (for the learned warm start).
//
// sgdg_coarse_values: the values of U = sum_l u_l at the nodes of the full
// grid (lx, lv).  Per component grid (l, L-l): in each dimension the coarse
// nodes are either nodes of the grid's (finer) level - take them by the
// composed injection - or the grid's (coarser) level is prolonged up to the
// coarse level by the embeddings E (Sect. 4.2).
// sgdg_coarse_diff: the same view of the difference of two functions.
// sgdg_add_coarse: adds the P1 function c on the full grid (lx, lv) to the
// component grid (lx, L-lx), prolonged in v from level lv to L-lx.
#include <cuda_runtime.h>

#include "handle.h"

namespace sgdg {

namespace {

constexpr int kTh = 256;
inline int nb(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + kTh - 1) / kTh, 8192)); }

__global__ void k_iota(int* m, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) m[i] = i;
}
// map[i] = inj[map[i]] (one refinement level deeper)
__global__ void k_compose(int* m, const int* inj, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) m[i] = inj[m[i]];
}
// t[r][c][s] = u[rmap[r]][cmap[c]][s]
__global__ void k_gather(const double* u, int n2u, const int* rmap, const int* cmap, int nr, int nc, int R,
                         double* t) {
  long long tot = (long long)nr * nc * R;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    int s = (int)(i % R);
    long long q = i / R;
    int c = (int)(q % nc), r = (int)(q / nc);
    t[i] = u[((size_t)rmap[r] * n2u + cmap[c]) * R + s];
  }
}
// rows: out[i][*] = sum_p E[i,p] in[col_p][*] (row length rl doubles)
__global__ void k_prolong_rows(const double* in, double* out, int nout, int rl, const int* rp, const int* ci,
                               const double* v) {
  long long tot = (long long)nout * rl;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    int r = (int)(i / rl), k = (int)(i % rl);
    double s = 0.0;
    for (int p = rp[r]; p < rp[r + 1]; ++p) s += v[p] * in[(size_t)ci[p] * rl + k];
    out[i] = s;
  }
}
// columns: out[r][j][s] = sum_p E[j,p] in[r][col_p][s]
__global__ void k_prolong_cols(const double* in, double* out, int n1, int n2i, int n2o, int R, const int* rp,
                               const int* ci, const double* v) {
  long long tot = (long long)n1 * n2o * R;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    int s = (int)(i % R);
    long long q = i / R;
    int j = (int)(q % n2o), r = (int)(q / n2o);
    double acc = 0.0;
    for (int p = rp[j]; p < rp[j + 1]; ++p) acc += v[p] * in[((size_t)r * n2i + ci[p]) * R + s];
    out[i] = acc;
  }
}
__global__ void k_sub(double* y, const double* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] -= x[i];
}
__global__ void k_add(double* y, const double* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}

#define CK(x)                                                               \
  do {                                                                      \
    cudaError_t e_ = (x);                                                   \
    if (e_ != cudaSuccess) return {SGDG_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// composed injection map from level lc (coarse) into level lf (>= lc) of one side
Status inj_map(const SideDev& sd, int lc, int lf, int* map, cudaStream_t s) {
  const int n = sd.n[lc];
  k_iota<<<(n + kTh - 1) / kTh, kTh, 0, s>>>(map, n);
  for (int k = lc; k < lf; ++k) k_compose<<<(n + kTh - 1) / kTh, kTh, 0, s>>>(map, sd.inj[k], n);
  CK(cudaGetLastError());
  return {};
}

}  // namespace

Status coarse_values(Handle& h, const double* u, int R, int lx, int lv, double* out, cudaStream_t s) {
  const int L = h.L;
  if ((R != 1 && R != 2) || lx < 0 || lv < 0 || lx > L || lv > L) return {SGDG_EINVAL, "bad coarse grid or R"};
  const int nx = h.X.n[lx], nv = h.V.n[lv];
  // every intermediate has at most nx rows and nv columns (finer grids are
  // injected first, coarser ones only grow up to the coarse levels)
  const long long big = (long long)nx * nv * R;
  double *t0, *t1;
  int *rm, *cm;
  CK(cudaMallocAsync((void**)&t0, sizeof(double) * big, s));
  CK(cudaMallocAsync((void**)&t1, sizeof(double) * big, s));
  CK(cudaMallocAsync((void**)&rm, sizeof(int) * std::max(nx, 1), s));
  CK(cudaMallocAsync((void**)&cm, sizeof(int) * std::max(nv, 1), s));
  CK(cudaMemsetAsync(out, 0, sizeof(double) * nx * nv * R, s));
  Status st;
  for (int l = 0; l <= L && !st.code; ++l) {
    const int l2 = L - l;
    const double* ug = u + (R == 2 ? h.off[l] : h.soff[l]);
    // rows: inject if the grid is finer in x, else keep all rows for prolongation
    const bool injx = l >= lx, injv = l2 >= lv;
    int nr = injx ? nx : h.n1[l], nc = injv ? nv : h.n2[l];
    if (injx) st = inj_map(h.X, lx, l, rm, s);
    else k_iota<<<(nr + kTh - 1) / kTh, kTh, 0, s>>>(rm, nr);
    if (st.code) break;
    if (injv) st = inj_map(h.V, lv, l2, cm, s);
    else k_iota<<<(nc + kTh - 1) / kTh, kTh, 0, s>>>(cm, nc);
    if (st.code) break;
    k_gather<<<nb((long long)nr * nc * R), kTh, 0, s>>>(ug, h.n2[l], rm, cm, nr, nc, R, t0);
    for (int k = l; !injx && k < lx; ++k) {   // prolong rows x level k -> k+1
      k_prolong_rows<<<nb((long long)h.X.n[k + 1] * nc * R), kTh, 0, s>>>(t0, t1, h.X.n[k + 1], nc * R,
                                                                           h.X.E_rowptr[k], h.X.E_col[k],
                                                                           h.X.v64.E[k]);
      std::swap(t0, t1);
      nr = h.X.n[k + 1];
    }
    for (int k = l2; !injv && k < lv; ++k) {  // prolong columns v level k -> k+1
      k_prolong_cols<<<nb((long long)nr * h.V.n[k + 1] * R), kTh, 0, s>>>(t0, t1, nr, nc, h.V.n[k + 1], R,
                                                                          h.V.E_rowptr[k], h.V.E_col[k],
                                                                          h.V.v64.E[k]);
      std::swap(t0, t1);
      nc = h.V.n[k + 1];
    }
    k_add<<<nb((long long)nx * nv * R), kTh, 0, s>>>(out, t0, (long long)nx * nv * R);
    if (cudaGetLastError() != cudaSuccess) st = {SGDG_ECUDA, "coarse values kernels"};
  }
  cudaFreeAsync(t0, s);
  cudaFreeAsync(t1, s);
  cudaFreeAsync(rm, s);
  cudaFreeAsync(cm, s);
  return st;
}

Status coarse_diff(Handle& h, const double* a, const double* b, int R, int lx, int lv, double* out,
                   cudaStream_t s) {
  const int L = h.L;
  if ((R != 1 && R != 2) || lx < 0 || lv < 0 || lx > L || lv > L) return {SGDG_EINVAL, "bad coarse grid or R"};
  const long long n = (long long)h.X.n[lx] * h.V.n[lv] * R;
  double* t = nullptr;
  CK(cudaMallocAsync((void**)&t, sizeof(double) * n, s));
  Status st = coarse_values(h, a, R, lx, lv, out, s);
  if (!st.code) st = coarse_values(h, b, R, lx, lv, t, s);
  if (!st.code) {
    k_sub<<<nb(n), kTh, 0, s>>>(out, t, n);
    if (cudaGetLastError() != cudaSuccess) st = {SGDG_ECUDA, "coarse difference kernel"};
  }
  cudaFreeAsync(t, s);
  return st;
}

Status add_coarse(Handle& h, const double* c, int lx, int lv, double* u, cudaStream_t s) {
  const int L = h.L;
  if (lx < 0 || lx > L || lv < 0 || lv > L - lx) return {SGDG_EINVAL, "need 0 <= lx <= L and lv <= L - lx"};
  const int nx = h.X.n[lx];
  double *t0, *t1;
  const long long big = (long long)nx * h.V.n[L - lx] * 2;
  CK(cudaMallocAsync((void**)&t0, sizeof(double) * big, s));
  CK(cudaMallocAsync((void**)&t1, sizeof(double) * big, s));
  CK(cudaMemcpyAsync(t0, c, sizeof(double) * nx * h.V.n[lv] * 2, cudaMemcpyDeviceToDevice, s));
  int nc = h.V.n[lv];
  for (int k = lv; k < L - lx; ++k) {
    k_prolong_cols<<<nb((long long)nx * h.V.n[k + 1] * 2), kTh, 0, s>>>(t0, t1, nx, nc, h.V.n[k + 1], 2,
                                                                        h.V.E_rowptr[k], h.V.E_col[k],
                                                                        h.V.v64.E[k]);
    std::swap(t0, t1);
    nc = h.V.n[k + 1];
  }
  k_add<<<nb(big), kTh, 0, s>>>(u + h.off[lx], t0, big);
  Status st;
  if (cudaGetLastError() != cudaSuccess) st = {SGDG_ECUDA, "add coarse kernels"};
  cudaFreeAsync(t0, s);
  cudaFreeAsync(t1, s);
  return st;
}

}  // namespace sgdg
