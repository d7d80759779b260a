// Device-side data structures and kernel launchers of the sgdg library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "internal.h"

namespace sgdg {

// A named NVTX range over one phase of the strip solve (strip, rhs, apply,
// ct, inner, orth), closed when the scope ends (early returns included).
// Without a profiler attached the push and pop are no-ops.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxTerms = 8;    // terms fused into one SpMM launch
constexpr int kMaxGrids = 24;   // grids fused into one launch

// One grid of a grouped SpMM launch.  Arrays are [n1][n2][2] (s fastest).
// Left:  out[k1][k2] (+)= sum_t tau_t (x) sum_p val_t[p] in[col[p]][k2]   (p in row k1)
// Right: out[k1][k2] (+)= sum_t tau_t (x) sum_p val_t[p] in[k1][col[p]]   (p in row k2)
template <typename T>
struct SpmmGrid {
  const T* in;
  const T* in2;        // optional: the input is in + in2
  T* out;
  int n1_in, n2_in, n1_out, n2_out;
  const int* rowptr;
  const int* col;
  const T* val[kMaxTerms];
  int block0;          // first block of this grid (set by the launcher)
  int ch;              // rows of k1 per thread (set by the launcher)
};

template <typename T>
struct SpmmLaunch {
  int ngrids = 0, nterms = 0;
  int accumulate = 0;  // out += ... instead of out = ...
  int identity = 0;    // single term with tau = I (transfers)
  T tau[kMaxTerms][4];
  SpmmGrid<T> g[kMaxGrids];
};

template <typename T>
cudaError_t launch_left(SpmmLaunch<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_right(SpmmLaunch<T>& a, cudaStream_t s);

// vector kernels (n = number of scalars)
template <typename T>
cudaError_t vec_fill(T* x, long long n, T v, cudaStream_t s);
template <typename TI, typename TO>
cudaError_t vec_convert(const TI* x, TO* y, long long n, cudaStream_t s);
template <typename T>
cudaError_t vec_axpby(long long n, double a, const T* x, double b, T* y, cudaStream_t s);   // y = a x + b y
// partial dot products of w with k vectors V + i*ldv: part[i*nb + b]; nb = gridDim
template <typename T>
cudaError_t vec_multidot(int k, const T* V, long long ldv, const T* w, long long n, double* part, int nb,
                         cudaStream_t s);
// y -= sum_i h[i] V_i (h on the device)
template <typename T>
cudaError_t vec_multiaxpy(int k, const T* V, long long ldv, const double* h, T* y, long long n, cudaStream_t s);
// y = sum_i h[i] V_i + beta y
template <typename T>
cudaError_t vec_combine(int k, const T* V, long long ldv, const double* h, double beta, T* y, long long n,
                        cudaStream_t s);
cudaError_t reduce_parts(int k, const double* part, int nb, double* out, cudaStream_t s);
// outer-product block: out[k1][k2][s] = e[s] * sum_p fx_p[k1] fv_p[k2]
cudaError_t outer_init(double* out, int n1, int n2, int np, const double* fx, const double* fv, double e0,
                       double e1, cudaStream_t s);
// out[k1][k2][s] += e_s * fx[k1] * fv[k2]   (FP64, R = 2)
cudaError_t outer_add(double* out, int n1, int n2, const double* fx, const double* fv, double e0, double e1,
                      cudaStream_t s);
// nodal injection along one dim: out[k1][k2] = in[idx[k1]][k2] (dim 1) / in[k1][idx[k2]] (dim 2); R = 1
cudaError_t inject_dim(const double* in, double* out, int n1_out, int n2_out, int n2_in, const int* idx, int dim,
                       int accumulate, cudaStream_t s);
// spatial vector SpMM along one dim with scalar values (R = 1), for nodal evaluation
cudaError_t spmm1(const double* in, double* out, int n1_in, int n2_in, int n1_out, int n2_out, const int* rowptr,
                  const int* col, const double* val, int dim, int accumulate, cudaStream_t s);

int num_sms();

}  // namespace sgdg
