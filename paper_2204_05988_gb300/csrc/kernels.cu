// CUDA kernels (sm_103a) of the sgdg library.
//
// The hot operations of the operator apply (Sect. 4.2) are Kronecker factor
// products on anisotropic full grids u[k1][k2][s]: a CSR matrix acting on the
// dim-1 index ("left": whole rows of the grid combined) or on the dim-2 index
// ("right": a stencil inside each row), fused with the 2x2 time coupling of
// up to kMaxTerms terms that share one input and one CSR pattern, over a group
// of up to kMaxGrids grids in one launch.  Each thread owns one (k1, k2) pair
// and both time coefficients (a 16 B / 8 B vector load per input entry).
#include <cuda_runtime.h>

#include "device.h"

namespace sgdg {

namespace {

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ int find_grid(const SpmmLaunch<T>& a) {
  int g = 0;
  const int b = blockIdx.x;
#pragma unroll 1
  for (int i = 1; i < a.ngrids; ++i)
    if (b >= a.g[i].block0) g = i;
  return g;
}

template <typename T>
__device__ __forceinline__ void store_terms(const SpmmLaunch<T>& a, T* out, const T (*acc)[2]) {
  T r0, r1;
  if (a.identity) {
    r0 = acc[0][0];
    r1 = acc[0][1];
  } else {
    r0 = 0;
    r1 = 0;
#pragma unroll
    for (int t = 0; t < kMaxTerms; ++t) {
      if (t < a.nterms) {
        r0 += a.tau[t][0] * acc[t][0] + a.tau[t][1] * acc[t][1];
        r1 += a.tau[t][2] * acc[t][0] + a.tau[t][3] * acc[t][1];
      }
    }
  }
  using T2 = typename V2<T>::type;
  T2* o = reinterpret_cast<T2*>(out);
  if (a.accumulate) {
    T2 y = *o;
    y.x += r0;
    y.y += r1;
    *o = y;
  } else {
    T2 y;
    y.x = r0;
    y.y = r1;
    *o = y;
  }
}

// Thread mapping (both kernels): virtual thread v over [0, nchunk * n2), with
// k2 = v % n2 (consecutive threads -> consecutive k2: coalesced 8/16 B loads
// and stores) and rows k1 in [c * ch, c * ch + ch), c = v / n2.  One 32-bit
// division per thread; the loop over ch rows reuses the matrix row (right) or
// the neighbouring input rows through L1 (left).
template <typename T, int NT>
__global__ void __launch_bounds__(kThreads) k_left(const __grid_constant__ SpmmLaunch<T> a) {
  using T2 = typename V2<T>::type;
  const int gi = find_grid(a);
  const SpmmGrid<T>& g = a.g[gi];
  const unsigned v = (unsigned)(blockIdx.x - g.block0) * kThreads + threadIdx.x;
  const unsigned n2 = (unsigned)g.n2_out;
  const unsigned c = v / n2;
  const unsigned k2 = v - c * n2;
  const int r0 = (int)c * g.ch;
  if (r0 >= g.n1_out) return;
  const int r1 = min(r0 + g.ch, g.n1_out);
  const T2* in = reinterpret_cast<const T2*>(g.in) + k2;
  const T2* in2 = g.in2 ? reinterpret_cast<const T2*>(g.in2) + k2 : nullptr;
  for (int k1 = r0; k1 < r1; ++k1) {
    T acc[kMaxTerms][2];
#pragma unroll
    for (int t = 0; t < kMaxTerms; ++t) acc[t][0] = acc[t][1] = 0;
    const int p0 = __ldg(g.rowptr + k1), p1 = __ldg(g.rowptr + k1 + 1);
    for (int p = p0; p < p1; ++p) {
      const size_t j = (size_t)__ldg(g.col + p) * n2;
      T2 u = in[j];
      if (in2) {
        const T2 w = in2[j];
        u.x += w.x;
        u.y += w.y;
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const T vv = __ldg(g.val[t] + p);
        acc[t][0] += vv * u.x;
        acc[t][1] += vv * u.y;
      }
    }
    store_terms(a, g.out + 2 * ((size_t)k1 * n2 + k2), acc);
  }
}

constexpr int kRowCache = 8;   // matrix entries per row held in registers

template <typename T, int NT>
__global__ void __launch_bounds__(kThreads) k_right(const __grid_constant__ SpmmLaunch<T> a) {
  using T2 = typename V2<T>::type;
  constexpr int NC = (NT <= 4) ? NT : 0;   // terms whose row values stay in registers
  const int gi = find_grid(a);
  const SpmmGrid<T>& g = a.g[gi];
  const unsigned v = (unsigned)(blockIdx.x - g.block0) * kThreads + threadIdx.x;
  const unsigned n2 = (unsigned)g.n2_out;
  const unsigned c = v / n2;
  const unsigned k2 = v - c * n2;
  const int r0 = (int)c * g.ch;
  if (r0 >= g.n1_out) return;
  const int r1 = min(r0 + g.ch, g.n1_out);
  const int p0 = __ldg(g.rowptr + k2), p1 = __ldg(g.rowptr + k2 + 1);
  const int nz = p1 - p0;
  int cols[kRowCache];
  T vals[NC > 0 ? NC : 1][kRowCache];
#pragma unroll
  for (int q = 0; q < kRowCache; ++q) {
    cols[q] = (q < nz) ? __ldg(g.col + p0 + q) : 0;
#pragma unroll
    for (int t = 0; t < NC; ++t) vals[t][q] = (q < nz) ? __ldg(g.val[t] + p0 + q) : (T)0;
  }
  const size_t n2i = (size_t)g.n2_in;
  for (int k1 = r0; k1 < r1; ++k1) {
    const T2* in = reinterpret_cast<const T2*>(g.in) + (size_t)k1 * n2i;
    const T2* in2 = g.in2 ? reinterpret_cast<const T2*>(g.in2) + (size_t)k1 * n2i : nullptr;
    T acc[kMaxTerms][2];
#pragma unroll
    for (int t = 0; t < kMaxTerms; ++t) acc[t][0] = acc[t][1] = 0;
#pragma unroll
    for (int q = 0; q < kRowCache; ++q) {
      if (q < nz) {
        T2 u = in[cols[q]];
        if (in2) {
          const T2 w = in2[cols[q]];
          u.x += w.x;
          u.y += w.y;
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const T vv = (t < NC) ? vals[t < NC ? t : 0][q] : __ldg(g.val[t] + p0 + q);
          acc[t][0] += vv * u.x;
          acc[t][1] += vv * u.y;
        }
      }
    }
    for (int p = p0 + kRowCache; p < p1; ++p) {   // rows longer than the register cache
      const int j = __ldg(g.col + p);
      T2 u = in[j];
      if (in2) {
        const T2 w = in2[j];
        u.x += w.x;
        u.y += w.y;
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const T vv = __ldg(g.val[t] + p);
        acc[t][0] += vv * u.x;
        acc[t][1] += vv * u.y;
      }
    }
    store_terms(a, g.out + 2 * ((size_t)k1 * n2 + k2), acc);
  }
}

// rows per thread: enough threads to fill the GPU several times over, at most
// 8 rows per thread
inline int rows_per_thread(long long n1, long long n2) {
  const long long want_threads = 152LL * 2048 * 4;
  long long ch = (n1 * n2 + want_threads - 1) / want_threads;
  if (ch < 1) ch = 1;
  if (ch > 8) ch = 8;
  if (ch > n1) ch = n1;
  return (int)ch;
}

template <typename T>
int assign_blocks(SpmmLaunch<T>& a) {
  int b = 0;
  for (int i = 0; i < a.ngrids; ++i) {
    SpmmGrid<T>& g = a.g[i];
    g.block0 = b;
    g.ch = rows_per_thread(g.n1_out, g.n2_out);
    const long long nchunk = (g.n1_out + g.ch - 1) / g.ch;
    const long long tot = nchunk * g.n2_out;
    b += (int)((tot + kThreads - 1) / kThreads);
  }
  return b;
}

template <typename T, template <typename, int> class K>
struct Dispatch;

}  // namespace

#define SGDG_DISPATCH_NT(KERNEL, T, a, nb, s)                                          \
  switch ((a).nterms) {                                                                \
    case 1: KERNEL<T, 1><<<nb, kThreads, 0, s>>>(a); break;                            \
    case 2: KERNEL<T, 2><<<nb, kThreads, 0, s>>>(a); break;                            \
    case 3: KERNEL<T, 3><<<nb, kThreads, 0, s>>>(a); break;                            \
    case 4: KERNEL<T, 4><<<nb, kThreads, 0, s>>>(a); break;                            \
    case 5: KERNEL<T, 5><<<nb, kThreads, 0, s>>>(a); break;                            \
    case 6: KERNEL<T, 6><<<nb, kThreads, 0, s>>>(a); break;                            \
    case 7: KERNEL<T, 7><<<nb, kThreads, 0, s>>>(a); break;                            \
    default: KERNEL<T, 8><<<nb, kThreads, 0, s>>>(a); break;                           \
  }

template <typename T>
cudaError_t launch_left(SpmmLaunch<T>& a, cudaStream_t s) {
  if (a.ngrids <= 0 || a.nterms <= 0 || a.nterms > kMaxTerms || a.ngrids > kMaxGrids) return cudaErrorInvalidValue;
  int nb = assign_blocks(a);
  if (nb == 0) return cudaSuccess;
  SGDG_DISPATCH_NT(k_left, T, a, nb, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_right(SpmmLaunch<T>& a, cudaStream_t s) {
  if (a.ngrids <= 0 || a.nterms <= 0 || a.nterms > kMaxTerms || a.ngrids > kMaxGrids) return cudaErrorInvalidValue;
  int nb = assign_blocks(a);
  if (nb == 0) return cudaSuccess;
  SGDG_DISPATCH_NT(k_right, T, a, nb, s);
  return cudaGetLastError();
}

template cudaError_t launch_left<double>(SpmmLaunch<double>&, cudaStream_t);
template cudaError_t launch_left<float>(SpmmLaunch<float>&, cudaStream_t);
template cudaError_t launch_right<double>(SpmmLaunch<double>&, cudaStream_t);
template cudaError_t launch_right<float>(SpmmLaunch<float>&, cudaStream_t);

// ---------------------------------------------------------------------------
// vector kernels
// ---------------------------------------------------------------------------

__global__ void k_outer_add(double* out, int n1, int n2, const double* fx, const double* fv, double e0, double e1) {
  const long long n = (long long)n1 * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long k1 = i / n2, k2 = i - k1 * n2;
    const double p = fx[k1] * fv[k2];
    out[2 * i] += e0 * p;
    out[2 * i + 1] += e1 * p;
  }
}

cudaError_t outer_add(double* out, int n1, int n2, const double* fx, const double* fv, double e0, double e1,
                      cudaStream_t s) {
  const long long n = (long long)n1 * n2;
  if (n <= 0) return cudaSuccess;
  const long long b = std::min<long long>((n + 255) / 256, (long long)num_sms() * 8);
  k_outer_add<<<(unsigned)b, 256, 0, s>>>(out, n1, n2, fx, fv, e0, e1);
  return cudaGetLastError();
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

static int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  long long cap = (long long)num_sms() * 8;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

template <typename T>
__global__ void k_fill(T* x, long long n, T v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}
template <typename T>
cudaError_t vec_fill(T* x, long long n, T v, cudaStream_t s) {
  k_fill<<<grid_for(n), kThreads, 0, s>>>(x, n, v);
  return cudaGetLastError();
}
template cudaError_t vec_fill<double>(double*, long long, double, cudaStream_t);
template cudaError_t vec_fill<float>(float*, long long, float, cudaStream_t);

template <typename TO, typename TI>
__device__ __forceinline__ TO convert_to(TI x) { return (TO)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 convert_to<__nv_bfloat16, double>(double x) { return __double2bfloat16(x); }
template <>
__device__ __forceinline__ double convert_to<double, __nv_bfloat16>(__nv_bfloat16 x) {
  return (double)__bfloat162float(x);   // exact: every bfloat16 is a float
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* x, TO* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = convert_to<TO>(x[i]);
}
template <typename TI, typename TO>
cudaError_t vec_convert(const TI* x, TO* y, long long n, cudaStream_t s) {
  k_convert<<<grid_for(n), kThreads, 0, s>>>(x, y, n);
  return cudaGetLastError();
}
template cudaError_t vec_convert<double, float>(const double*, float*, long long, cudaStream_t);
template cudaError_t vec_convert<float, double>(const float*, double*, long long, cudaStream_t);
template cudaError_t vec_convert<double, double>(const double*, double*, long long, cudaStream_t);
template cudaError_t vec_convert<double, __nv_bfloat16>(const double*, __nv_bfloat16*, long long, cudaStream_t);
template cudaError_t vec_convert<__nv_bfloat16, double>(const __nv_bfloat16*, double*, long long, cudaStream_t);

template <typename T>
__global__ void k_axpby(long long n, double a, const T* x, double b, T* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (T)(a * (double)x[i] + (b == 0.0 ? 0.0 : b * (double)y[i]));
}
template <typename T>
cudaError_t vec_axpby(long long n, double a, const T* x, double b, T* y, cudaStream_t s) {
  k_axpby<<<grid_for(n), kThreads, 0, s>>>(n, a, x, b, y);
  return cudaGetLastError();
}
template cudaError_t vec_axpby<double>(long long, double, const double*, double, double*, cudaStream_t);
template cudaError_t vec_axpby<float>(long long, double, const float*, double, float*, cudaStream_t);


// Deterministic multi-dot: block b reduces its grid-stride share of all k
// dots in a fixed order; the host-side or reduce_parts sum runs in block order.
constexpr int kMaxDots = 72;
template <typename T>
__global__ void __launch_bounds__(kThreads) k_multidot(int k, const T* V, long long ldv, const T* w, long long n,
                                                       double* part) {
  __shared__ double red[kThreads / 32];
  for (int i0 = 0; i0 < k; i0 += 8) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int cnt = min(8, k - i0);
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
      const double wx = (double)w[x];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j < cnt) acc[j] += (double)V[(long long)(i0 + j) * ldv + x] * wx;
    }
    for (int j = 0; j < cnt; ++j) {
      double v = acc[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) s += red[q];
        part[(long long)(i0 + j) * gridDim.x + blockIdx.x] = s;
      }
      __syncthreads();
    }
  }
}
template <typename T>
cudaError_t vec_multidot(int k, const T* V, long long ldv, const T* w, long long n, double* part, int nb,
                         cudaStream_t s) {
  if (k <= 0 || k > kMaxDots) return cudaErrorInvalidValue;
  k_multidot<<<nb, kThreads, 0, s>>>(k, V, ldv, w, n, part);
  return cudaGetLastError();
}
template cudaError_t vec_multidot<double>(int, const double*, long long, const double*, long long, double*, int,
                                          cudaStream_t);
template cudaError_t vec_multidot<float>(int, const float*, long long, const float*, long long, double*, int,
                                         cudaStream_t);

__global__ void k_reduce_parts(int k, const double* part, int nb, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(long long)i * nb + b];
  out[i] = s;
}
cudaError_t reduce_parts(int k, const double* part, int nb, double* out, cudaStream_t s) {
  k_reduce_parts<<<(k + 63) / 64, 64, 0, s>>>(k, part, nb, out);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_multiaxpy(int k, const T* V, long long ldv, const double* h, T* y, long long n, double beta,
                            int combine) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc += h[i] * (double)V[(long long)i * ldv + x];
    if (combine) y[x] = (T)(acc + (beta == 0.0 ? 0.0 : beta * (double)y[x]));
    else y[x] = (T)((double)y[x] - acc);
  }
}
template <typename T>
cudaError_t vec_multiaxpy(int k, const T* V, long long ldv, const double* h, T* y, long long n, cudaStream_t s) {
  k_multiaxpy<<<grid_for(n), kThreads, 0, s>>>(k, V, ldv, h, y, n, 0.0, 0);
  return cudaGetLastError();
}
template <typename T>
cudaError_t vec_combine(int k, const T* V, long long ldv, const double* h, double beta, T* y, long long n,
                        cudaStream_t s) {
  k_multiaxpy<<<grid_for(n), kThreads, 0, s>>>(k, V, ldv, h, y, n, beta, 1);
  return cudaGetLastError();
}
template cudaError_t vec_multiaxpy<double>(int, const double*, long long, const double*, double*, long long,
                                           cudaStream_t);
template cudaError_t vec_multiaxpy<float>(int, const float*, long long, const double*, float*, long long,
                                          cudaStream_t);
template cudaError_t vec_combine<double>(int, const double*, long long, const double*, double, double*, long long,
                                         cudaStream_t);
template cudaError_t vec_combine<float>(int, const float*, long long, const double*, double, float*, long long,
                                        cudaStream_t);

__global__ void k_outer(double* out, int n1, int n2, int np, const double* fx, const double* fv, double e0,
                        double e1) {
  long long tot = (long long)n1 * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    int k1 = (int)(i / n2), k2 = (int)(i - (long long)k1 * n2);
    double s = 0.0;
    for (int p = 0; p < np; ++p) s += fx[(long long)p * n1 + k1] * fv[(long long)p * n2 + k2];
    out[2 * i] = e0 * s;
    out[2 * i + 1] = e1 * s;
  }
}
cudaError_t outer_init(double* out, int n1, int n2, int np, const double* fx, const double* fv, double e0, double e1,
                       cudaStream_t s) {
  k_outer<<<grid_for((long long)n1 * n2), kThreads, 0, s>>>(out, n1, n2, np, fx, fv, e0, e1);
  return cudaGetLastError();
}

__global__ void k_inject(const double* in, double* out, int n1, int n2, int n2_in, const int* idx, int dim,
                         int accumulate) {
  long long tot = (long long)n1 * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    int k1 = (int)(i / n2), k2 = (int)(i - (long long)k1 * n2);
    double v = dim == 1 ? in[(long long)idx[k1] * n2_in + k2] : in[(long long)k1 * n2_in + idx[k2]];
    out[i] = accumulate ? out[i] + v : v;
  }
}
cudaError_t inject_dim(const double* in, double* out, int n1_out, int n2_out, int n2_in, const int* idx, int dim,
                       int accumulate, cudaStream_t s) {
  k_inject<<<grid_for((long long)n1_out * n2_out), kThreads, 0, s>>>(in, out, n1_out, n2_out, n2_in, idx, dim,
                                                                      accumulate);
  return cudaGetLastError();
}

__global__ void k_spmm1(const double* in, double* out, int n1_in, int n2_in, int n1_out, int n2_out,
                        const int* rowptr, const int* col, const double* val, int dim, int accumulate) {
  long long tot = (long long)n1_out * n2_out;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    int k1 = (int)(i / n2_out), k2 = (int)(i - (long long)k1 * n2_out);
    double s = 0.0;
    if (dim == 1) {
      for (int p = rowptr[k1]; p < rowptr[k1 + 1]; ++p) s += val[p] * in[(long long)col[p] * n2_in + k2];
    } else {
      for (int p = rowptr[k2]; p < rowptr[k2 + 1]; ++p) s += val[p] * in[(long long)k1 * n2_in + col[p]];
    }
    out[i] = accumulate ? out[i] + s : s;
  }
}
cudaError_t spmm1(const double* in, double* out, int n1_in, int n2_in, int n1_out, int n2_out, const int* rowptr,
                  const int* col, const double* val, int dim, int accumulate, cudaStream_t s) {
  k_spmm1<<<grid_for((long long)n1_out * n2_out), kThreads, 0, s>>>(in, out, n1_in, n2_in, n1_out, n2_out, rowptr,
                                                                      col, val, dim, accumulate);
  return cudaGetLastError();
}

}  // namespace sgdg
