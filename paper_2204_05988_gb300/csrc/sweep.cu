// Chain-step and final kernels of the sparse-grid operator sweep (sm_103a).
//
// Branch A (sources l1' <= l1), one chain per distinct factor V_b, grid i =
// (i, L-i):   S_{b,i} = P1 R2 S_{b,i-1} + U_i V_b^T            (k_chain<A>)
//             Y_i    += sum_{a in b} tau_a X_a S_{b,i}           (k_final<LEFT>)
// Branch B (sources l1' > l1), one chain per distinct factor X_c:
//             T'_{c,i} = R1 P2 T_{c,i+1},  T_{c,i} = T'_{c,i} + X_c U_i   (k_chain<B>)
//             Y_i    += sum_{a in c} tau_a T'_{c,i} V_a^T        (k_final<RIGHT>)
// A chain step advances up to G chains at once: the input rows of U_i and the
// transfer rows are loaded once and shared; the chain states of the previous
// grid are read through L1/L2.  The final kernels fold up to kFinalTerms terms
// of up to kFinalIn chains into one update of Y_i.
#include <cuda_runtime.h>

#include "sweep.h"

namespace sgdg {

namespace {

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };

constexpr int kThreads = 256;
constexpr int kRow = 8;   // matrix row entries cached in registers

inline int chunk_rows(long long n1, long long n2) {
  const long long want = 152LL * 2048 * 4;
  long long ch = (n1 * n2 + want - 1) / want;
  ch = ch < 1 ? 1 : (ch > 8 ? 8 : ch);
  return (int)(ch > n1 ? n1 : ch);
}

// Transfer contribution sum_{p in row k1 of T1} sum_{q in row k2 of T2} T1[p] T2[q] prev[c1(p)][c2(q)]
template <typename T, typename T2>
__device__ __forceinline__ void add_transfer(const T2* prev, int n2p, int k1, const int* t1_rowptr, const int* t1_col,
                                             const T* t1_val, int nq, const int* qc, const T* qv, T& ax, T& ay) {
  const int a0 = __ldg(t1_rowptr + k1), a1 = __ldg(t1_rowptr + k1 + 1);
  for (int p = a0; p < a1; ++p) {
    const T e = __ldg(t1_val + p);
    const T2* row = prev + (size_t)__ldg(t1_col + p) * n2p;
    T sx = 0, sy = 0;
#pragma unroll
    for (int q = 0; q < kRow; ++q) {
      if (q < nq) {
        const T2 w = row[qc[q]];
        sx += qv[q] * w.x;
        sy += qv[q] * w.y;
      }
    }
    ax += e * sx;
    ay += e * sy;
  }
}

// One chain per thread; consecutive blocks take consecutive chains of the same
// tile, so the chains of a launch read the same rows of U_i while they are in
// L2.
template <typename T, bool MODE_A>
__global__ void __launch_bounds__(kThreads, 4) k_chain(const __grid_constant__ ChainArgs<T> a) {
  using T2 = typename V2<T>::type;
  const int g = blockIdx.x % a.nchains;
  const unsigned tile = blockIdx.x / a.nchains;
  const unsigned v = tile * kThreads + threadIdx.x;
  const unsigned n2 = (unsigned)a.n2;
  const unsigned c = v / n2;
  const unsigned k2 = v - c * n2;
  const int r0 = (int)c * a.ch;
  if (r0 >= a.n1) return;
  const int r1 = min(r0 + a.ch, a.n1);
  // dim-2 transfer row k2 (A: R2, B: P2) in registers
  int qc[kRow];
  T qv[kRow];
  int nq = 0;
  if (a.has_prev) {
    const int b0 = __ldg(a.t2_rowptr + k2), b1 = __ldg(a.t2_rowptr + k2 + 1);
    nq = b1 - b0;
#pragma unroll
    for (int q = 0; q < kRow; ++q) {
      qc[q] = q < nq ? __ldg(a.t2_col + b0 + q) : 0;
      qv[q] = q < nq ? __ldg(a.t2_val + b0 + q) : (T)0;
    }
  }
  // A: the chain's first factor, row k2 of V_c, in registers
  int fc[kRow];
  T fv[kRow];
  int nf = 0;
  const T* fval = a.f_val[g];
  if (MODE_A) {
    const int f0 = __ldg(a.f_rowptr + k2), f1 = __ldg(a.f_rowptr + k2 + 1);
    nf = f1 - f0;
#pragma unroll
    for (int q = 0; q < kRow; ++q) {
      fc[q] = q < nf ? __ldg(a.f_col + f0 + q) : 0;
      fv[q] = q < nf ? __ldg(fval + f0 + q) : (T)0;
    }
  }
  const T2* U = reinterpret_cast<const T2*>(a.U);
  const T2* prev = reinterpret_cast<const T2*>(a.prev[g]);
  T2* out = reinterpret_cast<T2*>(a.out[g]);
  T2* strict = reinterpret_cast<T2*>(a.strict[g]);
  for (int k1 = r0; k1 < r1; ++k1) {
    T zx = 0, zy = 0;
    if (MODE_A) {
      const T2* urow = U + (size_t)k1 * n2;
#pragma unroll
      for (int q = 0; q < kRow; ++q) {
        if (q < nf) {
          const T2 u = urow[fc[q]];
          zx += fv[q] * u.x;
          zy += fv[q] * u.y;
        }
      }
    } else {
      const int f0 = __ldg(a.f_rowptr + k1), f1 = __ldg(a.f_rowptr + k1 + 1);
      for (int p = f0; p < f1; ++p) {
        const T2 u = U[(size_t)__ldg(a.f_col + p) * n2 + k2];
        const T xv = __ldg(fval + p);
        zx += xv * u.x;
        zy += xv * u.y;
      }
    }
    T tx = 0, ty = 0;
    if (a.has_prev)
      add_transfer<T, T2>(prev, a.n2_prev, k1, a.t1_rowptr, a.t1_col, a.t1_val, nq, qc, qv, tx, ty);
    const size_t o = (size_t)k1 * n2 + k2;
    T2 r;
    r.x = zx + tx;
    r.y = zy + ty;
    out[o] = r;
    if (!MODE_A && strict) {
      T2 sv;
      sv.x = tx;
      sv.y = ty;
      strict[o] = sv;
    }
  }
}

template <typename T, bool LEFT>
__global__ void __launch_bounds__(kThreads) k_final(const __grid_constant__ FinalArgs<T> a) {
  using T2 = typename V2<T>::type;
  const unsigned v = blockIdx.x * kThreads + threadIdx.x;
  const unsigned n2 = (unsigned)a.n2;
  const unsigned c = v / n2;
  const unsigned k2 = v - c * n2;
  const int r0 = (int)c * a.ch;
  if (r0 >= a.n1) return;
  const int r1 = min(r0 + a.ch, a.n1);
  int pc[kRow];
  int np = 0, pb = 0;
  if (!LEFT) {
    pb = __ldg(a.rowptr + k2);
    np = __ldg(a.rowptr + k2 + 1) - pb;
#pragma unroll
    for (int q = 0; q < kRow; ++q) pc[q] = q < np ? __ldg(a.col + pb + q) : 0;
  }
  for (int k1 = r0; k1 < r1; ++k1) {
    T yx = 0, yy = 0;
    int p0 = 0, p1 = 0;
    if (LEFT) {
      p0 = __ldg(a.rowptr + k1);
      p1 = __ldg(a.rowptr + k1 + 1);
    }
    for (int t = 0; t < a.nterms; ++t) {
      const T2* in = reinterpret_cast<const T2*>(a.in[a.tin[t]]);
      const T* val = a.val[t];
      T sx = 0, sy = 0;
      if (LEFT) {
        for (int p = p0; p < p1; ++p) {
          const T vv = __ldg(val + p);
          const T2 u = in[(size_t)__ldg(a.col + p) * n2 + k2];
          sx += vv * u.x;
          sy += vv * u.y;
        }
      } else {
        const T2* row = in + (size_t)k1 * n2;
#pragma unroll
        for (int q = 0; q < kRow; ++q) {
          if (q < np) {
            const T vv = __ldg(val + pb + q);
            const T2 u = row[pc[q]];
            sx += vv * u.x;
            sy += vv * u.y;
          }
        }
        for (int p = pb + kRow; p < pb + np; ++p) {
          const T vv = __ldg(val + p);
          const T2 u = row[__ldg(a.col + p)];
          sx += vv * u.x;
          sy += vv * u.y;
        }
      }
      yx += a.tau[t][0] * sx + a.tau[t][1] * sy;
      yy += a.tau[t][2] * sx + a.tau[t][3] * sy;
    }
    T2* y = reinterpret_cast<T2*>(a.y) + (size_t)k1 * n2 + k2;
    if (a.accumulate) {
      T2 o = *y;
      o.x += yx;
      o.y += yy;
      *y = o;
    } else {
      T2 o;
      o.x = yx;
      o.y = yy;
      *y = o;
    }
  }
}

inline int blocks_for(int n1, int n2, int ch) {
  const long long nchunk = ((long long)n1 + ch - 1) / ch;
  return (int)((nchunk * n2 + kThreads - 1) / kThreads);
}

}  // namespace

template <typename T>
cudaError_t launch_chain(ChainArgs<T>& a, bool mode_a, cudaStream_t s) {
  if (a.nchains < 1 || a.nchains > kChainSlots) return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  if (a.ch <= 0) a.ch = chunk_rows((long long)a.n1 * a.nchains, a.n2);
  if (a.ch > a.n1) a.ch = a.n1;
  const long long nb = (long long)blocks_for(a.n1, a.n2, a.ch) * a.nchains;
  if (nb > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (mode_a) k_chain<T, true><<<(unsigned)nb, kThreads, 0, s>>>(a);
  else k_chain<T, false><<<(unsigned)nb, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_final(FinalArgs<T>& a, bool left, cudaStream_t s) {
  if (a.nterms < 1 || a.nterms > kFinalTerms || a.nin < 1 || a.nin > kFinalIn) return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  if (a.ch <= 0) a.ch = chunk_rows(a.n1, a.n2);
  const int nb = blocks_for(a.n1, a.n2, a.ch);
  if (left) k_final<T, true><<<nb, kThreads, 0, s>>>(a);
  else k_final<T, false><<<nb, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_chain<double>(ChainArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_chain<float>(ChainArgs<float>&, bool, cudaStream_t);
template cudaError_t launch_final<double>(FinalArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_final<float>(FinalArgs<float>&, bool, cudaStream_t);

}  // namespace sgdg
