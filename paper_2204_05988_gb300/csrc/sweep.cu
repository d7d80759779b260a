// Restriction, chain-step and final kernels of the sparse-grid operator sweep
// (sm_103a).
//
// Branch A (sources l1' <= l1), one chain per distinct factor V_b, grid i =
// (i, L-i):   Z_b     = S_{b,i-1} R2^T                            (k_restrict<dim 2>)
//             S_{b,i} = P1 Z_b + U_i V_b^T                         (k_chain<A>)
//             Y_i    += sum_{a in b} tau_a X_a S_{b,i}             (k_final<LEFT>)
// Branch B (sources l1' > l1), one chain per distinct factor X_c:
//             Z_c      = R1 T_{c,i+1}                              (k_restrict<dim 1>)
//             T'_{c,i} = Z_c P2^T,  T_{c,i} = T'_{c,i} + X_c U_i    (k_chain<B>)
//             Y_i    += sum_{a in c} tau_a T'_{c,i} V_a^T          (k_final<RIGHT>)
// Restricting before prolonging keeps the intermediate Z on the coarse side
// of both dimensions (a quarter of a grid for 2-D sides, half for 1-D), so a
// transfer costs |R row| / ratio + |P row| multiply-adds per output instead
// of |R row| * |P row| for the fused tensor-product stencil.
//
// Every kernel maps one thread to one column k2 of a chunk of `ch` rows and
// loops over the chains (or inputs) of its launch inside the thread: the
// shared operands - rows of U_i, the matrix rows and the gather offsets - are
// loaded or computed once per element and reused by every chain.  Matrix rows
// come from ELL arrays with 16-byte vector loads and stay in registers; the
// operands of the next chain (or input) are loaded before the current one is
// combined and stored, so every thread keeps two chains' loads in flight.
#include <cuda_runtime.h>

#include "sweep.h"

namespace sgdg {

namespace {

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };

constexpr int kThreads = 256;

inline int chunk_rows(long long n1, long long n2) {
  const long long want = 152LL * 2048 * 2;
  long long ch = (n1 * n2 + want - 1) / want;
  ch = ch < 1 ? 1 : (ch > 8 ? 8 : ch);
  return (int)(ch > n1 ? n1 : ch);
}

constexpr int kChunksPerBlock = kThreads / kTileW;

inline long long blocks_for(int n1, int n2, int ch, int tiled) {
  const long long nchunk = ((long long)n1 + ch - 1) / ch;
  if (tiled) return ((n2 + kTileW - 1) / kTileW) * ((nchunk + kChunksPerBlock - 1) / kChunksPerBlock);
  return (nchunk * n2 + kThreads - 1) / kThreads;
}

// This thread's column k2 and rows [r0, r1); false when it has none.
__device__ __forceinline__ bool thread_rows(int n1, int n2, int ch, int tiled, unsigned& k2, int& r0, int& r1) {
  if (!tiled) {
    const unsigned v = blockIdx.x * kThreads + threadIdx.x;
    const unsigned c = v / (unsigned)n2;
    k2 = v - c * (unsigned)n2;
    r0 = (int)c * ch;
  } else {
    const unsigned nchunk = ((unsigned)n1 + ch - 1) / ch;
    const unsigned ngroups = (nchunk + kChunksPerBlock - 1) / kChunksPerBlock;
    const unsigned tile = blockIdx.x / ngroups;
    const unsigned grp = blockIdx.x - tile * ngroups;
    k2 = tile * kTileW + threadIdx.x % kTileW;
    if (k2 >= (unsigned)n2) return false;
    r0 = (int)((grp * kChunksPerBlock + threadIdx.x / kTileW) * ch);
  }
  if (r0 >= n1) return false;
  r1 = min(r0 + ch, n1);
  return true;
}

template <int ROW>
struct Ell {
  static constexpr int W = ROW <= 4 ? 4 : 8;
};

// ROW column indices of an ELL row (16-byte vector loads)
template <int ROW>
__device__ __forceinline__ void ell_cols(const int* p, unsigned (&c)[ROW]) {
  constexpr int W = Ell<ROW>::W;
  const int4* q = reinterpret_cast<const int4*>(p);
#pragma unroll
  for (int i = 0; i < W / 4; ++i) {
    const int4 v = __ldg(q + i);
    if (4 * i + 0 < ROW) c[(4 * i + 0) % ROW] = (unsigned)v.x;
    if (4 * i + 1 < ROW) c[(4 * i + 1) % ROW] = (unsigned)v.y;
    if (4 * i + 2 < ROW) c[(4 * i + 2) % ROW] = (unsigned)v.z;
    if (4 * i + 3 < ROW) c[(4 * i + 3) % ROW] = (unsigned)v.w;
  }
}

// ROW values of an ELL row
template <int ROW>
__device__ __forceinline__ void ell_vals(const float* p, float (&v)[ROW]) {
  constexpr int W = Ell<ROW>::W;
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < W / 4; ++i) {
    const float4 x = __ldg(q + i);
    if (4 * i + 0 < ROW) v[(4 * i + 0) % ROW] = x.x;
    if (4 * i + 1 < ROW) v[(4 * i + 1) % ROW] = x.y;
    if (4 * i + 2 < ROW) v[(4 * i + 2) % ROW] = x.z;
    if (4 * i + 3 < ROW) v[(4 * i + 3) % ROW] = x.w;
  }
}
template <int ROW>
__device__ __forceinline__ void ell_vals(const double* p, double (&v)[ROW]) {
  constexpr int W = Ell<ROW>::W;
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int i = 0; i < W / 2; ++i) {
    if (2 * i < ROW) {
      const double2 x = __ldg(q + i);
      v[(2 * i) % ROW] = x.x;
      if (2 * i + 1 < ROW) v[(2 * i + 1) % ROW] = x.y;
    }
  }
}

// A prolongation row (ELL width 2)
template <typename T>
__device__ __forceinline__ void prolong_row(const int* col, const T* val, unsigned r, unsigned (&c)[kProlongRow],
                                            T (&v)[kProlongRow]) {
  const int2 cc = __ldg(reinterpret_cast<const int2*>(col) + r);
  c[0] = (unsigned)cc.x;
  c[1] = (unsigned)cc.y;
  v[0] = __ldg(val + 2 * (size_t)r);
  v[1] = __ldg(val + 2 * (size_t)r + 1);
}

template <typename T2, int N>
__device__ __forceinline__ void gather(const T2* base, const unsigned (&off)[N], T2 (&w)[N]) {
#pragma unroll
  for (int j = 0; j < N; ++j) w[j] = base[off[j]];
}

template <typename T, bool DIM2, int ROW>
__global__ void __launch_bounds__(kThreads) k_restrict(const __grid_constant__ RestrictArgs<T> a) {
  using T2 = typename V2<T>::type;
  constexpr int W = Ell<ROW>::W;
  const unsigned n2 = (unsigned)a.n2;
  unsigned k2;
  int r0, r1;
  if (!thread_rows(a.n1, a.n2, a.ch, a.tiled, k2, r0, r1)) return;
  unsigned rc[ROW];
  T rv[ROW];
  if (DIM2) {
    // Z[k1][k2] = sum_j R[k2][j] in[k1][col_j]: row k2 of R, reused over the rows
    ell_cols<ROW>(a.col + (size_t)k2 * W, rc);
    ell_vals<ROW>(a.val + (size_t)k2 * W, rv);
  }
  for (int k1 = r0; k1 < r1; ++k1) {
    if (!DIM2) {
      // Z[k1][k2] = sum_j R[k1][j] in[col_j][k2]: row k1 of R (uniform in a warp)
      ell_cols<ROW>(a.col + (size_t)k1 * W, rc);
      ell_vals<ROW>(a.val + (size_t)k1 * W, rv);
    }
    unsigned off[ROW];
#pragma unroll
    for (int j = 0; j < ROW; ++j) off[j] = DIM2 ? (unsigned)k1 * (unsigned)a.n2_in + rc[j] : rc[j] * n2 + k2;
    const size_t o = (size_t)k1 * n2 + k2;
    for (int g = 0; g < a.nchains; ++g) {
      T2 w[ROW];
      gather(reinterpret_cast<const T2*>(a.in[g]), off, w);
      T sx = 0, sy = 0;
#pragma unroll
      for (int j = 0; j < ROW; ++j) {
        sx += rv[j] * w[j].x;
        sy += rv[j] * w[j].y;
      }
      T2 r;
      r.x = sx;
      r.y = sy;
      reinterpret_cast<T2*>(a.out[g])[o] = r;
    }
  }
}

template <typename T, bool MODE_A, int ROW>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 4 : 2) k_chain(const __grid_constant__ ChainArgs<T> a) {
  using T2 = typename V2<T>::type;
  constexpr int W = Ell<ROW>::W;
  const unsigned n2 = (unsigned)a.n2;
  unsigned k2;
  int r0, r1;
  if (!thread_rows(a.n1, a.n2, a.ch, a.tiled, k2, r0, r1)) return;
  unsigned fc[ROW];
  unsigned pc[kProlongRow] = {0, 0};
  T pv[kProlongRow] = {0, 0};
  if (MODE_A) ell_cols<ROW>(a.f_col + (size_t)k2 * W, fc);     // row k2 of the v pattern
  else if (a.has_prev) prolong_row(a.p_col, a.p_val, k2, pc, pv);   // P2 row k2
  const T2* U = reinterpret_cast<const T2*>(a.U);
  for (int k1 = r0; k1 < r1; ++k1) {
    // the shared operand of the chains: U gathered along the first factor's row
    T2 u[ROW];
    unsigned zo[kProlongRow];
    if (MODE_A) {
      unsigned off[ROW];
#pragma unroll
      for (int j = 0; j < ROW; ++j) off[j] = (unsigned)k1 * n2 + fc[j];
      gather(U, off, u);
      if (a.has_prev) prolong_row(a.p_col, a.p_val, (unsigned)k1, pc, pv);   // P1 row k1
#pragma unroll
      for (int q = 0; q < kProlongRow; ++q) zo[q] = pc[q] * n2 + k2;
    } else {
      ell_cols<ROW>(a.f_col + (size_t)k1 * W, fc);   // row k1 of the x pattern (uniform in a warp)
      unsigned off[ROW];
#pragma unroll
      for (int j = 0; j < ROW; ++j) off[j] = fc[j] * n2 + k2;
      gather(U, off, u);
#pragma unroll
      for (int q = 0; q < kProlongRow; ++q) zo[q] = (unsigned)k1 * (unsigned)a.nz2 + pc[q];
    }
    const size_t o = (size_t)k1 * n2 + k2;
    const size_t frow = (size_t)(MODE_A ? k2 : (unsigned)k1) * W;
    // chain g's factor row and Z values; the next chain's are loaded ahead
    T fv[ROW];
    T2 z[kProlongRow];
#pragma unroll
    for (int q = 0; q < kProlongRow; ++q) z[q].x = z[q].y = 0;
    ell_vals<ROW>(a.f_val[0] + frow, fv);
    if (a.has_prev) gather(reinterpret_cast<const T2*>(a.Z[0]), zo, z);
    for (int g = 0; g < a.nchains; ++g) {
      T cv[ROW];
      T2 cz[kProlongRow];
#pragma unroll
      for (int j = 0; j < ROW; ++j) cv[j] = fv[j];
#pragma unroll
      for (int q = 0; q < kProlongRow; ++q) cz[q] = z[q];
      if (g + 1 < a.nchains) {
        ell_vals<ROW>(a.f_val[g + 1] + frow, fv);
        if (a.has_prev) gather(reinterpret_cast<const T2*>(a.Z[g + 1]), zo, z);
      }
      T tx = 0, ty = 0;
      if (a.has_prev) {
#pragma unroll
        for (int q = 0; q < kProlongRow; ++q) {
          tx += pv[q] * cz[q].x;
          ty += pv[q] * cz[q].y;
        }
      }
      T zx = tx, zy = ty;
#pragma unroll
      for (int j = 0; j < ROW; ++j) {
        zx += cv[j] * u[j].x;
        zy += cv[j] * u[j].y;
      }
      T2 r;
      r.x = zx;
      r.y = zy;
      reinterpret_cast<T2*>(a.out[g])[o] = r;
      if (!MODE_A && a.has_prev) {
        T2 sv;
        sv.x = tx;
        sv.y = ty;
        reinterpret_cast<T2*>(a.strict[g])[o] = sv;
      }
    }
  }
}

template <typename T, bool LEFT, int ROW>
__global__ void __launch_bounds__(kThreads) k_final(const __grid_constant__ FinalArgs<T> a) {
  using T2 = typename V2<T>::type;
  constexpr int W = Ell<ROW>::W;
  const unsigned n2 = (unsigned)a.n2;
  unsigned k2;
  int r0, r1;
  if (!thread_rows(a.n1, a.n2, a.ch, a.tiled, k2, r0, r1)) return;
  unsigned fc[ROW];
  if (!LEFT) ell_cols<ROW>(a.col + (size_t)k2 * W, fc);
  for (int k1 = r0; k1 < r1; ++k1) {
    if (LEFT) ell_cols<ROW>(a.col + (size_t)k1 * W, fc);
    unsigned off[ROW];
#pragma unroll
    for (int j = 0; j < ROW; ++j) off[j] = LEFT ? fc[j] * n2 + k2 : (unsigned)k1 * n2 + fc[j];
    const size_t frow = (size_t)(LEFT ? (unsigned)k1 : k2) * W;
    const size_t o = (size_t)k1 * n2 + k2;
    T yx = 0, yy = 0;
    T2 w[ROW];
    gather(reinterpret_cast<const T2*>(a.in[0]), off, w);
    for (int ci = 0; ci < a.nin; ++ci) {
      T2 cw[ROW];
#pragma unroll
      for (int j = 0; j < ROW; ++j) cw[j] = w[j];
      if (ci + 1 < a.nin) gather(reinterpret_cast<const T2*>(a.in[ci + 1]), off, w);
      for (int t = a.tbeg[ci]; t < a.tbeg[ci + 1]; ++t) {
        T ev[ROW];
        ell_vals<ROW>(a.val[t] + frow, ev);
        T sx = 0, sy = 0;
#pragma unroll
        for (int j = 0; j < ROW; ++j) {
          sx += ev[j] * cw[j].x;
          sy += ev[j] * cw[j].y;
        }
        yx += a.tau[t][0] * sx + a.tau[t][1] * sy;
        yy += a.tau[t][2] * sx + a.tau[t][3] * sy;
      }
    }
    T2* y = reinterpret_cast<T2*>(a.y) + o;
    T2 r;
    if (a.accumulate) {
      r = *y;
      r.x += yx;
      r.y += yy;
    } else {
      r.x = yx;
      r.y = yy;
    }
    *y = r;
  }
}

}  // namespace

inline bool row_ok(int row) { return row == 3 || row == 4 || row == 7 || row == 8; }

#define SG_DISPATCH_ROW(KERNEL, T, FLAG, ROWV, ...)                         \
  switch (ROWV) {                                                           \
    case 3: KERNEL<T, FLAG, 3><<<__VA_ARGS__>>>(a); break;                  \
    case 4: KERNEL<T, FLAG, 4><<<__VA_ARGS__>>>(a); break;                  \
    case 7: KERNEL<T, FLAG, 7><<<__VA_ARGS__>>>(a); break;                  \
    default: KERNEL<T, FLAG, 8><<<__VA_ARGS__>>>(a); break;                 \
  }

template <typename T>
cudaError_t launch_restrict(RestrictArgs<T>& a, bool dim2, cudaStream_t s) {
  if (a.nchains < 1 || a.nchains > kChainSlots || !row_ok(a.row)) return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  if (a.ch <= 0) a.ch = chunk_rows(a.n1, a.n2);
  if (a.ch > a.n1) a.ch = a.n1;
  const long long nb = blocks_for(a.n1, a.n2, a.ch, a.tiled);
  if (nb > (1LL << 24)) return cudaErrorInvalidValue;   // thread index fits 32 bits
  const unsigned b = (unsigned)nb;
  if (dim2) { SG_DISPATCH_ROW(k_restrict, T, true, a.row, b, kThreads, 0, s) }
  else { SG_DISPATCH_ROW(k_restrict, T, false, a.row, b, kThreads, 0, s) }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chain(ChainArgs<T>& a, bool mode_a, cudaStream_t s) {
  if (a.nchains < 1 || a.nchains > kChainSlots || !row_ok(a.row)) return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  if (a.ch <= 0) a.ch = chunk_rows(a.n1, a.n2);
  if (a.ch > a.n1) a.ch = a.n1;
  const long long nb = blocks_for(a.n1, a.n2, a.ch, a.tiled);
  if (nb > (1LL << 24)) return cudaErrorInvalidValue;   // thread index fits 32 bits
  const unsigned b = (unsigned)nb;
  if (mode_a) { SG_DISPATCH_ROW(k_chain, T, true, a.row, b, kThreads, 0, s) }
  else { SG_DISPATCH_ROW(k_chain, T, false, a.row, b, kThreads, 0, s) }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_final(FinalArgs<T>& a, bool left, cudaStream_t s) {
  if (a.nterms < 1 || a.nterms > kFinalTerms || a.nin < 1 || a.nin > kFinalIn || !row_ok(a.row))
    return cudaErrorInvalidValue;
  if (a.tbeg[0] != 0 || a.tbeg[a.nin] != a.nterms) return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  if (a.ch <= 0) a.ch = chunk_rows(a.n1, a.n2);
  if (a.ch > a.n1) a.ch = a.n1;
  const long long nb = blocks_for(a.n1, a.n2, a.ch, a.tiled);
  if (nb > (1LL << 24)) return cudaErrorInvalidValue;   // thread index fits 32 bits
  const unsigned b = (unsigned)nb;
  if (left) { SG_DISPATCH_ROW(k_final, T, true, a.row, b, kThreads, 0, s) }
  else { SG_DISPATCH_ROW(k_final, T, false, a.row, b, kThreads, 0, s) }
  return cudaGetLastError();
}

template cudaError_t launch_restrict<double>(RestrictArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_restrict<float>(RestrictArgs<float>&, bool, cudaStream_t);
template cudaError_t launch_chain<double>(ChainArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_chain<float>(ChainArgs<float>&, bool, cudaStream_t);
template cudaError_t launch_final<double>(FinalArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_final<float>(FinalArgs<float>&, bool, cudaStream_t);

}  // namespace sgdg
