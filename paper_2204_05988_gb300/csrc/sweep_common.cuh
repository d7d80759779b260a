// Device helpers shared by the sweep kernels: thread-to-element mapping,
// ELL row loads and gathers.
#pragma once

#include <cuda_runtime.h>

#include "sweep.h"

namespace sgdg {
namespace sweep {

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };
template <> struct V2<__nv_bfloat16> { using type = __nv_bfloat162; };

// the (time slot 0, time slot 1) pair of one grid element: storage and
// arithmetic forms of precision T
template <typename T> using S2 = typename V2<Store<T>>::type;
template <typename T> using C2 = typename V2<Comp<T>>::type;

__device__ __forceinline__ double2 widen(double2 v) { return v; }
__device__ __forceinline__ float2 widen(float2 v) { return v; }
__device__ __forceinline__ float2 widen(__nv_bfloat162 v) { return __bfloat1622float2(v); }

// pair p of a grid array in arithmetic form
template <typename T>
__device__ __forceinline__ C2<T> load2(const Store<T>* g, size_t p) {
  return widen(reinterpret_cast<const S2<T>*>(g)[p]);
}
// store (x, y) as pair p (rounded to nearest for BF16 storage)
__device__ __forceinline__ void put2(double* g, size_t p, double x, double y) {
  reinterpret_cast<double2*>(g)[p] = make_double2(x, y);
}
__device__ __forceinline__ void put2(float* g, size_t p, float x, float y) {
  reinterpret_cast<float2*>(g)[p] = make_float2(x, y);
}
__device__ __forceinline__ void put2(__nv_bfloat16* g, size_t p, float x, float y) {
  reinterpret_cast<__nv_bfloat162*>(g)[p] = __floats2bfloat162_rn(x, y);
}

constexpr int kThreads = 256;
constexpr int kChunksPerBlock = kThreads / kTileW;

// rows per thread when the autotuner has not chosen one
inline int chunk_rows(long long n1, long long n2) {
  const long long want = 152LL * 2048 * 2;
  long long ch = (n1 * n2 + want - 1) / want;
  ch = ch < 1 ? 1 : (ch > 8 ? 8 : ch);
  return (int)(ch > n1 ? n1 : ch);
}

inline long long blocks_for(int n1, int n2, int ch, int tiled) {
  const long long nchunk = ((long long)n1 + ch - 1) / ch;
  if (tiled) return ((n2 + kTileW - 1) / kTileW) * ((nchunk + kChunksPerBlock - 1) / kChunksPerBlock);
  return (nchunk * n2 + kThreads - 1) / kThreads;
}

// Launch shape of an (n1 x n2) launch; false when the grid is too large for
// 32-bit thread indices.
inline bool launch_shape(int n1, int n2, int& ch, int tiled, unsigned& blocks) {
  if (ch <= 0) ch = chunk_rows(n1, n2);
  if (ch > n1) ch = n1;
  const long long nb = blocks_for(n1, n2, ch, tiled);
  if (nb > (1LL << 24)) return false;
  blocks = (unsigned)nb;
  return true;
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
  static constexpr int W = (ROW + 3) / 4 * 4;
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

// Hint: bring the L2 line holding p on chip ahead of its load (holds no
// register, never waits; the address is one the thread loads later).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// pairs off[j] of a grid array, widened to the arithmetic type
template <typename T, int N>
__device__ __forceinline__ void gather(const Store<T>* base, const unsigned (&off)[N], C2<T> (&w)[N]) {
  const S2<T>* b = reinterpret_cast<const S2<T>*>(base);
#pragma unroll
  for (int j = 0; j < N; ++j) w[j] = widen(b[off[j]]);
}

}  // namespace sweep
}  // namespace sgdg

// Launch KERNEL<T, FLAG, row> for the row classes up to MAXROW.
#define SG_SWEEP_DISPATCH(KERNEL, T, FLAG, ROWV, MAXROW, ...)                                   \
  switch (ROWV) {                                                                               \
    case 3: KERNEL<T, FLAG, 3><<<__VA_ARGS__>>>(a); break;                                      \
    case 4: KERNEL<T, FLAG, 4><<<__VA_ARGS__>>>(a); break;                                      \
    case 5: KERNEL<T, FLAG, 5><<<__VA_ARGS__>>>(a); break;                                      \
    case 7: KERNEL<T, FLAG, 7><<<__VA_ARGS__>>>(a); break;                                      \
    case 8: KERNEL<T, FLAG, 8><<<__VA_ARGS__>>>(a); break;                                      \
    case 12: if (MAXROW >= 12) KERNEL<T, FLAG, (MAXROW >= 12 ? 12 : 8)><<<__VA_ARGS__>>>(a); break; \
    case 16: if (MAXROW >= 16) KERNEL<T, FLAG, (MAXROW >= 16 ? 16 : 8)><<<__VA_ARGS__>>>(a); break; \
    case 19: if (MAXROW >= 19) KERNEL<T, FLAG, (MAXROW >= 19 ? 19 : 8)><<<__VA_ARGS__>>>(a); break; \
    case 20: if (MAXROW >= 20) KERNEL<T, FLAG, (MAXROW >= 20 ? 20 : 8)><<<__VA_ARGS__>>>(a); break; \
    case 24: if (MAXROW >= 24) KERNEL<T, FLAG, (MAXROW >= 24 ? 24 : 8)><<<__VA_ARGS__>>>(a); break; \
    default: break;                                                                             \
  }
