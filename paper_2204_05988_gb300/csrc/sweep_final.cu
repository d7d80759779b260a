// Final updates of the sparse-grid operator sweep (sm_103a):
//   y (+)= sum_c sum_{t in c} tau_t (x) F_t in_c
// with F_t along dim 1 (left) or dim 2 (right) on one shared pattern.  One
// thread per column k2 of a chunk of rows: the gather offsets of the
// pattern row are computed once and serve every input; the next input's
// values are loaded while the current one is combined with its terms.
#include "sweep_common.cuh"

namespace sgdg {

namespace {

using namespace sweep;

// MODE: bit 0 - left (dim 1) or right (dim 2); bit 1 - L2 prefetch hints
template <typename T, int MODE, int ROW>
__global__ void __launch_bounds__(kThreads) k_final(const __grid_constant__ FinalArgs<T> a) {
  constexpr bool LEFT = MODE & 1, PF = (MODE & 2) != 0;
  using C = Comp<T>;
  using CP = C2<T>;
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
    for (int j = 0; j < ROW; ++j) off[j] = LEFT ? fc[j] * n2 + k2 : (unsigned)k1 * (unsigned)a.nin2 + fc[j];
    const size_t frow = (size_t)(LEFT ? (unsigned)k1 : k2) * W;
    const size_t o = (size_t)k1 * n2 + k2;
    C yx = 0, yy = 0;
    CP w[ROW];
    gather<T>(a.in[0], off, w);
    for (int ci = 0; ci < a.nin; ++ci) {
      CP cw[ROW];
#pragma unroll
      for (int j = 0; j < ROW; ++j) cw[j] = w[j];
      if (ci + 1 < a.nin) gather<T>(a.in[ci + 1], off, w);
      if (PF && ci + 2 < a.nin) {
#pragma unroll
        for (int j = 0; j < ROW; ++j) prefetch_l2(reinterpret_cast<const S2<T>*>(a.in[ci + 2]) + off[j]);
      }
      for (int t = a.tbeg[ci]; t < a.tbeg[ci + 1]; ++t) {
        C ev[ROW];
        ell_vals<ROW>(a.val[t] + frow, ev);
        C sx = 0, sy = 0;
#pragma unroll
        for (int j = 0; j < ROW; ++j) {
          sx += ev[j] * cw[j].x;
          sy += ev[j] * cw[j].y;
        }
        yx += a.tau[t][0] * sx + a.tau[t][1] * sy;
        yy += a.tau[t][2] * sx + a.tau[t][3] * sy;
      }
    }
    if (a.accumulate) {
      const CP r = load2<T>(a.y, o);
      put2(a.y, o, r.x + yx, r.y + yy);
    } else {
      put2(a.y, o, yx, yy);
    }
  }
}

// Two outputs per thread that share the pattern row, its values and the
// time coupling: left - columns k2 and k2 + 32 of one row (the warp covers
// 64 consecutive columns, both loads coalesced); right - rows k1 and k1 + 1
// of one column.
template <typename T, int MODE, int ROW>
__global__ void __launch_bounds__(kThreads, sizeof(Comp<T>) == 4 ? 4 : 2) k_final2(const __grid_constant__ FinalArgs<T> a) {
  constexpr bool LEFT = MODE & 1, PF = (MODE & 2) != 0;
  using C = Comp<T>;
  using CP = C2<T>;
  constexpr int W = Ell<ROW>::W;
  const unsigned n2 = (unsigned)a.n2;
  // left: the thread grid runs over column pairs, 32 pairs per 64 columns
  const int ncol = LEFT ? (a.n2 + 63) / 64 * 32 : a.n2;
  unsigned kc;
  int r0, r1;
  if (!thread_rows(a.n1, ncol, a.ch, a.tiled, kc, r0, r1)) return;
  const unsigned k2 = LEFT ? (kc >> 5) * 64 + (kc & 31) : kc;
  if (k2 >= n2) return;
  const bool has_b = LEFT ? k2 + 32 < n2 : true;
  unsigned fc[ROW];
  if (!LEFT) ell_cols<ROW>(a.col + (size_t)k2 * W, fc);
  for (int k1 = r0; k1 < r1; k1 += LEFT ? 1 : 2) {
    const bool b_ok = LEFT ? has_b : k1 + 1 < r1;
    if (LEFT) ell_cols<ROW>(a.col + (size_t)k1 * W, fc);
    unsigned off[ROW];
#pragma unroll
    for (int j = 0; j < ROW; ++j) off[j] = LEFT ? fc[j] * n2 + k2 : (unsigned)k1 * (unsigned)a.nin2 + fc[j];
    const unsigned step_b = LEFT ? 32u : (unsigned)a.nin2;   // second output's gather offset
    const size_t frow = (size_t)(LEFT ? (unsigned)k1 : k2) * W;
    C ax = 0, ay = 0, bx = 0, by = 0;
    for (int ci = 0; ci < a.nin; ++ci) {
      const S2<T>* in = reinterpret_cast<const S2<T>*>(a.in[ci]);
      if (PF && ci + 1 < a.nin) {
        const S2<T>* nx = reinterpret_cast<const S2<T>*>(a.in[ci + 1]);
#pragma unroll
        for (int j = 0; j < ROW; ++j) {
          prefetch_l2(nx + off[j]);
          if (b_ok) prefetch_l2(nx + off[j] + step_b);
        }
      }
      CP wa[ROW], wb[ROW];
#pragma unroll
      for (int j = 0; j < ROW; ++j) {
        wa[j] = widen(in[off[j]]);
        if (b_ok) wb[j] = widen(in[off[j] + step_b]);
        else wb[j].x = wb[j].y = 0;
      }
      for (int t = a.tbeg[ci]; t < a.tbeg[ci + 1]; ++t) {
        C ev[ROW];
        ell_vals<ROW>(a.val[t] + frow, ev);
        C sax = 0, say = 0, sbx = 0, sby = 0;
#pragma unroll
        for (int j = 0; j < ROW; ++j) {
          sax += ev[j] * wa[j].x;
          say += ev[j] * wa[j].y;
          sbx += ev[j] * wb[j].x;
          sby += ev[j] * wb[j].y;
        }
        const C t0 = a.tau[t][0], t1 = a.tau[t][1], t2 = a.tau[t][2], t3 = a.tau[t][3];
        ax += t0 * sax + t1 * say;
        ay += t2 * sax + t3 * say;
        bx += t0 * sbx + t1 * sby;
        by += t2 * sbx + t3 * sby;
      }
    }
    const size_t oa = (size_t)k1 * n2 + k2;
    const size_t ob = LEFT ? oa + 32 : oa + n2;
    if (a.accumulate) {
      const CP r = load2<T>(a.y, oa);
      put2(a.y, oa, r.x + ax, r.y + ay);
    } else {
      put2(a.y, oa, ax, ay);
    }
    if (b_ok) {
      if (a.accumulate) {
        const CP r = load2<T>(a.y, ob);
        put2(a.y, ob, r.x + bx, r.y + by);
      } else {
        put2(a.y, ob, bx, by);
      }
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_final(FinalArgs<T>& a, bool left, cudaStream_t s) {
  if (a.nterms < 1 || a.nterms > kFinalTerms || a.nin < 1 || a.nin > kFinalIn || row_class(a.row) != a.row ||
      a.row > kMaxFinalRow)
    return cudaErrorInvalidValue;
  if (a.tbeg[0] != 0 || a.tbeg[a.nin] != a.nterms) return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  if (a.nin2 <= 0) a.nin2 = a.n2;
  unsigned b = 0;
  if (a.pair) {
    // left: column pairs (32 per 64 columns); right: row pairs (ch even)
    if (!left && (a.ch <= 0 || a.ch % 2)) a.ch = a.ch <= 0 ? 2 : a.ch + 1;
    const int ncol = left ? (a.n2 + 63) / 64 * 32 : a.n2;
    if (!launch_shape(a.n1, ncol, a.ch, a.tiled, b)) return cudaErrorInvalidValue;
    switch ((left ? 1 : 0) | (a.pf ? 2 : 0)) {
      case 0: SG_SWEEP_DISPATCH(k_final2, T, 0, a.row, kMaxFinalRow, b, kThreads, 0, s) break;
      case 1: SG_SWEEP_DISPATCH(k_final2, T, 1, a.row, kMaxFinalRow, b, kThreads, 0, s) break;
      case 2: SG_SWEEP_DISPATCH(k_final2, T, 2, a.row, kMaxFinalRow, b, kThreads, 0, s) break;
      default: SG_SWEEP_DISPATCH(k_final2, T, 3, a.row, kMaxFinalRow, b, kThreads, 0, s) break;
    }
    return cudaGetLastError();
  }
  if (!launch_shape(a.n1, a.n2, a.ch, a.tiled, b)) return cudaErrorInvalidValue;
  switch ((left ? 1 : 0) | (a.pf ? 2 : 0)) {
    case 0: SG_SWEEP_DISPATCH(k_final, T, 0, a.row, kMaxFinalRow, b, kThreads, 0, s) break;
    case 1: SG_SWEEP_DISPATCH(k_final, T, 1, a.row, kMaxFinalRow, b, kThreads, 0, s) break;
    case 2: SG_SWEEP_DISPATCH(k_final, T, 2, a.row, kMaxFinalRow, b, kThreads, 0, s) break;
    default: SG_SWEEP_DISPATCH(k_final, T, 3, a.row, kMaxFinalRow, b, kThreads, 0, s) break;
  }
  return cudaGetLastError();
}

template cudaError_t launch_final<double>(FinalArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_final<float>(FinalArgs<float>&, bool, cudaStream_t);
template cudaError_t launch_final<Bf16>(FinalArgs<Bf16>&, bool, cudaStream_t);

}  // namespace sgdg
