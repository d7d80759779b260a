// Restriction of chain intermediates along one dimension (sm_103a): the
// transfer half of a sweep step that moves a chain to the next grid.
//   dim 1:  Q_g = R in_g,    dim 2:  Q_g = in_g R^T
// One thread per column k2 of a chunk of rows; R's row is held in registers
// and applied to every chain of the launch (the gather offsets are shared).
#include "sweep_common.cuh"

namespace sgdg {

namespace {

using namespace sweep;

template <typename T, bool DIM2, int ROW>
__global__ void __launch_bounds__(kThreads) k_restrict(const __grid_constant__ RestrictArgs<T> a) {
  using C = Comp<T>;
  constexpr int W = Ell<ROW>::W;
  const unsigned n2 = (unsigned)a.n2;
  unsigned k2;
  int r0, r1;
  if (!thread_rows(a.n1, a.n2, a.ch, a.tiled, k2, r0, r1)) return;
  unsigned rc[ROW];
  C rv[ROW];
  if (DIM2) {
    // Q[k1][k2] = sum_j R[k2][j] in[k1][col_j]: row k2 of R, reused over the rows
    ell_cols<ROW>(a.col + (size_t)k2 * W, rc);
    ell_vals<ROW>(a.val + (size_t)k2 * W, rv);
  }
  for (int k1 = r0; k1 < r1; ++k1) {
    if (!DIM2) {
      // Q[k1][k2] = sum_j R[k1][j] in[col_j][k2]: row k1 of R (uniform in a warp)
      ell_cols<ROW>(a.col + (size_t)k1 * W, rc);
      ell_vals<ROW>(a.val + (size_t)k1 * W, rv);
    }
    unsigned off[ROW];
#pragma unroll
    for (int j = 0; j < ROW; ++j) off[j] = DIM2 ? (unsigned)k1 * (unsigned)a.n2_in + rc[j] : rc[j] * n2 + k2;
    const size_t o = (size_t)k1 * n2 + k2;
    for (int g = 0; g < a.nchains; ++g) {
      C2<T> w[ROW];
      gather<T>(a.in[g], off, w);
      C sx = 0, sy = 0;
#pragma unroll
      for (int j = 0; j < ROW; ++j) {
        sx += rv[j] * w[j].x;
        sy += rv[j] * w[j].y;
      }
      put2(a.out[g], o, sx, sy);
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_restrict(RestrictArgs<T>& a, bool dim2, cudaStream_t s) {
  if (a.nchains < 1 || a.nchains > kChainSlots || row_class(a.row) != a.row || a.row > kMaxRestrictRow)
    return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  unsigned b = 0;
  if (!launch_shape(a.n1, a.n2, a.ch, a.tiled, b)) return cudaErrorInvalidValue;
  if (dim2) { SG_SWEEP_DISPATCH(k_restrict, T, true, a.row, kMaxRestrictRow, b, kThreads, 0, s) }
  else { SG_SWEEP_DISPATCH(k_restrict, T, false, a.row, kMaxRestrictRow, b, kThreads, 0, s) }
  return cudaGetLastError();
}

template cudaError_t launch_restrict<double>(RestrictArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_restrict<float>(RestrictArgs<float>&, bool, cudaStream_t);
template cudaError_t launch_restrict<Bf16>(RestrictArgs<Bf16>&, bool, cudaStream_t);

}  // namespace sgdg
