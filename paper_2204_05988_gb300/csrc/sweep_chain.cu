// Chain steps of the sparse-grid operator sweep (sm_103a), for up to
// kChainSlots chains that share their first factor's pattern:
//  mode A: out_g[k1][k2] = sum_j F_g[k2][j] U[k1][col_j] + sum_q P[k1][q] Q_g[col_q][k2]
//  mode B: out_g[k1][k2] = sum_j F_g[k1][j] U[col_j][k2] + sum_q P[k2][q] Q_g[k1][col_q]
// One thread per column k2 of a chunk of rows.  The shared operand - U
// gathered along the pattern row - is loaded once per element into
// registers and used by every chain; for rows of at most 8 entries the next
// chain's factor row and Q values are loaded before the current chain is
// combined and stored.
#include "sweep_common.cuh"

namespace sgdg {

namespace {

using namespace sweep;

// resident blocks per SM the register budget is sized for: rows of up to 8
// entries keep 4 FP32 blocks; wide rows (restriction-factor products) keep 3
// in mode B and 2 in mode A, whose 2 x 19 gathered U values would spill at 3
template <typename T, int ROW, bool MODE_A>
struct ChainBounds {
  static constexpr int blocks = sizeof(Comp<T>) == 4 ? (ROW > 8 ? (MODE_A ? 2 : 3) : 4) : 2;
};

// MODE: bit 0 - mode A (else B); bit 1 - L2 prefetch hints for the factor
// row and Q values of the chain after next
template <typename T, int MODE, int ROW>
__global__ void __launch_bounds__(kThreads, (ChainBounds<T, ROW, (MODE & 1) != 0>::blocks)) k_chain(const __grid_constant__ ChainArgs<T> a) {
  constexpr bool MODE_A = MODE & 1, PF = (MODE & 2) != 0;
  using C = Comp<T>;
  using CP = C2<T>;
  constexpr int W = Ell<ROW>::W;
  constexpr bool kPrefetch = ROW <= 8;
  const unsigned n2 = (unsigned)a.n2;
  unsigned k2;
  int r0, r1;
  if (!thread_rows(a.n1, a.n2, a.ch, a.tiled, k2, r0, r1)) return;
  unsigned fc[ROW];
  unsigned pc[kProlongRow] = {0, 0};
  C pv[kProlongRow] = {0, 0};
  if (MODE_A) ell_cols<ROW>(a.f_col + (size_t)k2 * W, fc);          // F row k2
  else if (a.has_prev) prolong_row(a.p_col, a.p_val, k2, pc, pv);   // P row k2
  for (int k1 = r0; k1 < r1; ++k1) {
    // the shared operand of the chains: U gathered along the first factor's row
    CP u[ROW];
    unsigned zo[kProlongRow];
    if (MODE_A) {
      unsigned off[ROW];
#pragma unroll
      for (int j = 0; j < ROW; ++j) off[j] = (unsigned)k1 * (unsigned)a.nu2 + fc[j];
      gather<T>(a.U, off, u);
      if (a.has_prev) prolong_row(a.p_col, a.p_val, (unsigned)k1, pc, pv);   // P row k1
#pragma unroll
      for (int q = 0; q < kProlongRow; ++q) zo[q] = pc[q] * n2 + k2;
    } else {
      ell_cols<ROW>(a.f_col + (size_t)k1 * W, fc);   // F row k1 (uniform in a warp)
      unsigned off[ROW];
#pragma unroll
      for (int j = 0; j < ROW; ++j) off[j] = fc[j] * n2 + k2;
      gather<T>(a.U, off, u);
#pragma unroll
      for (int q = 0; q < kProlongRow; ++q) zo[q] = (unsigned)k1 * (unsigned)a.nz2 + pc[q];
    }
    const size_t o = (size_t)k1 * n2 + k2;
    const size_t frow = (size_t)(MODE_A ? k2 : (unsigned)k1) * W;
    C fv[ROW];
    CP z[kProlongRow];
#pragma unroll
    for (int q = 0; q < kProlongRow; ++q) z[q].x = z[q].y = 0;
    if (kPrefetch) ell_vals<ROW>(a.f_val[0] + frow, fv);
    if (a.has_prev) gather<T>(a.Z[0], zo, z);
    for (int g = 0; g < a.nchains; ++g) {
      C cv[ROW];
      CP cz[kProlongRow];
      if (kPrefetch) {
#pragma unroll
        for (int j = 0; j < ROW; ++j) cv[j] = fv[j];
      }
#pragma unroll
      for (int q = 0; q < kProlongRow; ++q) cz[q] = z[q];
      if (g + 1 < a.nchains) {
        if (kPrefetch) ell_vals<ROW>(a.f_val[g + 1] + frow, fv);
        if (a.has_prev) gather<T>(a.Z[g + 1], zo, z);
      }
      if (PF && g + 2 < a.nchains) {
        prefetch_l2(a.f_val[g + 2] + frow);
        if (a.has_prev) {
#pragma unroll
          for (int q = 0; q < kProlongRow; ++q) prefetch_l2(reinterpret_cast<const S2<T>*>(a.Z[g + 2]) + zo[q]);
        }
      }
      if (!kPrefetch) ell_vals<ROW>(a.f_val[g] + frow, cv);
      C zx = 0, zy = 0;
      if (a.has_prev) {
#pragma unroll
        for (int q = 0; q < kProlongRow; ++q) {
          zx += pv[q] * cz[q].x;
          zy += pv[q] * cz[q].y;
        }
      }
#pragma unroll
      for (int j = 0; j < ROW; ++j) {
        zx += cv[j] * u[j].x;
        zy += cv[j] * u[j].y;
      }
      put2(a.out[g], o, zx, zy);
    }
  }
}

// Mode A with rows of at most 8 entries, two rows (k1, k1 + 1) per thread:
// the factor row k2 is loaded once per chain for both rows (the
// diagonal-block products W_b = U V_b^T, and S_b = W_b + P1 Q_b); the next
// chain's Q values are loaded before the current chain is combined.
// MODE: bit 0 set (mode A); bit 1 - L2 prefetch hints for the factor row
// of the next chain and the Q values of the chain after next
template <typename T, int MODE, int ROW>
__global__ void __launch_bounds__(kThreads, (sizeof(Comp<T>) == 4 ? 3 : 2)) k_chain_pair(const __grid_constant__ ChainArgs<T> a) {
  static_assert((MODE & 1) && ROW <= 8, "row pairs: mode A, short rows");
  constexpr bool PF = (MODE & 2) != 0;
  using C = Comp<T>;
  using CP = C2<T>;
  constexpr int W = Ell<ROW>::W;
  const unsigned n2 = (unsigned)a.n2;
  unsigned k2;
  int r0, r1;
  if (!thread_rows(a.n1, a.n2, a.ch, a.tiled, k2, r0, r1)) return;
  unsigned fc[ROW];
  ell_cols<ROW>(a.f_col + (size_t)k2 * W, fc);
  const S2<T>* U = reinterpret_cast<const S2<T>*>(a.U);
  const size_t frow = (size_t)k2 * W;
  for (int k1 = r0; k1 < r1; k1 += 2) {
    const bool b_ok = k1 + 1 < r1;
    CP ua[ROW], ub[ROW];
#pragma unroll
    for (int j = 0; j < ROW; ++j) {
      const unsigned off = (unsigned)k1 * (unsigned)a.nu2 + fc[j];
      ua[j] = widen(U[off]);
      if (b_ok) ub[j] = widen(U[off + (unsigned)a.nu2]);
      else ub[j].x = ub[j].y = 0;
    }
    // prolongation rows k1, k1 + 1 and their Q offsets
    unsigned pca[kProlongRow] = {0, 0}, pcb[kProlongRow] = {0, 0};
    C pva[kProlongRow] = {0, 0}, pvb[kProlongRow] = {0, 0};
    unsigned zoa[kProlongRow] = {0, 0}, zob[kProlongRow] = {0, 0};
    if (a.has_prev) {
      prolong_row(a.p_col, a.p_val, (unsigned)k1, pca, pva);
      if (b_ok) prolong_row(a.p_col, a.p_val, (unsigned)k1 + 1, pcb, pvb);
      else pcb[0] = pcb[1] = pca[0];
#pragma unroll
      for (int q = 0; q < kProlongRow; ++q) {
        zoa[q] = pca[q] * n2 + k2;
        zob[q] = pcb[q] * n2 + k2;
      }
    }
    const size_t o = (size_t)k1 * n2 + k2;
    CP za[kProlongRow], zb[kProlongRow];
#pragma unroll
    for (int q = 0; q < kProlongRow; ++q) za[q].x = za[q].y = zb[q].x = zb[q].y = 0;
    if (a.has_prev) {
      gather<T>(a.Z[0], zoa, za);
      gather<T>(a.Z[0], zob, zb);
    }
    for (int g = 0; g < a.nchains; ++g) {
      C cv[ROW];
      CP cza[kProlongRow], czb[kProlongRow];
      ell_vals<ROW>(a.f_val[g] + frow, cv);
#pragma unroll
      for (int q = 0; q < kProlongRow; ++q) {
        cza[q] = za[q];
        czb[q] = zb[q];
      }
      if (g + 1 < a.nchains) {
        if (PF) prefetch_l2(a.f_val[g + 1] + frow);
        if (a.has_prev) {
          gather<T>(a.Z[g + 1], zoa, za);
          gather<T>(a.Z[g + 1], zob, zb);
        }
      }
      if (PF && a.has_prev && g + 2 < a.nchains) {
        const S2<T>* zn = reinterpret_cast<const S2<T>*>(a.Z[g + 2]);
#pragma unroll
        for (int q = 0; q < kProlongRow; ++q) {
          prefetch_l2(zn + zoa[q]);
          prefetch_l2(zn + zob[q]);
        }
      }
      C ax = 0, ay = 0, bx = 0, by = 0;
      if (a.has_prev) {
#pragma unroll
        for (int q = 0; q < kProlongRow; ++q) {
          ax += pva[q] * cza[q].x;
          ay += pva[q] * cza[q].y;
          bx += pvb[q] * czb[q].x;
          by += pvb[q] * czb[q].y;
        }
      }
#pragma unroll
      for (int j = 0; j < ROW; ++j) {
        ax += cv[j] * ua[j].x;
        ay += cv[j] * ua[j].y;
        bx += cv[j] * ub[j].x;
        by += cv[j] * ub[j].y;
      }
      put2(a.out[g], o, ax, ay);
      if (b_ok) put2(a.out[g], o + n2, bx, by);
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_chain(ChainArgs<T>& a, bool mode_a, cudaStream_t s) {
  if (a.nchains < 1 || a.nchains > kChainSlots || row_class(a.row) != a.row || a.row > kMaxChainRow)
    return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  if (a.nu2 <= 0) a.nu2 = a.n2;
  unsigned b = 0;
  if (a.pair && mode_a && a.row <= 8) {
    if (a.ch <= 0 || a.ch % 2) a.ch = a.ch <= 0 ? 2 : a.ch + 1;
    if (!launch_shape(a.n1, a.n2, a.ch, a.tiled, b)) return cudaErrorInvalidValue;
    if (a.pf) { SG_SWEEP_DISPATCH(k_chain_pair, T, 3, a.row, 8, b, kThreads, 0, s) }
    else { SG_SWEEP_DISPATCH(k_chain_pair, T, 1, a.row, 8, b, kThreads, 0, s) }
    return cudaGetLastError();
  }
  if (!launch_shape(a.n1, a.n2, a.ch, a.tiled, b)) return cudaErrorInvalidValue;
  switch ((mode_a ? 1 : 0) | (a.pf ? 2 : 0)) {
    case 0: SG_SWEEP_DISPATCH(k_chain, T, 0, a.row, kMaxChainRow, b, kThreads, 0, s) break;
    case 1: SG_SWEEP_DISPATCH(k_chain, T, 1, a.row, kMaxChainRow, b, kThreads, 0, s) break;
    case 2: SG_SWEEP_DISPATCH(k_chain, T, 2, a.row, kMaxChainRow, b, kThreads, 0, s) break;
    default: SG_SWEEP_DISPATCH(k_chain, T, 3, a.row, kMaxChainRow, b, kThreads, 0, s) break;
  }
  return cudaGetLastError();
}

template cudaError_t launch_chain<double>(ChainArgs<double>&, bool, cudaStream_t);
template cudaError_t launch_chain<float>(ChainArgs<float>&, bool, cudaStream_t);
template cudaError_t launch_chain<Bf16>(ChainArgs<Bf16>&, bool, cudaStream_t);

}  // namespace sgdg
