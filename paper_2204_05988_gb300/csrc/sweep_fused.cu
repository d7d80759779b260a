// Fused branch-A step of the sparse-grid operator sweep (sm_103a).
//
// Branch A of the sweep (sources l1' <= l1) carries, per distinct v factor
// b, the state S_{b,i} = U_i V_b^T + P1 Z_{b,i} of grid i; the grid's output
// takes Y_i = sum_a tau_a X_a S_{b(a),i} and the next grid receives
// Z_{b,i+1} = S_{b,i} R2^T.  Unfused, every S_b is a full-grid array written
// to HBM and read back twice.  Here one block takes one tile of the grid: an
// x patch of rows with the rows its dim-1 stencils reach, times a v patch of
// columns with the fine columns its restriction rows reach (both built on
// the host from the level patterns, so any mesh works).  For each group of G
// chains the block
//   1. forms S_b on every (row, column) of the tile in shared memory
//      (U gathered along V_b's pattern row, the prolonged coarse state P1 Z_b),
//   2. folds sum_a tau_a X_a S_b into per-thread accumulators for the tile's
//      interior outputs (the X stencil reads neighbouring rows of the tile),
//   3. writes Z'_b = S_b R2^T for the coarse columns the v patch owns,
// and finally stores the interior outputs.  HBM sees U, the coarse states
// and Y only.
#include "sweep_common.cuh"

namespace sgdg {

namespace {

using namespace sweep;

template <typename T, int W>
__global__ void __launch_bounds__(kFusedThreads, 1) k_fused_a(const __grid_constant__ FusedArgs<T> a) {
  using C = Comp<T>;
  using CP = C2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CP* S = reinterpret_cast<CP*>(smem_raw);
  const FusedTile t = a.tiles[blockIdx.x];
  const int nS = t.nxt * t.nvt;
  const int nO = t.nxi * t.nvi;
  const unsigned n2 = (unsigned)a.n2;
  C ax[kFusedOut], ay[kFusedOut];
#pragma unroll
  for (int k = 0; k < kFusedOut; ++k) ax[k] = ay[k] = 0;
  for (int g0 = 0; g0 < a.nchains; g0 += a.G) {
    const int gn = min(a.G, a.nchains - g0);
    // 1. S_b on the whole tile
    for (int idx = threadIdx.x; idx < nS; idx += blockDim.x) {
      const int r = idx / t.nvt, c = idx - r * t.nvt;
      const unsigned k1 = (unsigned)a.xrows[t.xs0 + r], k2 = (unsigned)a.vcols[t.vs0 + c];
      unsigned vc[W];
      ell_cols<W>(a.vcol + (size_t)k2 * W, vc);
      unsigned off[W];
#pragma unroll
      for (int j = 0; j < W; ++j) off[j] = k1 * n2 + vc[j];
      CP u[W];
      gather<T>(a.U, off, u);
      unsigned pc[kProlongRow] = {0, 0};
      C pv[kProlongRow] = {0, 0};
      if (a.has_prev) prolong_row(a.pcol, a.pval, k1, pc, pv);
      for (int g = 0; g < gn; ++g) {
        C fv[W];
        ell_vals<W>(a.vval[g0 + g] + (size_t)k2 * W, fv);
        C sx = 0, sy = 0;
        if (a.has_prev) {
#pragma unroll
          for (int q = 0; q < kProlongRow; ++q) {
            const CP z = load2<T>(a.zin[g0 + g], (size_t)pc[q] * n2 + k2);
            sx += pv[q] * z.x;
            sy += pv[q] * z.y;
          }
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
          sx += fv[j] * u[j].x;
          sy += fv[j] * u[j].y;
        }
        CP v;
        v.x = sx;
        v.y = sy;
        S[(size_t)g * nS + idx] = v;
      }
    }
    __syncthreads();
    // 2. y += sum_a tau_a X_a S_b on the interior
#pragma unroll
    for (int k = 0; k < kFusedOut; ++k) {
      const int idx = threadIdx.x + k * blockDim.x;
      if (idx < nO) {
        const int r = idx / t.nvi, c = idx - r * t.nvi;
        const unsigned k1 = (unsigned)a.xrows[t.xs0 + r];
        int loc[W];
#pragma unroll
        for (int j = 0; j < W; ++j) loc[j] = a.xnbr[t.xn0 + r * W + j] * t.nvt + c;
        for (int g = 0; g < gn; ++g) {
          const CP* Sg = S + (size_t)g * nS;
          CP w[W];
#pragma unroll
          for (int j = 0; j < W; ++j) w[j] = Sg[loc[j]];
          for (int tt = a.tbeg[g0 + g]; tt < a.tbeg[g0 + g + 1]; ++tt) {
            C ev[W];
            ell_vals<W>(a.xval[tt] + (size_t)k1 * W, ev);
            C sx = 0, sy = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) {
              sx += ev[j] * w[j].x;
              sy += ev[j] * w[j].y;
            }
            ax[k] += a.tau[tt][0] * sx + a.tau[tt][1] * sy;
            ay[k] += a.tau[tt][2] * sx + a.tau[tt][3] * sy;
          }
        }
      }
    }
    // 3. Z'_b = S_b R2^T on the owned coarse columns
    if (a.restrict_out) {
      const int nQ = t.nxi * t.nq;
      for (int idx = threadIdx.x; idx < nQ; idx += blockDim.x) {
        const int r = idx / t.nq, qi = idx - r * t.nq;
        const unsigned k1 = (unsigned)a.xrows[t.xs0 + r];
        const unsigned c2 = (unsigned)a.qcols[t.q0 + qi];
        int loc[W];
#pragma unroll
        for (int j = 0; j < W; ++j) loc[j] = r * t.nvt + a.qloc[(size_t)(t.q0 + qi) * W + j];
        C rv[W];
        ell_vals<W>(a.rval + (size_t)c2 * W, rv);
        for (int g = 0; g < gn; ++g) {
          const CP* Sg = S + (size_t)g * nS;
          C sx = 0, sy = 0;
#pragma unroll
          for (int j = 0; j < W; ++j) {
            const CP w = Sg[loc[j]];
            sx += rv[j] * w.x;
            sy += rv[j] * w.y;
          }
          put2(a.zout[g0 + g], (size_t)k1 * a.n2c + c2, sx, sy);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < kFusedOut; ++k) {
    const int idx = threadIdx.x + k * blockDim.x;
    if (idx < nO) {
      const int r = idx / t.nvi, c = idx - r * t.nvi;
      const size_t o = (size_t)a.xrows[t.xs0 + r] * n2 + (unsigned)a.vcols[t.vs0 + c];
      put2(a.Y, o, ax[k], ay[k]);
    }
  }
}

}  // namespace

// dynamic shared memory a block of the fused kernel may use
constexpr int kFusedSmemMax = 220 * 1024;

template <typename T, int W>
cudaError_t launch_w(const FusedArgs<T>& a, size_t smem, cudaStream_t s) {
  static bool attr[64] = {};   // the opt-in above 48 KB, once per instantiation and device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    if (cudaFuncSetAttribute(k_fused_a<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmemMax) !=
        cudaSuccess)
      return cudaErrorInvalidValue;
    attr[dev] = true;
  }
  k_fused_a<T, W><<<a.ntiles, kFusedThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fused_a(const FusedArgs<T>& a, size_t smem, cudaStream_t s) {
  if (a.ntiles <= 0) return cudaSuccess;
  if (a.nchains < 1 || a.nchains > kFusedChains || a.G < 1 || a.tbeg[a.nchains] > kFusedTerms ||
      smem > (size_t)kFusedSmemMax)
    return cudaErrorInvalidValue;
  switch (a.W) {
    case 4: return launch_w<T, 4>(a, smem, s);
    case 8: return launch_w<T, 8>(a, smem, s);
    case 16: return launch_w<T, 16>(a, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_fused_a<double>(const FusedArgs<double>&, size_t, cudaStream_t);
template cudaError_t launch_fused_a<float>(const FusedArgs<float>&, size_t, cudaStream_t);
template cudaError_t launch_fused_a<Bf16>(const FusedArgs<Bf16>&, size_t, cudaStream_t);

}  // namespace sgdg
