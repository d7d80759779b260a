// Final update along dim 1 on a 2-D structured lattice (sm_103a):
//   y[k1][k2] (+)= sum_c sum_{t in c} tau_t (x) sum_s F_t[k1][s] in_c[k1 + off_s][k2]
// for the x side of the sweep (Sect. 4.2, the factor X_a applied to the
// chain states S_b), when level lx is a lattice of nx x ny vertices whose
// cells are cut along the (1, 1) diagonal: the pattern rows are in
// stencil-slot order, offsets (dx, dy) = (-1,-1), (0,-1), (-1,0), (0,0),
// (1,0), (0,1), (1,1), absent neighbours with value 0.
//
// The generic final kernel gathers all 7 stencil inputs for every output.
// Here a thread runs along R consecutive vertices of one lattice row and
// keeps a window of the inputs in registers: rows iy-1 (2 values), iy (3)
// and iy+1 (2); one step along the row loads 3 new values, so R outputs
// gather 3 R + 4 input elements (3.5 per output at R = 8) instead of 7 R.
// Loads stay coalesced: the 32 threads of a warp take 32 consecutive k2
// (fewer columns: several runs per warp), and the warps of a column tile
// take neighbouring runs, so the three lattice rows a run reads are shared
// through L1 and L2.
// Absent neighbours at the lattice edges read a clamped in-range element and
// multiply it by 0.
#include "sweep_common.cuh"

namespace sgdg {

namespace {

using namespace sweep;

// Thread -> (column k2, work item q) of a lattice launch with nq work items
// (q = lattice row iy and run of vertices along it).  n2 >= 32: the warps of
// one column tile of 32 k2 take consecutive items, so the rows iy - 1 and
// iy + 1 that an item's window reads are read by neighbouring warps of the
// same or nearby blocks; n2 < 32: a warp takes 32 / n2 items of n2 lanes.
__device__ __forceinline__ bool lattice_item(unsigned n2, unsigned nq, unsigned& k2, unsigned& q) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned w = blockIdx.x * (kThreads / 32) + threadIdx.x / 32;
  if (n2 >= 32) {
    const unsigned tile = w / nq;
    q = w - tile * nq;
    k2 = tile * 32 + lane;
    return k2 < n2;
  }
  const unsigned per = 32 / n2, sub = lane / n2;
  if (sub >= per) return false;
  k2 = lane - sub * n2;
  q = w * per + sub;
  return q < nq;
}

// warps of a lattice launch (see lattice_item)
inline long long lattice_warps(long long n2, long long nq) {
  if (n2 >= 32) return (n2 + 31) / 32 * nq;
  const long long per = 32 / n2;
  return (nq + per - 1) / per;
}

template <typename T, int R>
__global__ void __launch_bounds__(kThreads) k_final_lat(const __grid_constant__ FinalArgs<T> a) {
  using C = Comp<T>;
  using CP = C2<T>;
  constexpr int W = 8;   // ELL width of the 7-slot rows
  const unsigned n2 = (unsigned)a.n2;
  const int nx = a.lat_nx, ny = a.n1 / a.lat_nx;
  const unsigned nchunk = (unsigned)((nx + R - 1) / R);
  unsigned k2, q;
  if (!lattice_item(n2, (unsigned)ny * nchunk, k2, q)) return;
  const int iy = (int)(q / nchunk);
  const int ix0 = (int)(q - (unsigned)iy * nchunk) * R;
  const int ym = iy > 0 ? iy - 1 : iy, yp = iy + 1 < ny ? iy + 1 : iy;
  // element (row y, column x clamped to the lattice row) of an input
  auto at = [&](int y, int x) -> size_t {
    x = x < 0 ? 0 : (x >= nx ? nx - 1 : x);
    return (size_t)(y * nx + x) * n2 + k2;
  };
  C ax[R], ay[R];
#pragma unroll
  for (int r = 0; r < R; ++r) ax[r] = ay[r] = 0;
  for (int ci = 0; ci < a.nin; ++ci) {
    const S2<T>* in = reinterpret_cast<const S2<T>*>(a.in[ci]);
    // window at ix0: a = row iy-1 (x-1, x), b = row iy (x-1, x, x+1), c = row iy+1 (x, x+1)
    CP a0 = widen(in[at(ym, ix0 - 1)]), a1 = widen(in[at(ym, ix0)]);
    CP b0 = widen(in[at(iy, ix0 - 1)]), b1 = widen(in[at(iy, ix0)]), b2 = widen(in[at(iy, ix0 + 1)]);
    CP c0 = widen(in[at(yp, ix0)]), c1 = widen(in[at(yp, ix0 + 1)]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int ix = ix0 + r;
      if (ix < nx) {
        const size_t frow = (size_t)(iy * nx + ix) * W;
        const CP w[7] = {a0, a1, b0, b1, b2, c0, c1};   // the slots of row (iy, ix)
        for (int t = a.tbeg[ci]; t < a.tbeg[ci + 1]; ++t) {
          C ev[7];
          ell_vals<7>(a.val[t] + frow, ev);
          // the generic kernel's sums, term by term in slot order
          C sx = 0, sy = 0;
#pragma unroll
          for (int j = 0; j < 7; ++j) {
            sx += ev[j] * w[j].x;
            sy += ev[j] * w[j].y;
          }
          ax[r] += a.tau[t][0] * sx + a.tau[t][1] * sy;
          ay[r] += a.tau[t][2] * sx + a.tau[t][3] * sy;
        }
      }
      if (r + 1 < R) {   // slide one vertex along the row
        a0 = a1;
        a1 = widen(in[at(ym, ix + 1)]);
        b0 = b1;
        b1 = b2;
        b2 = widen(in[at(iy, ix + 2)]);
        c0 = c1;
        c1 = widen(in[at(yp, ix + 2)]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int ix = ix0 + r;
    if (ix >= nx) break;
    const size_t o = (size_t)(iy * nx + ix) * n2 + k2;
    if (a.accumulate) {
      const CP y0 = load2<T>(a.y, o);
      put2(a.y, o, y0.x + ax[r], y0.y + ay[r]);
    } else {
      put2(a.y, o, ax[r], ay[r]);
    }
  }
}

// Chain step in mode A (the branch-A states of Sect. 4.2's sweep and the
// diagonal-block products of the component solves) on a 2-D lattice x level:
//   out_g[k1][k2] = sum_q P[k1][q] Q_g[col_q][k2] + sum_j F_g[k2][j] U[k1][col_j]
// A thread takes R consecutive vertices ix0 .. ix0 + R - 1 of lattice row iy
// and one column k2: U is gathered along the F row once per output (R rows
// in registers, used by every chain), the F row values once per chain for
// all R rows, and the prolongation P1 = E (level lx - 1, a lattice of
// (nx + 1) / 2 columns, cells cut along the same diagonal) from a window of
// the coarse row(s) above: a fine vertex is a coarse vertex (weight 1) or
// the midpoint of a coarse edge - along the row, along the column, or along
// the (1, 1) diagonal (weights 1/2, 1/2).  The sums are those of the generic
// kernel in the same order.
template <typename T, int R>
__global__ void __launch_bounds__(kThreads) k_chain_lat(const __grid_constant__ ChainArgs<T> a) {
  using C = Comp<T>;
  using CP = C2<T>;
  constexpr int ROW = 7, W = 8, M = R / 2 + 1;   // coarse window width
  const unsigned n2 = (unsigned)a.n2;
  const int nx = a.lat_nx, ny = a.n1 / a.lat_nx, nxc = (a.lat_nx + 1) / 2;
  const unsigned nchunk = (unsigned)((nx + R - 1) / R);
  unsigned k2, q;
  if (!lattice_item(n2, (unsigned)ny * nchunk, k2, q)) return;
  const int iy = (int)(q / nchunk);
  const int ix0 = (int)(q - (unsigned)iy * nchunk) * R;   // even (R even)
  unsigned fc[ROW];
  ell_cols<ROW>(a.f_col + (size_t)k2 * W, fc);
  const S2<T>* U = reinterpret_cast<const S2<T>*>(a.U);
  CP u[R][ROW];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int ix = ix0 + r < nx ? ix0 + r : nx - 1;
    const unsigned k1 = (unsigned)(iy * nx + ix);
#pragma unroll
    for (int j = 0; j < ROW; ++j) u[r][j] = widen(U[k1 * (unsigned)a.nu2 + fc[j]]);
  }
  const bool odd = iy & 1;
  const int cy0 = iy >> 1, cy1 = odd ? cy0 + 1 : cy0;
  const int cx0 = ix0 >> 1;
  for (int g = 0; g < a.nchains; ++g) {
    C fv[ROW];
    ell_vals<ROW>(a.f_val[g] + (size_t)k2 * W, fv);
    CP z0[M], z1[M];
    if (a.has_prev) {
      const S2<T>* Z = reinterpret_cast<const S2<T>*>(a.Z[g]);
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int cx = cx0 + m < nxc ? cx0 + m : nxc - 1;
        z0[m] = widen(Z[(size_t)(cy0 * nxc + cx) * n2 + k2]);
        z1[m] = odd ? widen(Z[(size_t)(cy1 * nxc + cx) * n2 + k2]) : z0[m];
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int ix = ix0 + r;
      if (ix >= nx) break;
      C sx = 0, sy = 0;
      if (a.has_prev) {
        const int m = r >> 1;   // coarse column of ix (even) or of ix - 1 (odd)
        if (!odd && !(r & 1)) {            // coarse vertex
          sx = (C)1 * z0[m].x;
          sy = (C)1 * z0[m].y;
        } else if (!odd) {                 // midpoint along the row
          sx = (C)0.5 * z0[m].x;
          sy = (C)0.5 * z0[m].y;
          sx += (C)0.5 * z0[m + 1].x;
          sy += (C)0.5 * z0[m + 1].y;
        } else if (!(r & 1)) {             // midpoint along the column
          sx = (C)0.5 * z0[m].x;
          sy = (C)0.5 * z0[m].y;
          sx += (C)0.5 * z1[m].x;
          sy += (C)0.5 * z1[m].y;
        } else {                           // midpoint of the (1, 1) diagonal
          sx = (C)0.5 * z0[m].x;
          sy = (C)0.5 * z0[m].y;
          sx += (C)0.5 * z1[m + 1].x;
          sy += (C)0.5 * z1[m + 1].y;
        }
      }
#pragma unroll
      for (int j = 0; j < ROW; ++j) {
        sx += fv[j] * u[r][j].x;
        sy += fv[j] * u[r][j].y;
      }
      put2(a.out[g], (size_t)(iy * nx + ix) * n2 + k2, sx, sy);
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_chain_lattice(ChainArgs<T>& a, cudaStream_t s) {
  if (a.nchains < 1 || a.nchains > kChainSlots || a.row != 7 || a.lat_nx < 3 || a.n1 % a.lat_nx ||
      a.nu2 != a.n2)
    return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  const int R = a.ch <= 2 ? 2 : 4;
  const long long nq = (long long)(a.n1 / a.lat_nx) * ((a.lat_nx + R - 1) / R);
  const long long nb = (lattice_warps(a.n2, nq) + kThreads / 32 - 1) / (kThreads / 32);
  if (nb * kThreads > 0xfffff000LL || nq > 0x7fffffffLL) return cudaErrorInvalidValue;   // 32-bit indices
  if (R == 2) k_chain_lat<T, 2><<<(unsigned)nb, kThreads, 0, s>>>(a);
  else k_chain_lat<T, 4><<<(unsigned)nb, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_chain_lattice<float>(ChainArgs<float>&, cudaStream_t);
template cudaError_t launch_chain_lattice<Bf16>(ChainArgs<Bf16>&, cudaStream_t);

template <typename T>
cudaError_t launch_final_lattice(FinalArgs<T>& a, cudaStream_t s) {
  if (a.nterms < 1 || a.nterms > kFinalTerms || a.nin < 1 || a.nin > kFinalIn || a.row != 7 || a.lat_nx < 2 ||
      a.n1 % a.lat_nx)
    return cudaErrorInvalidValue;
  if (a.tbeg[0] != 0 || a.tbeg[a.nin] != a.nterms) return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  const int R = a.ch <= 4 ? 4 : 8;
  const long long nq = (long long)(a.n1 / a.lat_nx) * ((a.lat_nx + R - 1) / R);
  const long long nb = (lattice_warps(a.n2, nq) + kThreads / 32 - 1) / (kThreads / 32);
  if (nb * kThreads > 0xfffff000LL || nq > 0x7fffffffLL) return cudaErrorInvalidValue;   // 32-bit indices
  if (R == 4) k_final_lat<T, 4><<<(unsigned)nb, kThreads, 0, s>>>(a);
  else k_final_lat<T, 8><<<(unsigned)nb, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_final_lattice<double>(FinalArgs<double>&, cudaStream_t);
template cudaError_t launch_final_lattice<float>(FinalArgs<float>&, cudaStream_t);
template cudaError_t launch_final_lattice<Bf16>(FinalArgs<Bf16>&, cudaStream_t);

}  // namespace sgdg
