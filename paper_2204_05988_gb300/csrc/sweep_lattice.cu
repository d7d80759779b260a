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
// Loads stay coalesced: the 32 threads of a warp take 32 consecutive k2.
// Absent neighbours at the lattice edges read a clamped in-range element and
// multiply it by 0.
#include "sweep_common.cuh"

namespace sgdg {

namespace {

using namespace sweep;

template <typename T, int R>
__global__ void __launch_bounds__(kThreads) k_final_lat(const __grid_constant__ FinalArgs<T> a) {
  using C = Comp<T>;
  using CP = C2<T>;
  constexpr int W = 8;   // ELL width of the 7-slot rows
  const unsigned n2 = (unsigned)a.n2;
  const int nx = a.lat_nx, ny = a.n1 / a.lat_nx;
  const unsigned nchunk = (unsigned)((nx + R - 1) / R);
  const unsigned v = blockIdx.x * kThreads + threadIdx.x;
  const unsigned q = v / n2;
  const unsigned k2 = v - q * n2;
  if (q >= (unsigned)ny * nchunk) return;
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
        for (int t = a.tbeg[ci]; t < a.tbeg[ci + 1]; ++t) {
          C ev[7];
          ell_vals<7>(a.val[t] + frow, ev);
          const C sx = ev[0] * a0.x + ev[1] * a1.x + ev[2] * b0.x + ev[3] * b1.x + ev[4] * b2.x + ev[5] * c0.x +
                       ev[6] * c1.x;
          const C sy = ev[0] * a0.y + ev[1] * a1.y + ev[2] * b0.y + ev[3] * b1.y + ev[4] * b2.y + ev[5] * c0.y +
                       ev[6] * c1.y;
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

}  // namespace

template <typename T>
cudaError_t launch_final_lattice(FinalArgs<T>& a, cudaStream_t s) {
  if (a.nterms < 1 || a.nterms > kFinalTerms || a.nin < 1 || a.nin > kFinalIn || a.row != 7 || a.lat_nx < 2 ||
      a.n1 % a.lat_nx)
    return cudaErrorInvalidValue;
  if (a.tbeg[0] != 0 || a.tbeg[a.nin] != a.nterms) return cudaErrorInvalidValue;
  if (a.n1 <= 0 || a.n2 <= 0) return cudaSuccess;
  const int R = a.ch <= 4 ? 4 : 8;
  const long long nchunk = (a.lat_nx + R - 1) / R;
  const long long threads = (long long)(a.n1 / a.lat_nx) * nchunk * a.n2;
  const long long nb = (threads + kThreads - 1) / kThreads;
  if (threads > 0xfffff000LL) return cudaErrorInvalidValue;   // 32-bit thread index
  if (R == 4) k_final_lat<T, 4><<<(unsigned)nb, kThreads, 0, s>>>(a);
  else k_final_lat<T, 8><<<(unsigned)nb, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_final_lattice<double>(FinalArgs<double>&, cudaStream_t);
template cudaError_t launch_final_lattice<float>(FinalArgs<float>&, cudaStream_t);
template cudaError_t launch_final_lattice<Bf16>(FinalArgs<Bf16>&, cudaStream_t);

}  // namespace sgdg
