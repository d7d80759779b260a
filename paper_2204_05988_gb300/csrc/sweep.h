// Arguments of the sweep kernels (sweep_restrict.cu, sweep_chain.cu,
// sweep_final.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sgdg {

// Precision of a sweep, named by a type: double and float store every grid
// array (inputs, chain states, outputs) and compute in that type; Bf16
// stores the grid arrays in bfloat16 and computes in FP32, with FP32 matrix
// values (the BF16-storage variant: half the bytes per grid element).
struct Bf16 {};
template <typename T> struct Prec { using S = T; using C = T; };
template <> struct Prec<Bf16> { using S = __nv_bfloat16; using C = float; };
template <typename T> using Store = typename Prec<T>::S;   // grid element
template <typename T> using Comp = typename Prec<T>::C;    // arithmetic and matrix values

template <typename T>
constexpr int kChainMax() { return 32; }   // chains per chain-step launch
constexpr int kChainSlots = 32;
constexpr int kFinalIn = 32;      // chain inputs per final launch
constexpr int kFinalTerms = 64;   // terms per final launch
constexpr int kProlongRow = 2;    // entries of a prolongation row (nested P1 refinement)

// Block orders of the sweep kernels (every kernel maps a thread to one
// column k2 and a chunk of `ch` consecutive rows k1):
//  tiled = 0: threads in row-major order over (row chunk, k2) - neighbours
//             along k2 (dim-2 stencils) are read by the same or the next block;
//  tiled = 1: column tiles of kTileW columns, a block holds kThreads / kTileW
//             row chunks of one tile and consecutive blocks take consecutive
//             row chunks - the rows a dim-1 stencil reaches (one mesh row
//             away) are read by blocks that run at the same time.
constexpr int kTileW = 64;

// Matrices reach the sweep kernels in ELL form: row r's entries at
// [r w, r w + w) of a column and a value array, w = the longest row rounded
// up to a multiple of 4 (16-byte rows for vector loads; prolongation: w = 2),
// zero values in the padding.  `row` is the register row length a launch is
// compiled for: row_class(longest row), with ELL width (row + 3) / 4 * 4.
inline int row_class(int r) {
  if (r <= 3) return 3;
  if (r <= 4) return 4;
  if (r <= 5) return 5;
  if (r <= 7) return 7;
  if (r <= 8) return 8;
  if (r <= 12) return 12;
  if (r <= 16) return 16;
  if (r <= 19) return 19;
  if (r <= 20) return 20;
  if (r <= 24) return 24;
  return -1;
}
constexpr int kMaxRestrictRow = 16;  // restriction rows (P1 nested meshes: 15 on 3D Kuhn lattices)
constexpr int kMaxFinalRow = 16;     // factor and factor-prolongation rows
constexpr int kMaxChainRow = 24;     // restriction-factor product rows

// Restriction of up to kChainSlots chain intermediates:
//   dim 1:  Q_g = R in_g          (R rows n1, cols n1_in; n2 == n2_in)
//   dim 2:  Q_g = in_g R^T        (R rows n2, cols n2_in; n1 == n1_in)
// All arrays are (rows x cols) with the time index innermost ([..][2]).
template <typename T>
struct RestrictArgs {
  int n1 = 0, n2 = 0, n1_in = 0, n2_in = 0;
  int nchains = 0, ch = 0, row = 8;   // ch: rows per thread (0: heuristic)
  int tiled = 0;                      // block order: 0 row-major, 1 column tiles (see kTileW)
  const int* col = nullptr;           // R, ELL
  const Comp<T>* val = nullptr;
  const Store<T>* in[kChainSlots] = {};
  Store<T>* out[kChainSlots] = {};
};

// One chain step producing (n1 x n2) outputs for up to kChainSlots chains,
// with the chains' first factors F_g on one shared pattern:
//  mode A: out_g[k1][k2] = sum_j F_g[k2][j] U[k1][col_j]   (U rows of length nu2)
//                        + sum_q P[k1][q] Q_g[col_q][k2]   (Q rows of length n2)
//  mode B: out_g[k1][k2] = sum_j F_g[k1][j] U[col_j][k2]   (U rows of length n2)
//                        + sum_q P[k2][q] Q_g[k1][col_q]   (Q rows of length nz2)
// The Q part is present when has_prev; P is a prolongation (ELL width 2).
template <typename T>
struct ChainArgs {
  int n1 = 0, n2 = 0, nu2 = 0, nz2 = 0;
  int nchains = 0, has_prev = 0, ch = 0, row = 8;
  int tiled = 0;
  int pair = 0;   // mode A, rows of at most 8: two rows per thread
  int pf = 0;     // L2 prefetch hints for the operands of the chain after next
  const Store<T>* U = nullptr;
  const int* f_col = nullptr;    // ELL
  const Comp<T>* f_val[kChainSlots] = {};
  const int* p_col = nullptr;    // ELL, width 2
  const Comp<T>* p_val = nullptr;
  const Store<T>* Z[kChainSlots] = {};  // the Q inputs
  Store<T>* out[kChainSlots] = {};
  int lat_nx = 0;   // mode A on a 2-D lattice x level (and, with has_prev, a lattice level below)
};

// y (+)= sum_c sum_{t in c} tau_t (x) F_t in_c on one (n1 x n2) grid, all F_t
// on one shared pattern:
//   left:  y[k1][k2] += sum_j F_t[k1][j] in_c[col_j][k2]   (in rows of length n2)
//   right: y[k1][k2] += sum_j F_t[k2][j] in_c[k1][col_j]   (in rows of length nin2)
// The terms of input c are tbeg[c] .. tbeg[c+1]-1.
template <typename T>
struct FinalArgs {
  int n1 = 0, n2 = 0, nin2 = 0, ch = 0, row = 8, accumulate = 0, tiled = 0;
  int pair = 0;   // two outputs per thread: left - columns k2, k2 + 32; right - rows k1, k1 + 1
  int pf = 0;     // L2 prefetch hints for the gathers of an input ahead of its loads
  int nin = 0, nterms = 0;
  const Store<T>* in[kFinalIn] = {};
  int tbeg[kFinalIn + 1] = {};
  const Comp<T>* val[kFinalTerms] = {};   // ELL
  Comp<T> tau[kFinalTerms][4] = {};
  const int* col = nullptr;               // ELL
  Store<T>* y = nullptr;
  int lat_nx = 0;                         // left on a 2-D lattice level: vertices per lattice row
};

// Fused branch-A step on one grid (sweep_fused.cu).  The grid's (k1, k2)
// index set is cut into tiles: an x patch of rows (interior rows first, then
// the rows the dim-1 stencils of the interior reach) times a v patch of
// columns (interior columns first, then the fine columns the restriction rows
// of the coarse columns it owns reach).  Per tile and per group of G chains
// the kernel forms S_b = U V_b^T + P1 Z_b on the whole tile in shared memory,
// folds y += sum_a tau_a X_a S_b into registers on the interior, and writes
// the restricted states Z'_b = S_b R2^T of the owned coarse columns; S_b never
// leaves the SM.
constexpr int kFusedChains = 32;
constexpr int kFusedTerms = 64;
constexpr int kFusedThreads = 512;
constexpr int kFusedOut = 4;   // interior outputs per thread (<= kFusedThreads * kFusedOut per tile)

struct FusedTile {
  int xs0, nxi, nxt, xn0;   // rows: xrows[xs0 ..), interior / total; neighbour table xnbr[xn0 ..)
  int vs0, nvi, nvt;        // columns: vcols[vs0 ..)
  int q0, nq;               // owned coarse columns qcols[q0 ..), their positions qloc[q0 * W ..)
};

template <typename T>
struct FusedArgs {
  const FusedTile* tiles = nullptr;
  const int* xrows = nullptr;
  const int* vcols = nullptr;
  const unsigned short* xnbr = nullptr;   // [interior row][W]: local row of each X pattern entry
  const int* qcols = nullptr;
  const unsigned short* qloc = nullptr;   // [owned coarse column][W]: local column of each R2 entry
  int ntiles = 0, W = 8;
  int n2 = 0, n2c = 0;                    // row lengths of the grid and of the restricted states
  int has_prev = 0, restrict_out = 0;
  int nchains = 0, G = 1;
  const Store<T>* U = nullptr;
  Store<T>* Y = nullptr;
  const int* vcol = nullptr;              // V pattern, ELL (level lv)
  const Comp<T>* vval[kFusedChains] = {};
  const Store<T>* zin[kFusedChains] = {};   // Z_{b,i}: [nx(lx - 1)][n2]
  Store<T>* zout[kFusedChains] = {};        // Z_{b,i+1}: [n1][n2c]
  const int* pcol = nullptr;              // prolongation E_{lx <- lx-1}, ELL width 2
  const Comp<T>* pval = nullptr;
  const int* rcol = nullptr;              // restriction R_{lv-1 <- lv}, ELL width W
  const Comp<T>* rval = nullptr;
  int tbeg[kFusedChains + 1] = {};
  const Comp<T>* xval[kFusedTerms] = {};  // X_a, ELL width W (level lx)
  Comp<T> tau[kFusedTerms][4] = {};
};

template <typename T>
cudaError_t launch_fused_a(const FusedArgs<T>& a, size_t smem, cudaStream_t s);

template <typename T>
cudaError_t launch_restrict(RestrictArgs<T>& a, bool dim2, cudaStream_t s);
template <typename T>
cudaError_t launch_chain(ChainArgs<T>& a, bool mode_a, cudaStream_t s);
template <typename T>
cudaError_t launch_final(FinalArgs<T>& a, bool left, cudaStream_t s);
// left final on a 2-D lattice level (sweep_lattice.cu): rows in stencil-slot
// order, a.row == 7, a.lat_nx = vertices per lattice row, a.ch <= 4: runs of
// 4 vertices per thread, else 8
template <typename T>
cudaError_t launch_final_lattice(FinalArgs<T>& a, cudaStream_t s);
// mode-A chain step on a 2-D lattice x level (sweep_lattice.cu; FP32 and BF16
// storage): a.row == 7, a.lat_nx = vertices per lattice row, a.ch <= 2: runs
// of 2 vertices per thread, else 4
template <typename T>
cudaError_t launch_chain_lattice(ChainArgs<T>& a, cudaStream_t s);

}  // namespace sgdg
