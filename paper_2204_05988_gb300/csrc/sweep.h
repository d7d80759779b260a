// Arguments of the sweep kernels (sweep.cu).
#pragma once

#include <cuda_runtime.h>

namespace sgdg {

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
// [r w, r w + w) of a column and a value array, w = 4 for rows of at most 4
// entries and 8 otherwise (prolongation: w = 2), zero values in the padding.
// `row` (3, 4, 7 or 8) is the longest row; the kernels keep that many entries
// in registers.

// Restriction of up to kChainSlots chain states of the previous grid, the
// first half of a chain step's transfer (restriction before prolongation
// keeps the intermediate on the coarser of the two grids):
//   dim 1:  Z_g = R in_g          (R rows n1, cols n1_in; n2 == n2_in)
//   dim 2:  Z_g = in_g R^T        (R rows n2, cols n2_in; n1 == n1_in)
// All arrays are (rows x cols) with the time index innermost ([..][2]).
template <typename T>
struct RestrictArgs {
  int n1 = 0, n2 = 0, n1_in = 0, n2_in = 0;
  int nchains = 0, ch = 0, row = 8;   // ch: rows per thread (0: heuristic); row: longest R row
  int tiled = 0;                      // block order: 0 row-major, 1 column tiles (see kTileW)
  const int* col = nullptr;           // R, ELL
  const T* val = nullptr;
  const T* in[kChainSlots] = {};
  T* out[kChainSlots] = {};
};

// One chain step on grid i = (n1 x n2) for up to kChainSlots chains:
//  mode A: out = P1 Z + U V_c^T               (Z = prev R2^T, n1_prev x n2)
//  mode B: strict = Z P2^T, out = strict + X_c U   (Z = R1 prev, n1 x n2_prev)
// f_*: the chains' first factor on one shared pattern (A: v level, rows n2;
// B: x level, rows n1); p_*: the prolongation (A: P1 rows n1, B: P2 rows n2).
template <typename T>
struct ChainArgs {
  int n1 = 0, n2 = 0, nz2 = 0;   // nz2: row length of Z (A: n2, B: n2_prev)
  int nchains = 0, has_prev = 0, ch = 0, row = 8;   // row: longest first-factor row
  int tiled = 0;
  const T* U = nullptr;
  const int* f_col = nullptr;    // ELL
  const T* f_val[kChainSlots] = {};
  const int* p_col = nullptr;    // ELL, width 2
  const T* p_val = nullptr;
  const T* Z[kChainSlots] = {};
  T* out[kChainSlots] = {};
  T* strict[kChainSlots] = {};
};

// y (+)= sum_c sum_{t in c} tau_t (x) F_t in_c on one grid: F_t along dim 1
// (left) or dim 2 (right), all F_t on one shared pattern.  The terms of input
// c are tbeg[c] .. tbeg[c+1]-1.
template <typename T>
struct FinalArgs {
  int n1 = 0, n2 = 0, ch = 0, row = 8, accumulate = 0, tiled = 0;
  int nin = 0, nterms = 0;
  const T* in[kFinalIn] = {};
  int tbeg[kFinalIn + 1] = {};
  const T* val[kFinalTerms] = {};   // ELL
  T tau[kFinalTerms][4] = {};
  const int* col = nullptr;         // ELL
  T* y = nullptr;
};

template <typename T>
cudaError_t launch_restrict(RestrictArgs<T>& a, bool dim2, cudaStream_t s);
template <typename T>
cudaError_t launch_chain(ChainArgs<T>& a, bool mode_a, cudaStream_t s);
template <typename T>
cudaError_t launch_final(FinalArgs<T>& a, bool left, cudaStream_t s);

}  // namespace sgdg
