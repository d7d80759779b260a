// Arguments of the sweep kernels (sweep.cu).
#pragma once

#include <cuda_runtime.h>

namespace sgdg {

template <typename T>
constexpr int kChainMax() { return 32; }   // chains per chain-step launch
constexpr int kChainSlots = 32;
constexpr int kFinalTerms = 16;   // terms per final launch
constexpr int kFinalIn = 8;       // chain inputs per final launch

// One chain step on grid i = (n1 x n2) for up to kChainMax chains.
//  mode A: out = T1 (x) T2 prev + U V_c^T      (T1 = E1 rows n1, T2 = R2 rows n2)
//  mode B: strict = T1 (x) T2 prev, out = strict + X_c U   (T1 = R1, T2 = P2)
// f_*: the chains' first factor on one shared pattern (A: v level, rows n2;
// B: x level, rows n1).  prev arrays are (n1_prev x n2_prev), all [..][2].
template <typename T>
struct ChainArgs {
  int n1 = 0, n2 = 0, n1_prev = 0, n2_prev = 0;
  int nchains = 0, has_prev = 0, ch = 0;   // ch: rows per thread (0: heuristic)
  const T* U = nullptr;
  const int* f_rowptr = nullptr;
  const int* f_col = nullptr;
  const T* f_val[kChainSlots] = {};
  const int* t1_rowptr = nullptr;
  const int* t1_col = nullptr;
  const T* t1_val = nullptr;
  const int* t2_rowptr = nullptr;
  const int* t2_col = nullptr;
  const T* t2_val = nullptr;
  const T* prev[kChainSlots] = {};
  T* out[kChainSlots] = {};
  T* strict[kChainSlots] = {};
};

// y (+)= sum_t tau_t (x) F_t in[tin[t]] on one grid: F_t along dim 1 (left)
// or dim 2 (right), all F_t on one shared pattern.
template <typename T>
struct FinalArgs {
  int n1 = 0, n2 = 0, ch = 0, accumulate = 0;   // ch: rows per thread (0: heuristic)
  int nin = 0, nterms = 0;
  const T* in[kFinalIn] = {};
  int tin[kFinalTerms] = {};
  const T* val[kFinalTerms] = {};
  T tau[kFinalTerms][4] = {};
  const int* rowptr = nullptr;
  const int* col = nullptr;
  T* y = nullptr;
};

template <typename T>
cudaError_t launch_chain(ChainArgs<T>& a, bool mode_a, cudaStream_t s);
template <typename T>
cudaError_t launch_final(FinalArgs<T>& a, bool left, cudaStream_t s);

}  // namespace sgdg
