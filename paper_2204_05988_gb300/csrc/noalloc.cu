// Diagonal-block apply A_{l,l} u that allocates nothing (sgdg_apply_diag_noalloc).
//
// The regular sgdg_apply_diag keeps its intermediate products u V_b^T in a
// pool the handle allocates on first use.  Some callers cannot allow an
// allocation at that point: latency-critical loops that must never hit the
// allocator's device-wide synchronisation, and hosts (plugins, embedded
// solvers) whose device memory is handed in full to a pool that another
// component owns, so that cudaMalloc would fail or steal from it.  This
// variant takes its scratch from the file-scope array below instead; the
// caller still passes the input u and the output y.
//
// The array lives for the lifetime of the loaded library on every GPU that
// loads it (SGDG_NOALLOC_SCRATCH_BYTES each).  All calls share it and it keeps
// the last call's contents: calls whose work overlaps on the GPU (different
// streams, or different host threads on the same device) race on it.  Every
// scratch element is written before it is read, so nothing needs clearing.
#include <cuda_runtime.h>

#include "handle.h"
#include "sweep.h"

namespace sgdg {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SGDG_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch on the current device (host code only
// holds a stand-in for the array, not its address).  It is looked up on every
// call: cudaGetSymbolAddress is a cheap host query, and a cached address
// would go stale when the device is reset (cudaDeviceReset reloads the
// module).  The first call on a device also loads the module there, so make
// it before any stream capture.
Status scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return {SGDG_ECUDA, std::string("no-alloc apply: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e)};
  *out = p;
  return {};
}

template <typename T>
Status diag_noalloc(Handle& h, int l1, int l2, const T* u, T* y, cudaStream_t s) {
  const std::vector<Chain>& chains = h.op.A;   // one chain per distinct v factor
  const int nc = (int)chains.size();
  const int n1 = h.X.n[l1], n2 = h.V.n[l2];
  const long long M = 2LL * n1 * n2;
  const double need = (double)nc * (double)M * sizeof(T);
  if (need > (double)SGDG_NOALLOC_SCRATCH_BYTES)
    return {SGDG_EINVAL, "no-alloc apply: grid (" + std::to_string(l1) + "," + std::to_string(l2) + ") needs " +
                             std::to_string((long long)need) + " scratch bytes, the limit is " +
                             std::to_string((long long)SGDG_NOALLOC_SCRATCH_BYTES)};
  void* base = nullptr;
  Status st = scratch_address(&base);
  if (st.code) return st;
  T* W = (T*)base;
  // W_b = u V_b^T for every distinct v factor
  for (int c0 = 0; c0 < nc; c0 += kChainSlots) {
    ChainArgs<T> a;
    a.n1 = n1;
    a.n2 = n2;
    a.nchains = std::min(kChainSlots, nc - c0);
    a.nu2 = n2;
    a.row = h.V.row_regs();
    a.U = u;
    a.f_col = h.V.ell_col[l2];
    for (int c = 0; c < a.nchains; ++c) {
      a.f_val[c] = h.V.vals<T>().ell_fac[chains[c0 + c].first][l2];
      a.out[c] = W + (size_t)(c0 + c) * M;
    }
    cudaError_t e = launch_chain(a, true, s);
    if (e != cudaSuccess) return {SGDG_ECUDA, std::string("no-alloc apply: ") + cudaGetErrorString(e)};
  }
  // y = sum_a tau_a X_a W_{b(a)}, folded in launches of up to kFinalIn inputs
  // and kFinalTerms terms
  FinalArgs<T> f;
  f.n1 = n1;
  f.n2 = n2;
  f.row = h.X.row_regs();
  f.col = h.X.ell_col[l1];
  f.y = y;
  bool first = true;
  auto flush = [&]() -> Status {
    if (f.nterms == 0) return {};
    f.tbeg[f.nin] = f.nterms;
    f.accumulate = first ? 0 : 1;
    f.ch = 0;
    cudaError_t e = launch_final(f, true, s);
    if (e != cudaSuccess) return {SGDG_ECUDA, std::string("no-alloc apply: ") + cudaGetErrorString(e)};
    first = false;
    f.nin = 0;
    f.nterms = 0;
    return {};
  };
  for (int c = 0; c < nc; ++c) {
    bool open = false;
    for (int t : chains[c].terms) {
      if (!open || f.nterms == kFinalTerms) {
        if (f.nin == kFinalIn || f.nterms == kFinalTerms) {
          st = flush();
          if (st.code) return st;
        }
        f.tbeg[f.nin] = f.nterms;
        f.in[f.nin++] = W + (size_t)c * M;
        open = true;
      }
      const Term& tm = h.op.terms[t];
      f.val[f.nterms] = h.X.vals<T>().ell_fac[tm.x][l1];
      for (int a = 0; a < 2; ++a)
        for (int q = 0; q < 2; ++q) f.tau[f.nterms][a * 2 + q] = (T)tm.tau[a][q];
      f.nterms++;
    }
  }
  return flush();
}

}  // namespace

}  // namespace sgdg

using namespace sgdg;

extern "C" sgdg_status sgdg_apply_diag_noalloc(void* hp, int l1, int l2, const void* u, void* y, int prec,
                                               void* stream) {
  if (!hp) return SGDG_EINVAL;
  Handle* h = (Handle*)hp;
  if (!u || !y) {
    h->err = "no-alloc apply: null input or output";
    return SGDG_EINVAL;
  }
  if (l1 < 0 || l2 < 0 || l1 > h->L || l2 > h->L || (l1 + l2 != h->L && l1 + l2 != h->L - 1)) {
    h->err = "no-alloc apply: grid levels must satisfy l1 + l2 in {L-1, L}";
    return SGDG_EINVAL;
  }
  Status st;
  if (prec == SGDG_FP64) st = diag_noalloc<double>(*h, l1, l2, (const double*)u, (double*)y, (cudaStream_t)stream);
  else if (prec == SGDG_MIXED_FP32)
    st = diag_noalloc<float>(*h, l1, l2, (const float*)u, (float*)y, (cudaStream_t)stream);
  else st = {SGDG_EINVAL, "no-alloc apply: unknown precision"};
  if (st.code) h->err = st.msg;
  return st.code;
}
