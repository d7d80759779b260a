// The sparse-grid operator apply as a linear-cost sweep over the grids.
//
// Sect. 4.2 applies A = sum_{l,l'} A_{l,l'} block by block.  With the Galerkin
// projection X_{l1,l1'} = E^T X E and nested embeddings (E_{L<-l'} =
// E_{L<-l} E_{l<-l'}), every off-diagonal factor splits into a same-level
// factor and a chain of transfers:
//   l1' <= l1:  X_{l1,l1'} = X_{l1} E_{l1<-l1'},   V_{l2,l2'} = E_{l2'<-l2}^T V_{l2'}
//   l1' >  l1:  X_{l1,l1'} = E_{l1'<-l1}^T X_{l1'}, V_{l2,l2'} = V_{l2} E_{l2<-l2'}
// so that, per term a = (tau, X, V) and grids i = 0..L (grid i = (i, L-i)):
//   branch A:  S_0 = U_0 V_{L}^T,  S_i = P1(R2(S_{i-1})) + U_i V_{L-i}^T,   Y_i += tau X_i S_i
//   branch B:  T'_L = 0, T'_i = R1(P2(T'_{i+1} + X_{i+1} U_{i+1})),        Y_i += tau T'_i V_{L-i}^T
// (P = prolongation E, R = restriction E^T, subscript = the dimension).  This
// reaches the blockwise sum of Sect. 4.2 exactly in exact arithmetic with
// O(#terms * N) work; intermediates never exceed one component grid, like
// the ordering rule of Sect. 4.2.  Terms sharing the factor applied first are
// grouped into one chain; the others are fused in the multi-term kernels.
#include <algorithm>

#include "handle.h"

namespace sgdg {

#define SG_CU(x)                                                              \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) return {SGDG_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

template <typename T>
cudaError_t run_spmm(Handle& h, bool left, SpmmLaunch<T>& a, cudaStream_t s, int kind, double mat_bytes) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h.prof) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  cudaError_t e = left ? launch_left(a, s) : launch_right(a, s);
  h.launches++;
  if (h.prof) {
    cudaEventRecord(e1, s);
    double bytes = mat_bytes;
    for (int g = 0; g < a.ngrids; ++g) {
      double in = 2.0 * sizeof(T) * (double)a.g[g].n1_in * a.g[g].n2_in;
      double out = 2.0 * sizeof(T) * (double)a.g[g].n1_out * a.g[g].n2_out;
      bytes += in * (a.g[g].in2 ? 2 : 1) + out * (a.accumulate ? 2 : 1);
    }
    h.kev.push_back({kind, bytes, e0, e1});
  }
  return e;
}
template cudaError_t run_spmm<double>(Handle&, bool, SpmmLaunch<double>&, cudaStream_t, int, double);
template cudaError_t run_spmm<float>(Handle&, bool, SpmmLaunch<float>&, cudaStream_t, int, double);

namespace {

// bytes of a level's CSR pattern plus nvals value arrays
template <typename T>
double pattern_bytes(const SideDev& sd, int lev, int nvals) {
  return 4.0 * (sd.n[lev] + 1) + (4.0 + nvals * (double)sizeof(T)) * sd.nnz[lev];
}

template <typename T>
void set_terms(Handle& h, SpmmLaunch<T>& a, const std::vector<Term>& terms, const std::vector<int>& idx, int lo,
               int hi, bool x_side, int level_of_grid[], int ngrids) {
  (void)ngrids;
  a.nterms = hi - lo;
  a.identity = 0;
  for (int t = lo; t < hi; ++t) {
    const Term& tm = terms[idx[t]];
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < 2; ++q) a.tau[t - lo][s * 2 + q] = (T)tm.tau[s][q];
  }
  SideDev& sd = x_side ? h.X : h.V;
  for (int g = 0; g < a.ngrids; ++g) {
    int lev = level_of_grid[g];
    a.g[g].rowptr = sd.rowptr[lev];
    a.g[g].col = sd.col[lev];
    for (int t = lo; t < hi; ++t) {
      const Term& tm = terms[idx[t]];
      a.g[g].val[t - lo] = sd.vals<T>().fac[x_side ? tm.x : tm.v][lev];
    }
  }
}

template <typename T>
void set_single(Handle& h, SpmmLaunch<T>& a, int factor, bool x_side, int level_of_grid[]) {
  a.nterms = 1;
  a.identity = 1;
  SideDev& sd = x_side ? h.X : h.V;
  for (int g = 0; g < a.ngrids; ++g) {
    int lev = level_of_grid[g];
    a.g[g].rowptr = sd.rowptr[lev];
    a.g[g].col = sd.col[lev];
    a.g[g].val[0] = sd.vals<T>().fac[factor][lev];
  }
}

// Launch "first" (chain-defining) or "last" (fused multi-term) stage of a chain
// over grids [g0, g1) of the sparse grid; in/out are full sparse-grid vectors.
template <typename T>
Status stage(Handle& h, const std::vector<Term>& terms, const Chain& c, bool first, bool left, const T* in, T* out,
             int g0, int g1, bool accumulate, cudaStream_t s) {
  const bool x_side = left;
  int lev[kMaxGrids];
  SpmmLaunch<T> a;
  a.ngrids = g1 - g0;
  if (a.ngrids <= 0) return {};
  for (int g = g0; g < g1; ++g) {
    SpmmGrid<T>& G = a.g[g - g0];
    G.in = in + h.off[g];
    G.in2 = nullptr;
    G.out = out + h.off[g];
    G.n1_in = G.n1_out = h.n1[g];
    G.n2_in = G.n2_out = h.n2[g];
    lev[g - g0] = x_side ? g : h.L - g;
  }
  // the single-factor stage applies c.first with tau = I; the other stage
  // applies every term's own factor with its tau
  const bool single = (first == true);
  const SideDev& sd = x_side ? h.X : h.V;
  const int kind = left ? KIND_LEFT : KIND_RIGHT;
  if (single) {
    set_single(h, a, c.first, x_side, lev);
    a.accumulate = accumulate;
    double mb = 0.0;
    for (int g = 0; g < a.ngrids; ++g) mb += pattern_bytes<T>(sd, lev[g], 1);
    SG_CU(run_spmm(h, left, a, s, kind, mb));
    return {};
  }
  const int nt = (int)c.terms.size();
  for (int t0 = 0; t0 < nt; t0 += kMaxTerms) {
    int t1 = std::min(nt, t0 + kMaxTerms);
    set_terms(h, a, terms, c.terms, t0, t1, x_side, lev, a.ngrids);
    a.accumulate = (t0 > 0) ? 1 : accumulate;
    double mb = 0.0;
    for (int g = 0; g < a.ngrids; ++g) mb += pattern_bytes<T>(sd, lev[g], t1 - t0);
    SG_CU(run_spmm(h, left, a, s, kind, mb));
  }
  return {};
}

// One transfer: out = Op(in [+ in2]) on a single (n1 x n2) array.
template <typename T>
Status transfer(Handle& h, bool left, const int* rowptr, const int* col, const T* val, int nrows, int nnz,
                const T* in, const T* in2, T* out, int n1_in, int n2_in, int n1_out, int n2_out, bool accumulate,
                T scale, cudaStream_t s) {
  SpmmLaunch<T> a;
  a.ngrids = 1;
  a.nterms = 1;
  a.identity = scale == (T)1 ? 1 : 0;
  a.tau[0][0] = scale; a.tau[0][1] = 0; a.tau[0][2] = 0; a.tau[0][3] = scale;
  a.accumulate = accumulate;
  SpmmGrid<T>& G = a.g[0];
  G.in = in; G.in2 = in2; G.out = out;
  G.n1_in = n1_in; G.n2_in = n2_in; G.n1_out = n1_out; G.n2_out = n2_out;
  G.rowptr = rowptr; G.col = col; G.val[0] = val;
  const double mb = 4.0 * (nrows + 1) + (4.0 + sizeof(T)) * (double)nnz;
  SG_CU(run_spmm(h, left, a, s, left ? KIND_XFER_LEFT : KIND_XFER_RIGHT, mb));
  return {};
}

template <typename T>
Handle::Bufs& bufs(Handle& h);
template <> Handle::Bufs& bufs<double>(Handle& h) { return h.b64; }
template <> Handle::Bufs& bufs<float>(Handle& h) { return h.b32; }

template <typename T>
Status ensure_bufs(Handle& h) {
  Handle::Bufs& b = bufs<T>(h);
  if (b.S) return {};
  size_t full = sizeof(T) * (size_t)h.n_coeffs;
  size_t tmp = sizeof(T) * (size_t)h.tmp_elems;
  if (dev_alloc(h, &b.S, full) != cudaSuccess || dev_alloc(h, &b.Z, full) != cudaSuccess ||
      dev_alloc(h, &b.TP, full) != cudaSuccess || dev_alloc(h, &b.tmp, tmp) != cudaSuccess ||
      dev_alloc(h, &b.W, full) != cudaSuccess)
    return {SGDG_ENOMEM, "sweep buffers"};
  return {};
}

}  // namespace

template <typename T>
Status apply_plan(Handle& h, const Plan& p, const T* u, T* y, cudaStream_t s) {
  Status st = ensure_bufs<T>(h);
  if (st.code) return st;
  Handle::Bufs& b = bufs<T>(h);
  T* S = (T*)b.S;
  T* Z = (T*)b.Z;
  T* TP = (T*)b.TP;
  T* tmp = (T*)b.tmp;
  const int L = h.L;
  SG_CU(vec_fill<T>(y, h.n_coeffs, (T)0, s));
  // ---- branch A: sources with l1' <= l1 (diagonal included)
  for (const Chain& c : p.A) {
    // first factor: right (V) if by_v, else the fused multi-term right stage
    if (c.by_v) st = stage<T>(h, p.terms, c, true, false, u, S, 0, L + 1, false, s);
    else st = stage<T>(h, p.terms, c, false, false, u, S, 0, L + 1, false, s);
    if (st.code) return st;
    for (int i = 1; i <= L; ++i) {
      // tmp = R2(S_{i-1}): restrict dim 2 from v-level L-i+1 to L-i
      const int lv = L - i;
      st = transfer<T>(h, false, h.V.R_rowptr[lv], h.V.R_col[lv], h.V.vals<T>().R[lv], h.V.n[lv], h.V.R_nnz[lv],
                       S + h.off[i - 1], nullptr, tmp,
                       h.n1[i - 1], h.n2[i - 1], h.n1[i - 1], h.V.n[lv], false, (T)1, s);
      if (st.code) return st;
      // S_i += P1(tmp): prolong dim 1 from x-level i-1 to i
      st = transfer<T>(h, true, h.X.E_rowptr[i - 1], h.X.E_col[i - 1], h.X.vals<T>().E[i - 1], h.X.n[i],
                       h.X.E_nnz[i - 1], tmp, nullptr,
                       S + h.off[i], h.n1[i - 1], h.V.n[lv], h.n1[i], h.n2[i], true, (T)1, s);
      if (st.code) return st;
    }
    if (c.by_v) st = stage<T>(h, p.terms, c, false, true, S, y, 0, L + 1, true, s);
    else st = stage<T>(h, p.terms, c, true, true, S, y, 0, L + 1, true, s);
    if (st.code) return st;
  }
  // ---- branch B: sources with l1' > l1
  if (L >= 1) {
    for (const Chain& c : p.B) {
      if (c.by_v) st = stage<T>(h, p.terms, c, false, true, u, Z, 1, L + 1, false, s);
      else st = stage<T>(h, p.terms, c, true, true, u, Z, 1, L + 1, false, s);
      if (st.code) return st;
      for (int i = L - 1; i >= 0; --i) {
        // tmp = P2(Z_{i+1} + T'_{i+1}): prolong dim 2 from v-level L-i-1 to L-i
        const int lvc = L - i - 1;
        st = transfer<T>(h, false, h.V.E_rowptr[lvc], h.V.E_col[lvc], h.V.vals<T>().E[lvc], h.V.n[lvc + 1],
                         h.V.E_nnz[lvc], Z + h.off[i + 1],
                         (i + 1 < L) ? TP + h.off[i + 1] : nullptr, tmp, h.n1[i + 1], h.n2[i + 1], h.n1[i + 1],
                         h.V.n[L - i], false, (T)1, s);
        if (st.code) return st;
        // T'_i = R1(tmp): restrict dim 1 from x-level i+1 to i
        st = transfer<T>(h, true, h.X.R_rowptr[i], h.X.R_col[i], h.X.vals<T>().R[i], h.X.n[i], h.X.R_nnz[i], tmp,
                         nullptr, TP + h.off[i],
                         h.n1[i + 1], h.V.n[L - i], h.n1[i], h.n2[i], false, (T)1, s);
        if (st.code) return st;
      }
      if (c.by_v) st = stage<T>(h, p.terms, c, true, false, TP, y, 0, L, true, s);
      else st = stage<T>(h, p.terms, c, false, false, TP, y, 0, L, true, s);
      if (st.code) return st;
    }
  }
  return {};
}

template Status apply_plan<double>(Handle&, const Plan&, const double*, double*, cudaStream_t);
template Status apply_plan<float>(Handle&, const Plan&, const float*, float*, cudaStream_t);

// Diagonal blocks A_{l,l} on a list of grids (l1[g], l2[g]) at once: the
// component systems of the combination-technique preconditioner.
template <typename T>
Status apply_diag_grids(Handle& h, int ng, const int* l1, const int* l2, const T* const* u, T* const* y,
                        cudaStream_t s) {
  Status st = ensure_bufs<T>(h);
  if (st.code) return st;
  if (ng > kMaxGrids) return {SGDG_EINVAL, "too many grids in one diagonal apply"};
  T* W = (T*)bufs<T>(h).W;
  std::vector<long long> woff(ng + 1, 0);
  for (int g = 0; g < ng; ++g) woff[g + 1] = woff[g] + 2LL * h.X.n[l1[g]] * h.V.n[l2[g]];
  if (woff[ng] > h.n_coeffs) return {SGDG_EINVAL, "diagonal apply workspace too small"};
  for (size_t ci = 0; ci < h.op.D.size(); ++ci) {
    const Chain& c = h.op.D[ci];
    // stage 1 into W (right, V side), stage 2 into y (left, X side)
    for (int pass = 0; pass < 2; ++pass) {
      const bool left = (pass == 1);
      const bool single = c.by_v ? (pass == 0) : (pass == 1);
      int lev[kMaxGrids];
      SpmmLaunch<T> a;
      a.ngrids = ng;
      for (int g = 0; g < ng; ++g) {
        SpmmGrid<T>& G = a.g[g];
        G.in = pass == 0 ? u[g] : W + woff[g];
        G.in2 = nullptr;
        G.out = pass == 0 ? W + woff[g] : y[g];
        G.n1_in = G.n1_out = h.X.n[l1[g]];
        G.n2_in = G.n2_out = h.V.n[l2[g]];
        lev[g] = left ? l1[g] : l2[g];
      }
      const SideDev& sd = left ? h.X : h.V;
      const int kind = left ? KIND_LEFT : KIND_RIGHT;
      if (single) {
        set_single(h, a, c.first, left, lev);
        a.accumulate = pass == 1 ? (ci > 0) : 0;
        double mb = 0.0;
        for (int g = 0; g < ng; ++g) mb += pattern_bytes<T>(sd, lev[g], 1);
        SG_CU(run_spmm(h, left, a, s, kind, mb));
      } else {
        const int nt = (int)c.terms.size();
        for (int t0 = 0; t0 < nt; t0 += kMaxTerms) {
          int t1 = std::min(nt, t0 + kMaxTerms);
          set_terms(h, a, h.op.terms, c.terms, t0, t1, left, lev, ng);
          a.accumulate = (t0 > 0) ? 1 : (pass == 1 ? (ci > 0) : 0);
          double mb = 0.0;
          for (int g = 0; g < ng; ++g) mb += pattern_bytes<T>(sd, lev[g], t1 - t0);
          SG_CU(run_spmm(h, left, a, s, kind, mb));
        }
      }
    }
  }
  return {};
}

template Status apply_diag_grids<double>(Handle&, int, const int*, const int*, const double* const*,
                                         double* const*, cudaStream_t);
template Status apply_diag_grids<float>(Handle&, int, const int*, const int*, const float* const*, float* const*,
                                        cudaStream_t);

// Values of a spatial sparse-grid function at the nodes of every grid:
//   out_i = sum_{j<=i} P1 I2 u_j + sum_{j>i} I1 P2 u_j  (P: prolongation, I: injection)
// by the same two chains as the operator sweep.
Status nodal_eval(Handle& h, const double* u, double* out, cudaStream_t s) {
  Status st = ensure_bufs<double>(h);
  if (st.code) return st;
  double* A = (double*)h.b64.S;     // chain A (spatial layout, uses soff)
  double* B = (double*)h.b64.TP;
  double* tmp = (double*)h.b64.tmp;
  const int L = h.L;
  SG_CU(cudaMemcpyAsync(A, u, sizeof(double) * h.n_spatial, cudaMemcpyDeviceToDevice, s));
  for (int i = 1; i <= L; ++i) {
    const int lv = L - i;   // inject dim 2 from v-level lv+1 to lv, then prolong dim 1
    SG_CU(inject_dim(A + h.soff[i - 1], tmp, h.n1[i - 1], h.V.n[lv], h.n2[i - 1], h.V.inj[lv], 2, 0, s));
    SG_CU(spmm1(tmp, A + h.soff[i], h.n1[i - 1], h.V.n[lv], h.n1[i], h.n2[i], h.X.E_rowptr[i - 1],
                h.X.E_col[i - 1], h.X.v64.E[i - 1], 1, 1, s));
  }
  SG_CU(cudaMemcpyAsync(out, A, sizeof(double) * h.n_spatial, cudaMemcpyDeviceToDevice, s));
  if (L >= 1) {
    // B_L = u_L; B_i (strict part) = I1(P2(u_{i+1} + B_{i+1}))
    SG_CU(cudaMemcpyAsync(B + h.soff[L], u + h.soff[L], sizeof(double) * h.n1[L] * h.n2[L],
                          cudaMemcpyDeviceToDevice, s));
    for (int i = L - 1; i >= 0; --i) {
      const int lvc = L - i - 1;
      SG_CU(spmm1(B + h.soff[i + 1], tmp, h.n1[i + 1], h.n2[i + 1], h.n1[i + 1], h.V.n[L - i], h.V.E_rowptr[lvc],
                  h.V.E_col[lvc], h.V.v64.E[lvc], 2, 0, s));
      SG_CU(inject_dim(tmp, B + h.soff[i], h.n1[i], h.n2[i], h.V.n[L - i], h.X.inj[i], 1, 0, s));
      SG_CU(vec_axpby<double>((long long)h.n1[i] * h.n2[i], 1.0, B + h.soff[i], 1.0, out + h.soff[i], s));
      SG_CU(vec_axpby<double>((long long)h.n1[i] * h.n2[i], 1.0, u + h.soff[i], 1.0, B + h.soff[i], s));
    }
  }
  return {};
}

}  // namespace sgdg
