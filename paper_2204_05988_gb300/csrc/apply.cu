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
#include "sweep.h"

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
    h.kev.push_back({kind, bytes, e0, e1, -1});
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

// Chain-state pool of the sweep: 2 ring slots per branch-A chain, 2 ring
// slots + 1 strict slot per branch-B chain, then the restriction
// intermediates Z of one launch group; each slot holds one largest grid.
inline long long pool_slots(const Plan& q) {
  const long long a = (long long)q.A.size(), b = (long long)q.B.size();
  return std::max(2 * a, 3 * b) + std::min<long long>(kChainSlots, std::max(a, b));
}

template <typename T>
Status ensure_pool(Handle& h, const Plan& p, T** pool, long long* slot, T** zbase) {
  long long M = 2;
  for (int l = 0; l <= h.L; ++l) M = std::max(M, 2LL * h.n1[l] * h.n2[l]);
  // sized once for the largest plan of the handle (the operator's)
  const long long need = M * std::max(pool_slots(h.op), pool_slots(p));
  Handle::Bufs& b = bufs<T>(h);
  if (!b.pool) {
    if (dev_alloc(h, &b.pool, sizeof(T) * (size_t)need) != cudaSuccess) return {SGDG_ENOMEM, "sweep chain pool"};
    b.pool_elems = need;
  }
  if (b.pool_elems < M * pool_slots(p)) return {SGDG_EINVAL, "sweep chain pool too small for this plan"};
  *pool = (T*)b.pool;
  *slot = M;
  *zbase = (T*)b.pool + (size_t)M * std::max(2LL * (long long)p.A.size(), 3LL * (long long)p.B.size());
  return {};
}

template <typename T>
double csr_bytes(int rows, int nnz, int nvals) {
  return 4.0 * (rows + 1) + (4.0 + (double)nvals * sizeof(T)) * nnz;
}

// launch site: kind (< 16), chains or terms (< 64), element size, grid shape (< 2^24 each)
inline long long site_key(int kind, int n1, int n2, int count, int elem) {
  const long long head = ((long long)kind * 64 + count) * 16 + elem;
  return (((head << 24) | (long long)n1) << 24) | (long long)n2;
}

// Launch shape of a site: rows per thread (ch, 0 = heuristic) and block order
// (tiled).  Tuned choices are stored as ch | tiled << 4.  Untuned sites take
// the column tiles when the launch's stencil runs along dim 1 and rows are
// long enough to fill a tile.
struct Shape {
  int ch = 0, tiled = 0;
};

template <typename T>
Shape pick_shape(Handle& h, long long site, bool dim1_stencil, int n1, int n2) {
  int code = h.force_ch > 0 ? h.force_ch : 0;
  if (!code) {
    auto it = h.tuned_ch.find(site);
    if (it != h.tuned_ch.end()) code = it->second;
  }
  Shape sh;
  if (code) {
    sh.ch = std::min(code & 15, n1);
    sh.tiled = code >> 4;
  } else {
    sh.tiled = dim1_stencil && n2 >= kTileW ? 1 : 0;
  }
  return sh;
}

struct ProfScope {
  Handle& h;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ProfScope(Handle& hh, cudaStream_t ss) : h(hh), s(ss) {
    if (h.prof) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, s);
    }
  }
  void done(int kind, double bytes, long long site) {
    h.launches++;
    if (!h.prof) return;
    cudaEventRecord(e1, s);
    h.kev.push_back({kind, bytes, e0, e1, site});
  }
};

template <typename T>
double grid_bytes(long long n1, long long n2) {
  return 2.0 * sizeof(T) * (double)n1 * (double)n2;
}

template <typename T>
Status run_restrict(Handle& h, RestrictArgs<T>& a, bool dim2, cudaStream_t s, double mat_bytes) {
  const int kind = dim2 ? KIND_XFER_RIGHT : KIND_XFER_LEFT;
  const long long site = site_key(kind, a.n1, a.n2, a.nchains, sizeof(T));
  const Shape sh = pick_shape<T>(h, site, !dim2, a.n1, a.n2);
  a.ch = sh.ch;
  a.tiled = sh.tiled;
  ProfScope ps(h, s);
  SG_CU(launch_restrict(a, dim2, s));
  ps.done(kind, mat_bytes + a.nchains * (grid_bytes<T>(a.n1_in, a.n2_in) + grid_bytes<T>(a.n1, a.n2)), site);
  return {};
}

// extra_bytes: matrices and the restriction intermediates the launch reads
template <typename T>
Status run_chain(Handle& h, ChainArgs<T>& a, bool mode_a, cudaStream_t s, double extra_bytes) {
  const int kind = mode_a ? KIND_CHAIN_A : KIND_CHAIN_B;
  const long long site = site_key(kind, a.n1, a.n2, a.nchains, sizeof(T));
  const Shape sh = pick_shape<T>(h, site, mode_a, a.n1, a.n2);
  a.ch = sh.ch;
  a.tiled = sh.tiled;
  ProfScope ps(h, s);
  SG_CU(launch_chain(a, mode_a, s));
  const double g = grid_bytes<T>(a.n1, a.n2);
  ps.done(kind, extra_bytes + g + a.nchains * g * (!mode_a && a.has_prev ? 2.0 : 1.0), site);
  return {};
}

template <typename T>
Status run_final(Handle& h, FinalArgs<T>& f, bool left, int lev_rows, int lev_nnz, cudaStream_t s) {
  const int kind = left ? KIND_FINAL_LEFT : KIND_FINAL_RIGHT;
  const long long site = site_key(kind, f.n1, f.n2, f.nin, sizeof(T));
  const Shape sh = pick_shape<T>(h, site, left, f.n1, f.n2);
  f.ch = sh.ch;
  f.tiled = sh.tiled;
  ProfScope ps(h, s);
  SG_CU(launch_final(f, left, s));
  const double g = grid_bytes<T>(f.n1, f.n2);
  ps.done(kind, csr_bytes<T>(lev_rows, lev_nnz, f.nterms) + f.nin * g + g * (f.accumulate ? 2.0 : 1.0), site);
  return {};
}

// y_i (+)= sum over the chains' terms of tau_a F_a in_c on grid i (F on the
// x pattern at level i when left, on the v pattern at level L-i otherwise).
template <typename T, typename InOf>
Status finals_on(Handle& h, const Plan& p, const std::vector<Chain>& chains, bool left, int n1, int n2, int lev,
                 InOf in_of, bool accumulate_first, T* ygrid, cudaStream_t s) {
  const SideDev& sd = left ? h.X : h.V;
  FinalArgs<T> f;
  f.n1 = n1;
  f.n2 = n2;
  f.row = sd.row_regs();
  f.col = sd.ell_col[lev];
  f.y = ygrid;
  bool first = true;
  auto flush = [&]() -> Status {
    if (f.nterms == 0) return {};
    f.tbeg[f.nin] = f.nterms;
    f.accumulate = first ? (accumulate_first ? 1 : 0) : 1;
    Status st = run_final(h, f, left, sd.n[lev], sd.nnz[lev], s);
    first = false;
    f.nin = 0;
    f.nterms = 0;
    return st;
  };
  for (size_t c = 0; c < chains.size(); ++c) {
    const Chain& ch = chains[c];
    bool open = false;
    for (int t : ch.terms) {
      if (!open || f.nterms == kFinalTerms) {
        if (f.nin == kFinalIn || f.nterms == kFinalTerms) {
          Status st = flush();
          if (st.code) return st;
        }
        f.tbeg[f.nin] = f.nterms;
        f.in[f.nin++] = in_of((int)c);
        open = true;
      }
      const Term& tm = p.terms[t];
      f.val[f.nterms] = sd.vals<T>().ell_fac[left ? tm.x : tm.v][lev];
      for (int a = 0; a < 2; ++a)
        for (int q = 0; q < 2; ++q) f.tau[f.nterms][a * 2 + q] = (T)tm.tau[a][q];
      f.nterms++;
    }
  }
  return flush();
}

template <typename T, typename InOf>
Status finals(Handle& h, const Plan& p, const std::vector<Chain>& chains, bool left, int i, InOf in_of,
              bool accumulate_first, T* y, cudaStream_t s) {
  return finals_on<T>(h, p, chains, left, h.n1[i], h.n2[i], left ? i : h.L - i, in_of, accumulate_first,
                      y + h.off[i], s);
}

}  // namespace

template <typename T>
Status apply_plan(Handle& h, const Plan& p, const T* u, T* y, cudaStream_t s) {
  T* pool;
  T* zb;
  long long M;
  Status st = ensure_pool<T>(h, p, &pool, &M, &zb);
  if (st.code) return st;
  const int L = h.L;
  const int G = kChainMax<T>();
  const int nA = (int)p.A.size(), nB = (int)p.B.size();
  auto slotA = [&](int c, int par) { return pool + (size_t)(2 * c + par) * M; };
  auto slotT = [&](int c, int par) { return pool + (size_t)(3 * c + par) * M; };
  auto slotTP = [&](int c) { return pool + (size_t)(3 * c + 2) * M; };
  auto slotZ = [&](int g) { return zb + (size_t)g * M; };
  // ---- branch A (sources l1' <= l1): chains by the v factor
  for (int i = 0; i <= L; ++i) {
    const int lv = L - i;
    for (int c0 = 0; c0 < nA; c0 += G) {
      const int nc = std::min(G, nA - c0);
      double zbytes = 0.0;
      if (i > 0) {
        // Z_g = S_{g,i-1} R2^T  (n1[i-1] x n2[i])
        RestrictArgs<T> r;
        r.n1 = h.n1[i - 1];
        r.n2 = h.n2[i];
        r.n1_in = h.n1[i - 1];
        r.n2_in = h.n2[i - 1];
        r.nchains = nc;
        r.row = h.V.row_regs();
        r.col = h.V.R_ell_col[lv];
        r.val = h.V.vals<T>().ell_R[lv];
        for (int g = 0; g < nc; ++g) {
          r.in[g] = slotA(c0 + g, (i - 1) & 1);
          r.out[g] = slotZ(g);
        }
        st = run_restrict(h, r, true, s, csr_bytes<T>(h.V.n[lv], h.V.R_nnz[lv], 1));
        if (st.code) return st;
        zbytes = nc * grid_bytes<T>(r.n1, r.n2) + csr_bytes<T>(h.X.n[i], h.X.E_nnz[i - 1], 1);
      }
      ChainArgs<T> a;
      a.n1 = h.n1[i];
      a.n2 = h.n2[i];
      a.nz2 = h.n2[i];
      a.nchains = nc;
      a.has_prev = i > 0;
      a.row = h.V.row_regs();
      a.U = u + h.off[i];
      a.f_col = h.V.ell_col[lv];
      for (int g = 0; g < nc; ++g) {
        a.f_val[g] = h.V.vals<T>().ell_fac[p.A[c0 + g].first][lv];
        a.out[g] = slotA(c0 + g, i & 1);
        a.Z[g] = i > 0 ? slotZ(g) : nullptr;
      }
      if (i > 0) {
        a.p_col = h.X.E_ell_col[i - 1];
        a.p_val = h.X.vals<T>().ell_E[i - 1];
      }
      st = run_chain(h, a, true, s, csr_bytes<T>(h.V.n[lv], h.V.nnz[lv], nc) + zbytes);
      if (st.code) return st;
    }
    st = finals<T>(h, p, p.A, true, i, [&](int c) { return (const T*)slotA(c, i & 1); }, false, y, s);
    if (st.code) return st;
  }
  // ---- branch B (sources l1' > l1): chains by the x factor
  if (L >= 1) {
    for (int i = L; i >= 0; --i) {
      for (int c0 = 0; c0 < nB; c0 += G) {
        const int nc = std::min(G, nB - c0);
        double zbytes = 0.0;
        if (i < L) {
          // Z_g = R1 T_{g,i+1}  (n1[i] x n2[i+1])
          RestrictArgs<T> r;
          r.n1 = h.n1[i];
          r.n2 = h.n2[i + 1];
          r.n1_in = h.n1[i + 1];
          r.n2_in = h.n2[i + 1];
          r.nchains = nc;
          r.row = h.X.row_regs();
          r.col = h.X.R_ell_col[i];
          r.val = h.X.vals<T>().ell_R[i];
          for (int g = 0; g < nc; ++g) {
            r.in[g] = slotT(c0 + g, (i + 1) & 1);
            r.out[g] = slotZ(g);
          }
          st = run_restrict(h, r, false, s, csr_bytes<T>(h.X.n[i], h.X.R_nnz[i], 1));
          if (st.code) return st;
          zbytes = nc * grid_bytes<T>(r.n1, r.n2) + csr_bytes<T>(h.V.n[L - i], h.V.E_nnz[L - i - 1], 1);
        }
        ChainArgs<T> a;
        a.n1 = h.n1[i];
        a.n2 = h.n2[i];
        a.nz2 = i < L ? h.n2[i + 1] : 0;
        a.nchains = nc;
        a.has_prev = i < L;
        a.row = h.X.row_regs();
        a.U = u + h.off[i];
        a.f_col = h.X.ell_col[i];
        for (int g = 0; g < nc; ++g) {
          a.f_val[g] = h.X.vals<T>().ell_fac[p.B[c0 + g].first][i];
          a.out[g] = slotT(c0 + g, i & 1);
          a.Z[g] = i < L ? slotZ(g) : nullptr;
          a.strict[g] = i < L ? slotTP(c0 + g) : nullptr;
        }
        if (i < L) {
          a.p_col = h.V.E_ell_col[L - i - 1];
          a.p_val = h.V.vals<T>().ell_E[L - i - 1];
        }
        st = run_chain(h, a, false, s, csr_bytes<T>(h.X.n[i], h.X.nnz[i], nc) + zbytes);
        if (st.code) return st;
      }
      if (i < L) {
        st = finals<T>(h, p, p.B, false, i, [&](int c) { return (const T*)slotTP(c); }, true, y, s);
        if (st.code) return st;
      }
    }
  }
  return {};
}

template Status apply_plan<double>(Handle&, const Plan&, const double*, double*, cudaStream_t);
template Status apply_plan<float>(Handle&, const Plan&, const float*, float*, cudaStream_t);

// Diagonal blocks A_{l,l} on a list of grids (l1[g], l2[g]): the component
// systems of the combination-technique preconditioner.  Per grid: one launch
// forms W_b = u V_b^T for every distinct v factor (the chain-step kernel
// without a transfer), then fused final launches fold all terms into y.
template <typename T>
Status apply_diag_grids(Handle& h, int ng, const int* l1, const int* l2, const T* const* u, T* const* y,
                        cudaStream_t s) {
  T* pool;
  T* zb;
  long long M;
  Status st = ensure_pool<T>(h, h.op, &pool, &M, &zb);
  if (st.code) return st;
  const std::vector<Chain>& chains = h.op.A;   // by v factor
  const int nc = (int)chains.size();
  for (int g = 0; g < ng; ++g) {
    const int n1 = h.X.n[l1[g]], n2 = h.V.n[l2[g]];
    if (2LL * n1 * n2 > M) return {SGDG_EINVAL, "diagonal apply grid larger than the sweep slots"};
    for (int c0 = 0; c0 < nc; c0 += kChainSlots) {
      ChainArgs<T> a;
      a.n1 = n1;
      a.n2 = n2;
      a.nchains = std::min(kChainSlots, nc - c0);
      a.has_prev = 0;
      a.row = h.V.row_regs();
      a.U = u[g];
      a.f_col = h.V.ell_col[l2[g]];
      for (int c = 0; c < a.nchains; ++c) {
        a.f_val[c] = h.V.vals<T>().ell_fac[chains[c0 + c].first][l2[g]];
        a.out[c] = pool + (size_t)(c0 + c) * M;
      }
      st = run_chain(h, a, true, s, csr_bytes<T>(n2, h.V.nnz[l2[g]], a.nchains));
      if (st.code) return st;
    }
    st = finals_on<T>(h, h.op, chains, true, n1, n2, l1[g], [&](int c) { return (const T*)(pool + (size_t)c * M); },
                      false, y[g], s);
    if (st.code) return st;
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

template <typename T>
Status autotune(Handle& h, const T* u, T* y, cudaStream_t s) {
  // rows per thread x block order, encoded as ch | tiled << 4
  const int cand[] = {1, 2, 4, 8, 1 | 16, 2 | 16, 4 | 16, 8 | 16};
  std::map<long long, std::pair<float, int>> best;
  const bool prof_was = h.prof;
  for (int c : cand) {
    h.force_ch = c;
    for (auto& k : h.kev) { cudaEventDestroy(k.e0); cudaEventDestroy(k.e1); }
    h.kev.clear();
    h.prof = true;
    Status st = apply_plan<T>(h, h.op, u, y, s);
    h.prof = false;
    if (st.code) { h.force_ch = 0; h.prof = prof_was; return st; }
    SG_CU(cudaStreamSynchronize(s));
    std::map<long long, float> tot;
    for (auto& k : h.kev) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, k.e0, k.e1);
      if (k.site >= 0) tot[k.site] += ms;
      cudaEventDestroy(k.e0);
      cudaEventDestroy(k.e1);
    }
    h.kev.clear();
    for (auto& kv : tot) {
      auto it = best.find(kv.first);
      if (it == best.end() || kv.second < it->second.first) best[kv.first] = {kv.second, c};
    }
  }
  h.force_ch = 0;
  h.prof = prof_was;
  for (auto& kv : best) h.tuned_ch[kv.first] = kv.second.second;
  return {};
}

template Status autotune<double>(Handle&, const double*, double*, cudaStream_t);
template Status autotune<float>(Handle&, const float*, float*, cudaStream_t);

}  // namespace sgdg
