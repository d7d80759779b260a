// The sparse-grid operator apply as a linear-cost sweep over the grids.
//
// Sect. 4.2 applies A = sum_{l,l'} A_{l,l'} block by block.  With the Galerkin
// projection X_{l1,l1'} = E^T X E and nested embeddings (E_{L<-l'} =
// E_{L<-l} E_{l<-l'}), every off-diagonal factor splits into a same-level
// factor and a chain of transfers:
//   l1' <= l1:  X_{l1,l1'} = X_{l1} E_{l1<-l1'},   V_{l2,l2'} = E_{l2'<-l2}^T V_{l2'}
//   l1' >  l1:  X_{l1,l1'} = E_{l1'<-l1}^T X_{l1'}, V_{l2,l2'} = V_{l2} E_{l2<-l2'}
// Per term a = (tau, X, V) and grids i = 0..L (grid i = (i, L-i)), summing
// over the sources gives two recursions, each chain keyed by the factor
// applied first (P = prolongation E, R = restriction E^T, subscript = the
// dimension, U_i the input on grid i):
//   branch A (sources l1' <= l1), chains b by V:
//     S_{b,i} = U_i V_b^T + P1 Z_{b,i},   Z_{b,i+1} = S_{b,i} R2^T,   Z_{b,0} = 0
//     Y_i = sum_a tau_a X_a S_{b,i}
//   branch B (sources l1' > l1), chains c by X:
//     Z_{c,L-1} = (R1 X_c) U_L,   Z_{c,i} = (R1 Z_{c,i+1}) P2^T + (R1 X_c) U_{i+1}
//     Y_i += tau_a Z_{c,i} (V_a P2)^T
// Z_{b,i} = S_{b,i-1} R2^T and Z_{c,i} = R1 T_{c,i+1} are the chain states of
// the plain recursions S_i = P1 R2 S_{i-1} + U_i V^T and T'_i = R1 P2 (T'_{i+1}
// + X U_{i+1}) taken one transfer early, restriction before prolongation:
// they live on the coarse side of both dimensions (a quarter of a grid for
// 2-D sides).  S_{b,i}, which includes the diagonal blocks, is formed on every
// grid for its final update and restricted once to carry the chains on;
// branch B never forms T or T' at full size.  The products R1 X_c and V_a P2
// are formed once per level on the host.  On 3D Kuhn lattices R1 X_c has rows
// of 65 entries; there branch B forms T_c = X_c U_{i+1} + Z_{c,i+1} P2^T on
// grid i + 1 and restricts it (Z_{c,i} = R1 T_c), one launch group at a time.  This reaches
// the blockwise sum of Sect. 4.2 exactly in exact arithmetic with
// O(#terms * N) work; no intermediate exceeds one component grid, like the
// ordering rule of Sect. 4.2.
#include <algorithm>
#include <type_traits>

#include "handle.h"
#include "sweep.h"

namespace sgdg {

#define SG_CU(x)                                                              \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) return {SGDG_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)}; \
  } while (0)


namespace {

// bytes of a level's CSR pattern plus nvals value arrays



template <typename T>
Handle::Bufs& bufs(Handle& h);
template <> Handle::Bufs& bufs<double>(Handle& h) { return h.b64; }
template <> Handle::Bufs& bufs<float>(Handle& h) { return h.b32; }
template <> Handle::Bufs& bufs<Bf16>(Handle& h) { return h.b16; }

template <typename T>
Status ensure_bufs(Handle& h) {
  Handle::Bufs& b = bufs<T>(h);
  if (b.S) return {};
  size_t full = sizeof(Store<T>) * (size_t)h.n_coeffs;
  size_t tmp = sizeof(Store<T>) * (size_t)h.tmp_elems;
  if (dev_alloc(h, &b.S, full) != cudaSuccess || dev_alloc(h, &b.Z, full) != cudaSuccess ||
      dev_alloc(h, &b.TP, full) != cudaSuccess || dev_alloc(h, &b.tmp, tmp) != cudaSuccess ||
      dev_alloc(h, &b.W, full) != cudaSuccess)
    return {SGDG_ENOMEM, "sweep buffers"};
  return {};
}

// Sweep pool: the diagonal-block products W_b (one grid each, all A chains;
// on sides without R X products also the full-size branch-B states T_c of
// one launch group), a ring of two chain states Z per chain of both branches,
// and the restricted states Q of one launch group.
struct PoolShape {
  long long mg = 2, mz = 2, mq = 2;   // elements per W, Z and Q slot
  bool wide_b = false;                // branch B through full-size states (no R X products)
  long long nw(const Plan& p) const {
    return std::max<long long>((long long)p.A.size(),
                               wide_b ? std::min<long long>(kChainSlots, (long long)p.B.size()) : 0);
  }
  long long elems(const Plan& p) const {
    const long long a = (long long)p.A.size(), b = (long long)p.B.size();
    return nw(p) * mg + 2 * (a + b) * mz + std::min<long long>(kChainSlots, std::max(a, b)) * mq;
  }
};

inline PoolShape pool_shape(const Handle& h) {
  PoolShape ps;
  const int L = h.L;
  ps.wide_b = !h.X.has_rf;
  for (int l = 0; l <= L; ++l) ps.mg = std::max(ps.mg, 2LL * h.n1[l] * h.n2[l]);
  for (int i = 1; i <= L; ++i) ps.mz = std::max(ps.mz, 2LL * h.X.n[i - 1] * h.V.n[L - i]);
  for (int i = 0; i < L; ++i) ps.mz = std::max(ps.mz, 2LL * h.X.n[i] * h.V.n[L - i - 1]);
  for (int i = 1; i < L; ++i) ps.mq = std::max(ps.mq, 2LL * h.X.n[i - 1] * h.V.n[L - i - 1]);
  for (int i = 0; i + 2 <= L; ++i) ps.mq = std::max(ps.mq, 2LL * h.X.n[i] * h.V.n[L - i - 2]);
  return ps;
}

template <typename T>
struct Pool {
  Store<T>* base = nullptr;
  PoolShape ps;
  size_t nA = 0, nB = 0, nW = 0;
  Store<T>* W(int b) const { return base + (size_t)b * ps.mg; }
  Store<T>* ZA(int b, int par) const { return base + nW * ps.mg + (size_t)(2 * b + par) * ps.mz; }
  Store<T>* ZB(int c, int par) const { return base + nW * ps.mg + 2 * nA * ps.mz + (size_t)(2 * c + par) * ps.mz; }
  Store<T>* Q(int g) const { return base + nW * ps.mg + 2 * (nA + nB) * ps.mz + (size_t)g * ps.mq; }
};

template <typename T>
Status ensure_pool(Handle& h, const Plan& p, Pool<T>& pool) {
  pool.ps = pool_shape(h);
  pool.nA = p.A.size();
  pool.nB = p.B.size();
  pool.nW = (size_t)pool.ps.nw(p);
  // sized once for the largest plan of the handle (the operator's)
  const long long need = std::max(pool.ps.elems(h.op), pool.ps.elems(p));
  Handle::Bufs& b = bufs<T>(h);
  if (!b.pool) {
    if (dev_alloc(h, &b.pool, sizeof(Store<T>) * (size_t)need) != cudaSuccess) return {SGDG_ENOMEM, "sweep chain pool"};
    b.pool_elems = need;
  }
  if (b.pool_elems < pool.ps.elems(p)) return {SGDG_EINVAL, "sweep chain pool too small for this plan"};
  pool.base = (Store<T>*)b.pool;
  return {};
}


// launch site: kind (< 16), chains or terms (< 64), element size, grid shape (< 2^24 each)
inline long long site_key(int kind, int n1, int n2, int count, int elem) {
  const long long head = ((long long)kind * 64 + count) * 16 + elem;
  return (((head << 24) | (long long)n1) << 24) | (long long)n2;
}

// Launch shape of a site: rows per thread (ch, 0 = heuristic), block order
// (tiled), two outputs per thread (pair: final kernels and short-row mode-A
// chain steps), L2 prefetch hints for operands a step ahead (pf: final
// and chain kernels) and the lattice kernels (lat: left finals and mode-A
// chain steps on 2-D lattice x levels, run length from ch).  Tuned choices
// are stored as ch | tiled << 4 | pair << 5 | pf << 6 | lat << 7.  Untuned sites take the column tiles
// when the launch's stencil runs along dim 1 and rows are long enough to fill
// a tile.
struct Shape {
  int ch = 0, tiled = 0, pair = 0, pf = 0, lat = 0;   // lat: the lattice kernel where the level allows it
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
    sh.tiled = (code >> 4) & 1;
    sh.pair = (code >> 5) & 1;
    sh.pf = (code >> 6) & 1;
    sh.lat = (code >> 7) & 1;
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
  // bytes: algorithmic bytes; flops: 2 per multiply-add the launch executes
  // (padded ELL entries included)
  void done(int kind, double bytes, long long site, double flops) {
    h.launches++;
    if (!h.prof) return;
    cudaEventRecord(e1, s);
    h.kev.push_back({kind, bytes, e0, e1, site, flops});
  }
};

template <typename T>
double grid_bytes(long long n1, long long n2) {
  return 2.0 * sizeof(Store<T>) * (double)n1 * (double)n2;
}

template <typename T>
Status run_restrict(Handle& h, RestrictArgs<T>& a, bool dim2, cudaStream_t s, double mat_bytes) {
  const int kind = dim2 ? KIND_XFER_RIGHT : KIND_XFER_LEFT;
  const long long site = site_key(kind, a.n1, a.n2, a.nchains, sizeof(Store<T>));
  const Shape sh = pick_shape<T>(h, site, !dim2, a.n1, a.n2);
  a.ch = sh.ch;
  a.tiled = sh.tiled;
  ProfScope ps(h, s);
  SG_CU(launch_restrict(a, dim2, s));
  ps.done(kind, mat_bytes + a.nchains * (grid_bytes<T>(a.n1_in, a.n2_in) + grid_bytes<T>(a.n1, a.n2)), site,
          4.0 * a.row * a.nchains * (double)a.n1 * a.n2);
  return {};
}

// in_bytes: the matrices, U and the Q inputs the launch reads
template <typename T>
Status run_chain(Handle& h, ChainArgs<T>& a, bool mode_a, int kind, cudaStream_t s, double in_bytes) {
  const long long site = site_key(kind, a.n1, a.n2, a.nchains, sizeof(Store<T>));
  const Shape sh = pick_shape<T>(h, site, !mode_a, a.n1, a.n2);
  a.ch = sh.ch;
  a.tiled = sh.tiled;
  a.pair = sh.pair;
  a.pf = sh.pf;
  ProfScope ps(h, s);
  bool lat = false;
  if constexpr (!std::is_same<T, double>::value) {
    if (mode_a && sh.lat && a.lat_nx > 0 && h.sweep_variant == 1 && a.row == 7) {
      SG_CU(launch_chain_lattice(a, s));
      lat = true;
    }
  }
  if (!lat) SG_CU(launch_chain(a, mode_a, s));
  ps.done(kind, in_bytes + a.nchains * grid_bytes<T>(a.n1, a.n2), site,
          4.0 * (a.row + (a.has_prev ? kProlongRow : 0)) * a.nchains * (double)a.n1 * a.n2);
  return {};
}

// mat_bytes: pattern and value rows the launch reads; in_bytes: one input
template <typename T>
Status run_final(Handle& h, FinalArgs<T>& f, bool left, int kind, cudaStream_t s, double mat_bytes, double in_bytes) {
  const long long site = site_key(kind, f.n1, f.n2, f.nin, sizeof(Store<T>));
  const Shape sh = pick_shape<T>(h, site, left, f.n1, f.n2);
  f.ch = sh.ch;
  f.tiled = sh.tiled;
  f.pair = sh.pair;
  f.pf = sh.pf;
  ProfScope ps(h, s);
  if (left && sh.lat && f.lat_nx > 0 && h.sweep_variant == 1 && f.row == 7) SG_CU(launch_final_lattice(f, s));
  else SG_CU(launch_final(f, left, s));
  const double g = grid_bytes<T>(f.n1, f.n2);
  ps.done(kind, mat_bytes + f.nin * in_bytes + g * (f.accumulate ? 2.0 : 1.0), site,
          2.0 * (2.0 * f.row + 4.0) * f.nterms * (double)f.n1 * f.n2);
  return {};
}

// ELL bytes of `rows` rows of width w: the columns plus nvals value arrays
template <typename T>
double ell_bytes(long long rows, int w, int nvals) {
  return (double)rows * w * (4.0 + (double)nvals * sizeof(Comp<T>));
}

// One final launch family: y (+)= sum over the chains' terms of tau_a F_a in_c
// with F on one ELL pattern (rows: the pattern's rows, w its width).
struct FinalSpec {
  bool left = true;
  int kind = KIND_FINAL_LEFT;
  int n1 = 0, n2 = 0, nin2 = 0;      // output grid, input row length (right)
  const int* col = nullptr;
  int row = 8, w = 8;
  long long mat_rows = 0;
  double in_bytes = 0.0;
  int lat_nx = 0;                    // left on a 2-D lattice level: vertices per lattice row
};

template <typename T, typename InOf, typename ValOf>
Status finals_on(Handle& h, const Plan& p, const std::vector<Chain>& chains, const FinalSpec& fs, InOf in_of,
                 ValOf val_of, bool accumulate_first, Store<T>* ygrid, cudaStream_t s) {
  FinalArgs<T> f;
  f.n1 = fs.n1;
  f.n2 = fs.n2;
  f.nin2 = fs.nin2 > 0 ? fs.nin2 : fs.n2;
  f.row = fs.row;
  f.col = fs.col;
  f.y = ygrid;
  f.lat_nx = fs.lat_nx;
  bool first = true;
  auto flush = [&]() -> Status {
    if (f.nterms == 0) return {};
    f.tbeg[f.nin] = f.nterms;
    f.accumulate = first ? (accumulate_first ? 1 : 0) : 1;
    Status st = run_final(h, f, fs.left, fs.kind, s, ell_bytes<T>(fs.mat_rows, fs.w, f.nterms), fs.in_bytes);
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
      f.val[f.nterms] = val_of(tm);
      for (int a = 0; a < 2; ++a)
        for (int q = 0; q < 2; ++q) f.tau[f.nterms][a * 2 + q] = (Comp<T>)tm.tau[a][q];
      f.nterms++;
    }
  }
  return flush();
}

// Diagonal blocks on one grid (n1 x n2) = (x level lx, v level lv):
//   S_b = u V_b^T (+ P1 Z_b when zin is given: the chain states of branch A)
//   for the chains b (by v factor), then y (+)= sum tau_a X_a S_b
template <typename T, typename ZOf>
Status diag_block(Handle& h, const Plan& p, const Pool<T>& pool, int lx, int lv, const Store<T>* u, Store<T>* y,
                  bool accumulate, cudaStream_t s, ZOf zin) {
  const int n1 = h.X.n[lx], n2 = h.V.n[lv];
  const int nc = (int)p.A.size();
  if (2LL * n1 * n2 > pool.ps.mg) return {SGDG_EINVAL, "diagonal block larger than the sweep slots"};
  const double g = grid_bytes<T>(n1, n2);
  const bool prev = zin(0) != nullptr;
  for (int c0 = 0; c0 < nc; c0 += kChainSlots) {
    ChainArgs<T> a;
    a.n1 = n1;
    a.n2 = n2;
    a.nu2 = n2;
    a.nchains = std::min(kChainSlots, nc - c0);
    a.has_prev = prev;
    a.row = h.V.row_regs();
    a.U = u;
    a.f_col = h.V.ell_col[lv];
    // lattice x level (and, for the prolongation, the lattice level below)
    if (lx < (int)h.X.lat_nx.size() && h.X.lat_nx[lx] && (!prev || h.X.lat_E[lx])) a.lat_nx = h.X.lat_nx[lx];
    for (int c = 0; c < a.nchains; ++c) {
      a.f_val[c] = h.V.vals<Comp<T>>().ell_fac[p.A[c0 + c].first][lv];
      a.out[c] = pool.W(c0 + c);
      a.Z[c] = zin(c0 + c);
    }
    double in = g + ell_bytes<T>(n2, h.V.ell_w(), a.nchains);
    if (prev) {
      a.p_col = h.X.E_ell_col[lx - 1];
      a.p_val = h.X.vals<Comp<T>>().ell_E[lx - 1];
      in += a.nchains * grid_bytes<T>(h.X.n[lx - 1], n2) + ell_bytes<T>(n1, kEllE, 1);
    }
    Status st = run_chain(h, a, true, KIND_S_CHAIN, s, in);
    if (st.code) return st;
  }
  FinalSpec fs;
  fs.left = true;
  fs.kind = KIND_FINAL_LEFT;
  fs.n1 = n1;
  fs.n2 = n2;
  fs.col = h.X.ell_col[lx];
  fs.row = h.X.row_regs();
  fs.w = h.X.ell_w();
  fs.mat_rows = n1;
  fs.in_bytes = g;
  fs.lat_nx = lx < (int)h.X.lat_nx.size() ? h.X.lat_nx[lx] : 0;
  return finals_on<T>(h, p, p.A, fs, [&](int c) { return (const Store<T>*)pool.W(c); },
                      [&](const Term& tm) { return (const Comp<T>*)h.X.vals<Comp<T>>().ell_fac[tm.x][lx]; }, accumulate, y, s);
}

// Branch A on grid i in one fused launch (sweep_fused.cu): S_b formed per
// tile in shared memory, Y_i = sum_a tau_a X_a S_b written, and the
// restricted states Z_{b,i+1} passed on.  False in *done when no plan fits
// (the caller then runs the unfused kernels).
template <typename T>
Status fused_branch_a(Handle& h, const Plan& p, const Pool<T>& pool, int i, const Store<T>* u, Store<T>* y,
                      cudaStream_t s, bool* done) {
  *done = false;
  const int L = h.L, lx = i, lv = L - i;
  const int nA = (int)p.A.size();
  int nterms = 0;
  for (const Chain& c : p.A) nterms += (int)c.terms.size();
  const Handle::FusedGrid* fg = nullptr;
  Status st = fused_plan(h, i, (int)(2 * sizeof(Comp<T>)), nA, nterms, &fg);
  if (st.code || !fg) return st;
  SideDev& X = h.X;
  SideDev& V = h.V;
  FusedArgs<T> a;
  a.tiles = fg->tiles;
  a.xrows = fg->xrows;
  a.vcols = fg->vcols;
  a.xnbr = fg->xnbr;
  a.qcols = fg->qcols;
  a.qloc = fg->qloc;
  a.ntiles = fg->ntiles;
  a.W = fg->W;
  a.n2 = V.n[lv];
  a.n2c = lv >= 1 ? V.n[lv - 1] : 0;
  a.has_prev = i >= 1;
  a.restrict_out = i < L;
  a.nchains = nA;
  a.G = fg->G;
  a.U = u;
  a.Y = y;
  a.vcol = V.ell_col[lv];
  int nt = 0;
  for (int c = 0; c < nA; ++c) {
    a.vval[c] = V.vals<Comp<T>>().ell_fac[p.A[c].first][lv];
    a.zin[c] = i >= 1 ? pool.ZA(c, i & 1) : nullptr;
    a.zout[c] = i < L ? pool.ZA(c, (i + 1) & 1) : nullptr;
    a.tbeg[c] = nt;
    for (int t : p.A[c].terms) {
      const Term& tm = p.terms[t];
      a.xval[nt] = X.vals<Comp<T>>().ell_fac[tm.x][lx];
      for (int q = 0; q < 2; ++q)
        for (int r = 0; r < 2; ++r) a.tau[nt][q * 2 + r] = (Comp<T>)tm.tau[q][r];
      nt++;
    }
  }
  a.tbeg[nA] = nt;
  if (a.has_prev) {
    a.pcol = X.E_ell_col[lx - 1];
    a.pval = X.vals<Comp<T>>().ell_E[lx - 1];
  }
  if (a.restrict_out) {
    a.rcol = V.R_ell_col[lv - 1];
    a.rval = V.vals<Comp<T>>().ell_R[lv - 1];
  }
  ProfScope ps(h, s);
  SG_CU(launch_fused_a(a, fg->smem, s));
  const int n1 = X.n[lx], n2 = V.n[lv], W = fg->W;
  const double g = grid_bytes<T>(n1, n2);
  double bytes = 2.0 * g + ell_bytes<T>(n1, W, nt) + ell_bytes<T>(n2, W, nA);
  if (a.has_prev) bytes += nA * grid_bytes<T>(X.n[lx - 1], n2) + ell_bytes<T>(n1, kEllE, 1);
  if (a.restrict_out) bytes += nA * grid_bytes<T>(n1, a.n2c) + ell_bytes<T>(a.n2c, W, 1);
  const double flops = 2.0 * (fg->s_points * nA * (2.0 * W + (a.has_prev ? 4.0 : 0.0)) +
                              (double)n1 * n2 * nt * (2.0 * W + 4.0) + fg->q_points * nA * 2.0 * W);
  ps.done(KIND_FUSED_A, bytes, -1, flops);
  *done = true;
  return {};
}

}  // namespace

template <typename T>
Status apply_plan(Handle& h, const Plan& p, const Store<T>* u, Store<T>* y, cudaStream_t s, const ApplyHooks* hooks) {
  NvtxRange range("sgdg.apply");
  Pool<T> pool;
  Status st = ensure_pool<T>(h, p, pool);
  if (st.code) return st;
  const int L = h.L;
  const int G = kChainMax<T>();
  const int nA = (int)p.A.size(), nB = (int)p.B.size();
  SideDev& X = h.X;
  SideDev& V = h.V;
  // ---- diagonal blocks and branch A (sources l1' < l1): chains by the v factor
  for (int i = 0; i <= L; ++i) {
    const int lv = L - i;
    // S_{b,i} = U_i V_b^T + P1 Z_{b,i};  Y_i = sum_a tau_a X_a S_{b,i}
    if (hooks && hooks->ready) SG_CU(cudaStreamWaitEvent(s, hooks->ready[i], 0));
    Store<T>* yi = y + h.off[i];
    bool fused = false;
    if (h.sweep_variant == 0) {
      st = fused_branch_a<T>(h, p, pool, i, u + h.off[i], yi, s, &fused);
      if (st.code) return st;
    }
    if (fused) {
      if (i == L && hooks && hooks->done) {
        st = hooks->done(hooks->ctx, L);
        if (st.code) return st;
      }
      if (i == L) break;
      continue;
    }
    st = diag_block<T>(h, p, pool, i, lv, u + h.off[i], yi, false, s,
                       [&](int c) { return i >= 1 ? (const Store<T>*)pool.ZA(c, i & 1) : (const Store<T>*)nullptr; });
    if (st.code) return st;
    if (i == L) {
      if (hooks && hooks->done) {   // grid L gets no branch-B contribution
        st = hooks->done(hooks->ctx, L);
        if (st.code) return st;
      }
      break;
    }
    // Z_{b,i+1} = S_{b,i} R2^T  (nx[i] x nv[lv-1]): S_{b,i} is already formed
    // for the final update, so one restriction carries every chain forward
    for (int c0 = 0; c0 < nA; c0 += G) {
      const int nc = std::min(G, nA - c0);
      RestrictArgs<T> r;
      r.n1 = X.n[i];
      r.n2 = V.n[lv - 1];
      r.n1_in = X.n[i];
      r.n2_in = V.n[lv];
      r.nchains = nc;
      r.row = V.row_regs();
      r.col = V.R_ell_col[lv - 1];
      r.val = V.vals<Comp<T>>().ell_R[lv - 1];
      for (int g = 0; g < nc; ++g) {
        r.in[g] = pool.W(c0 + g);
        r.out[g] = pool.ZA(c0 + g, (i + 1) & 1);
      }
      st = run_restrict(h, r, true, s, ell_bytes<T>(V.n[lv - 1], V.ell_w(), 1));
      if (st.code) return st;
    }
  }
  // ---- branch B (sources l1' > l1): chains by the x factor
  for (int i = L - 1; i >= 0; --i) {
    const int lv = L - i;   // output v level; Z_{c,i}: (nx[i] x nv[lv-1])
    for (int c0 = 0; c0 < nB; c0 += G) {
      const int nc = std::min(G, nB - c0);
      const bool prev = i < L - 1;
      if (!X.has_rf) {
        // no R X products (3D): T_c = X_c U_{i+1} + Z_{c,i+1} P2^T on grid
        // i + 1 (nx[i+1] x nv[lv-1]), then Z_{c,i} = R1 T_c
        ChainArgs<T> a;
        a.n1 = X.n[i + 1];
        a.n2 = V.n[lv - 1];
        a.nu2 = V.n[lv - 1];
        a.nz2 = prev ? V.n[lv - 2] : 0;
        a.nchains = nc;
        a.has_prev = prev;
        a.row = X.row_regs();
        a.U = u + h.off[i + 1];
        a.f_col = X.ell_col[i + 1];
        for (int g = 0; g < nc; ++g) {
          a.f_val[g] = X.vals<Comp<T>>().ell_fac[p.B[c0 + g].first][i + 1];
          a.out[g] = pool.W(g);
          a.Z[g] = prev ? pool.ZB(c0 + g, (i + 1) & 1) : nullptr;
        }
        double in = grid_bytes<T>(h.n1[i + 1], h.n2[i + 1]) + ell_bytes<T>(X.n[i + 1], X.ell_w(), nc);
        if (prev) {
          a.p_col = V.E_ell_col[lv - 2];
          a.p_val = V.vals<Comp<T>>().ell_E[lv - 2];
          in += nc * grid_bytes<T>(X.n[i + 1], V.n[lv - 2]) + ell_bytes<T>(V.n[lv - 1], kEllE, 1);
        }
        st = run_chain(h, a, false, KIND_CHAIN_B, s, in);
        if (st.code) return st;
        RestrictArgs<T> r;
        r.n1 = X.n[i];
        r.n2 = V.n[lv - 1];
        r.n1_in = X.n[i + 1];
        r.n2_in = V.n[lv - 1];
        r.nchains = nc;
        r.row = X.row_regs();
        r.col = X.R_ell_col[i];
        r.val = X.vals<Comp<T>>().ell_R[i];
        for (int g = 0; g < nc; ++g) {
          r.in[g] = pool.W(g);
          r.out[g] = pool.ZB(c0 + g, i & 1);
        }
        st = run_restrict(h, r, false, s, ell_bytes<T>(X.n[i], X.ell_w(), 1));
        if (st.code) return st;
        continue;
      }
      double qbytes = 0.0;
      if (prev) {
        RestrictArgs<T> r;   // Q_g = R1 Z_{c,i+1}: (nx[i] x nv[lv-2])
        r.n1 = X.n[i];
        r.n2 = V.n[lv - 2];
        r.n1_in = X.n[i + 1];
        r.n2_in = V.n[lv - 2];
        r.nchains = nc;
        r.row = X.row_regs();
        r.col = X.R_ell_col[i];
        r.val = X.vals<Comp<T>>().ell_R[i];
        for (int g = 0; g < nc; ++g) {
          r.in[g] = pool.ZB(c0 + g, (i + 1) & 1);
          r.out[g] = pool.Q(g);
        }
        st = run_restrict(h, r, false, s, ell_bytes<T>(X.n[i], X.ell_w(), 1));
        if (st.code) return st;
        qbytes = nc * grid_bytes<T>(r.n1, r.n2) + ell_bytes<T>(V.n[lv - 1], kEllE, 1);
      }
      // Z_{c,i} = Q P2^T + (R1 X_c) U_{i+1}
      ChainArgs<T> a;
      a.n1 = X.n[i];
      a.n2 = V.n[lv - 1];
      a.nu2 = V.n[lv - 1];
      a.nz2 = prev ? V.n[lv - 2] : 0;
      a.nchains = nc;
      a.has_prev = prev;
      a.row = row_class(X.rf_row);
      a.U = u + h.off[i + 1];
      a.f_col = X.RF_ell_col[i];
      for (int g = 0; g < nc; ++g) {
        a.f_val[g] = X.vals<Comp<T>>().ell_RF[p.B[c0 + g].first][i];
        a.out[g] = pool.ZB(c0 + g, i & 1);
        a.Z[g] = prev ? pool.Q(g) : nullptr;
      }
      if (prev) {
        a.p_col = V.E_ell_col[lv - 2];
        a.p_val = V.vals<Comp<T>>().ell_E[lv - 2];
      }
      st = run_chain(h, a, false, KIND_CHAIN_B, s,
                     qbytes + grid_bytes<T>(h.n1[i + 1], h.n2[i + 1]) + ell_bytes<T>(X.n[i], X.rf_w(), nc));
      if (st.code) return st;
    }
    // Y_i += sum_a tau_a Z_{c,i} (V_a P2)^T
    FinalSpec fs;
    fs.left = false;
    fs.kind = KIND_FINAL_RIGHT;
    fs.n1 = h.n1[i];
    fs.n2 = h.n2[i];
    fs.nin2 = V.n[lv - 1];
    fs.col = V.FP_ell_col[lv];
    fs.row = row_class(V.fp_row);
    fs.w = V.fp_w();
    fs.mat_rows = V.n[lv];
    fs.in_bytes = grid_bytes<T>(X.n[i], V.n[lv - 1]);
    st = finals_on<T>(h, p, p.B, fs, [&](int c) { return (const Store<T>*)pool.ZB(c, i & 1); },
                      [&](const Term& tm) { return (const Comp<T>*)V.vals<Comp<T>>().ell_FP[tm.v][lv]; }, true, y + h.off[i], s);
    if (st.code) return st;
    if (hooks && hooks->done) {
      st = hooks->done(hooks->ctx, i);
      if (st.code) return st;
    }
  }
  return {};
}

template Status apply_plan<double>(Handle&, const Plan&, const double*, double*, cudaStream_t, const ApplyHooks*);
template Status apply_plan<float>(Handle&, const Plan&, const float*, float*, cudaStream_t, const ApplyHooks*);
template Status apply_plan<Bf16>(Handle&, const Plan&, const __nv_bfloat16*, __nv_bfloat16*, cudaStream_t,
                                 const ApplyHooks*);

// Diagonal blocks A_{l,l} on a list of grids (l1[g], l2[g]): the component
// systems of the combination-technique preconditioner.  Per grid: one launch
// forms W_b = u V_b^T for every distinct v factor (the chain-step kernel
// without a transfer), then fused final launches fold all terms into y.
template <typename T>
Status apply_diag_grids(Handle& h, int ng, const int* l1, const int* l2, const Store<T>* const* u,
                        Store<T>* const* y, cudaStream_t s) {
  Pool<T> pool;
  Status st = ensure_pool<T>(h, h.op, pool);
  if (st.code) return st;
  for (int g = 0; g < ng; ++g) {
    st = diag_block<T>(h, h.op, pool, l1[g], l2[g], u[g], y[g], false, s, [](int) { return (const Store<T>*)nullptr; });
    if (st.code) return st;
  }
  return {};
}

template Status apply_diag_grids<double>(Handle&, int, const int*, const int*, const double* const*,
                                         double* const*, cudaStream_t);
template Status apply_diag_grids<float>(Handle&, int, const int*, const int*, const float* const*, float* const*,
                                        cudaStream_t);
template Status apply_diag_grids<Bf16>(Handle&, int, const int*, const int*, const __nv_bfloat16* const*,
                                       __nv_bfloat16* const*, cudaStream_t);

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
Status autotune(Handle& h, const Store<T>* u, Store<T>* y, cudaStream_t s) {
  // rows per thread x block order x paired outputs x L2 prefetch hints,
  // encoded as ch | tiled << 4 | pair << 5 | pf << 6; plus the lattice
  // kernels (bit 7) with their run lengths (from ch), used where a level is
  // a 2-D lattice and ignored elsewhere
  std::vector<int> cand;
  for (int pf = 0; pf < 2; ++pf)
    for (int pair = 0; pair < 2; ++pair)
      for (int tiled = 0; tiled < 2; ++tiled)
        for (int ch : {1, 2, 4, 8}) cand.push_back(ch | tiled << 4 | pair << 5 | pf << 6);
  if (h.X.lat_nx.size() && *std::max_element(h.X.lat_nx.begin(), h.X.lat_nx.end()) > 0)
    for (int ch : {2, 4, 8}) cand.push_back(ch | 1 << 7);
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
template Status autotune<Bf16>(Handle&, const __nv_bfloat16*, __nv_bfloat16*, cudaStream_t);

}  // namespace sgdg
