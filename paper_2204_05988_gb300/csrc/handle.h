// The library handle: host description + device-resident data of one problem.
#pragma once

#include <map>
#include <memory>

#include "device.h"
#include "sweep.h"

namespace sgdg {

// FNV-1a, 64 bit (Fowler, Noll, Vo): h ^= byte, h *= 1099511628211 per
// byte, starting from the offset basis 14695981039346656037.  The problem
// identity and the checksum of checkpoint files.
constexpr unsigned long long kFnvBasis = 14695981039346656037ULL;
inline void fnv1a64(unsigned long long& hsh, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    hsh ^= b[i];
    hsh *= 1099511628211ULL;
  }
}

// Device copies of one side's (Omega_x or Omega_v) level data.
template <typename T>
struct SideValues {
  std::vector<T*> E, R;               // E[l]: level l -> l+1 values;  R[l] = E[l]^T values
  std::vector<T*> dinv;               // inverse diagonal of the mass matrix per level
  // ELL copies read by the sweep kernels: row r's entries at [r w, r w + len),
  // zero padding (w = SideDev::ell_w(); E: kEllE)
  std::vector<std::vector<T*>> ell_fac;   // [factor][level]
  std::vector<T*> ell_E, ell_R;
  // products with the transfers, ELL: RF[f][l] = R_l F_{l+1} (l < L, width
  // rf_w; sides with has_rf), FP[f][l] = F_l E_{l-1} (1 <= l <= L, width fp_w;
  // sides with has_fp)
  std::vector<std::vector<T*>> ell_RF, ell_FP;
};

constexpr int kEllE = 2;   // ELL width of the prolongation (rows of at most 2 entries)

struct SideDev {
  std::vector<int> n, nnz, E_nnz, R_nnz;
  std::vector<int*> rowptr, col;                  // P1 pattern per level
  std::vector<int*> E_rowptr, E_col, R_rowptr, R_col;
  std::vector<int*> inj;                          // level l vertex -> index on level l+1
  int mass = -1;                                  // factor id of the plain mass matrix
  int maxrow = 8;                                 // longest pattern or restriction row
  // row length the sweep kernels keep in registers (3, 4, 7, 8 or 16: P1
  // rows of 3 in 1D, 7 in 2D, 15 on 3D Kuhn lattices) and the ELL width of
  // the patterns and restrictions (4, 8 or 16, 16-byte rows for vector loads)
  int row_regs() const { return maxrow <= 3 ? 3 : maxrow <= 4 ? 4 : maxrow <= 7 ? 7 : maxrow <= 8 ? 8 : 16; }
  int ell_w() const { return maxrow <= 4 ? 4 : maxrow <= 8 ? 8 : 16; }
  std::vector<int*> ell_col, R_ell_col, E_ell_col;   // ELL column indices (padding repeats the first column)
  // patterns of the factor-transfer products (shared by all factors of the side)
  std::vector<int*> RF_ell_col, FP_ell_col;          // [l] as SideValues::ell_RF / ell_FP
  int rf_row = 0, fp_row = 0;                        // longest product rows
  bool has_rf = false, has_fp = false;               // R F / F E products formed for this side
  static int ell_width(int row) { return (row + 3) / 4 * 4; }
  int rf_w() const { return ell_width(rf_row); }
  int fp_w() const { return ell_width(fp_row); }
  std::vector<Csr> RF_pat, FP_pat;                   // host patterns (FP_pat[0] empty)
  // 2-D structured lattice levels (lexicographic vertex order, every cell
  // cut along the (1, 1) diagonal): lat_nx[l] = vertices per lattice row, 0
  // when level l is not such a lattice.  Their pattern ELL rows (columns and
  // every factor's values) are in stencil-slot order - offsets -nx-1, -nx,
  // -1, 0, 1, nx, nx+1, then one padding slot - with column = the row itself
  // and value 0 for an absent neighbour; lat_pos[l][r w + s] is the CSR
  // position of slot s of row r (-1: absent or padding)
  std::vector<int> lat_nx;
  std::vector<std::vector<int>> lat_pos;
  bool lattice_ok = false;            // look for lattice levels (the x side)
  // lat_E[l] (l >= 1): levels l and l - 1 are lattices and E_{l <- l-1} is
  // the P1 prolongation of the lattice (1 at coarse vertices, 1/2 + 1/2 at
  // the midpoints of row, column and (1, 1)-diagonal edges)
  std::vector<char> lat_E;
  SideValues<double> v64;
  SideValues<float> v32;
  template <typename T> SideValues<T>& vals();
  template <typename T> const SideValues<T>& vals() const;
};
template <> inline SideValues<double>& SideDev::vals<double>() { return v64; }
template <> inline SideValues<float>& SideDev::vals<float>() { return v32; }
template <> inline const SideValues<double>& SideDev::vals<double>() const { return v64; }
template <> inline const SideValues<float>& SideDev::vals<float>() const { return v32; }

// A grouping of terms that share the factor applied first in a sweep branch.
struct Chain {
  int first;               // factor id applied first (V for by_v, X otherwise)
  bool by_v;               // first factor is on the v side
  std::vector<int> terms;  // term indices
};

struct Plan {
  std::vector<Term> terms;
  std::vector<Chain> A, B;  // branch A: sources l1' <= l1; branch B: l1' > l1
  std::vector<Chain> D;     // diagonal-block apply grouping
};

struct Workspace;  // solver buffers (solve.cu)

struct Handle {
  sgdg_config cfg{};
  int d = 0, L = 0;
  std::string err;
  TermTable tt;
  SideDev X, V;
  std::vector<int> n1, n2;           // grid l: (n1[l], n2[l]) = (nx[l], nv[L-l])
  std::vector<long long> off;        // element offsets (with the time index)
  std::vector<long long> soff;       // spatial offsets
  long long n_coeffs = 0, n_spatial = 0;
  Plan op, mass;
  Plan h1;   // H^1(I_j x Omega) Gram form: (M_t + C_t) (x) M (x) M + M_t (x) (K_p (x) M + M (x) K_p)
  // sweep buffers per precision (FP64, FP32, BF16 storage), allocated lazily
  struct Bufs {
    void* S = nullptr; void* Z = nullptr; void* TP = nullptr; void* tmp = nullptr; void* W = nullptr;
    void* cvt_in = nullptr; void* cvt_out = nullptr;
    void* pool = nullptr; long long pool_elems = 0;   // sweep chain states
  } b64, b32, b16;
  // host-buffer apply: compute and copy streams, per-grid events
  cudaStream_t host_s = nullptr, host_c = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_out;
  long long tmp_elems = 0;
  // host copies of the u0 load vectors per level (for set_initial)
  std::vector<std::vector<std::vector<double>>> u0x, u0v;   // [product][level][n]
  std::vector<double> u0coef;
  // source terms of the strip right-hand side (Sect. 2, b_j): per term the x
  // and v load vectors per level (device) and which time weight scales them:
  // kind 0 - int ft eta_s + delta int ft eta_s',  kind 1 - delta int ft eta_s,
  // kind 2 - minus int gt eta_s (inflow data on Gamma^-)
  // one Kronecker term of the source or inflow data; tfn: time factor of a
  // beta component (coef_t id) in the integrand, -1 none; gate_*: an inflow
  // part active where sign(gate_coef factor(t)) == gate_sign (Sect. 4.2)
  struct SourceTerm {
    int src = 0, kind = 0;
    double coef = 0.0;
    std::vector<double*> lx, lv;
    int tfn = -1, gate_fn = -1, gate_sign = 0;
    double gate_coef = 0.0;
  };
  std::vector<SourceTerm> src_terms;
  std::vector<std::pair<sgdg_tfn, void*>> src_t;   // time factor per source
  double t_now = 0.0;                              // start of the next strip
  // time factors of the coefficients (function ids: beta 0..2 kMaxDim - 1,
  // then sigma; NULL = 1), the Gauss points per strip, and a counter bumped
  // whenever the time couplings of h.op change (batch graphs re-capture)
  std::vector<std::pair<sgdg_tfn, void*>> coef_t;
  int time_quad = 3;
  long long tau_version = 0;
  // strip state
  double* U_end = nullptr;   // spatial, n_spatial
  double* u_sol = nullptr;   // last strip solution, n_coeffs
  double* rhs = nullptr;     // n_coeffs
  bool have_initial = false, first_strip = true, solved = false;
  int warm = 0;              // initial guess of the next strip: 0 zero, 1 last solution, 2 guess,
                             // 3 extrapolation of the last two solutions
  double* guess = nullptr;   // n_coeffs, allocated by sgdg_set_guess
  double* u_prev2 = nullptr; // the solution before the last one (for mode 3)
  int nsolved = 0;           // strips solved since set_initial
  size_t device_bytes = 0;
  Workspace* ws = nullptr;      // owned; released by solver_free
  cudaStream_t cur = nullptr;
  // launch accounting: every SpMM launch is counted; with profiling on, each
  // one is bracketed by CUDA events and its algorithmic bytes recorded
  long long launches = 0;
  bool prof = false;
  struct KEvent { int kind; double bytes; cudaEvent_t e0, e1; long long site; double flops = 0.0; };
  std::vector<KEvent> kev;
  // autotuner: launch shape per launch site (kind and grid shape), stored as
  // rows per thread | block order << 4 | paired outputs << 5 | L2 prefetch
  // hints << 6; force_ch > 0
  // overrides every site while tuning
  std::map<long long, int> tuned_ch;
  int force_ch = 0;
  // Vlasov-Poisson coupling (kept only when cfg.vlasov_poisson)
  struct Field {
    Hierarchy hx;                              // Omega_x levels (finest level for assembly)
    SideFns fx;                                // x function table; E ids carry cell fields
    std::vector<std::vector<double>> E;        // E_i per finest x cell, i < d
    std::vector<std::vector<double>> mv;       // int phi^(2)_k per v level
    std::vector<double*> d_mv;                 // device copies
    std::vector<double> rho0;                  // density of u0 at the finest x vertices
    std::vector<double> rho, phi;              // last density and potential
    Csr K, M;                                  // finest-level stiffness and mass (FP64)
    double* d_rowsum = nullptr;                // per-grid int U dv (device, sum of n1)
    bool updated = false;                      // E comes from a field update (not the create-time callback)
  };
  std::unique_ptr<Field> field;
  int vp_stop = 0;                 // fixed-point stop: 0 relative change of phi, 1 Sect. 5.3's norms
  double* vp_prev = nullptr;       // previous iterate f^(k) (n_coeffs), allocated on first use
  double* vp_tmp = nullptr;
  // host level hierarchies (patterns, transfers, coordinates), kept for the
  // fused sweep's tile planner
  std::shared_ptr<Hierarchy> hx_host, hv_host;
  // fused branch-A launch plans per (grid, bytes of an S pair), built on first use
  struct FusedGrid {
    bool tried = false, ok = false;
    int G = 0, ntiles = 0, W = 0;
    size_t smem = 0;
    double s_points = 0.0;        // S_b entries formed per chain (interior and halo)
    double q_points = 0.0;        // restricted outputs per chain
    std::string why;              // reason when no plan fits
    FusedTile* tiles = nullptr;
    int* xrows = nullptr;
    int* vcols = nullptr;
    unsigned short* xnbr = nullptr;
    int* qcols = nullptr;
    unsigned short* qloc = nullptr;
  };
  std::map<long long, FusedGrid> fused;
  int sweep_variant = 1;          // 0: fused branch A where a plan fits; 1 (default): unfused kernels, the
                                  // lattice final on 2-D lattice levels; 2: unfused, generic finals only
  // identity of the discrete problem (meshes, levels, dt, delta, term table,
  // finest-level factor values at creation), checked by sgdg_restore
  unsigned long long problem_hash = 0;
  size_t budget = 0;   // device-memory budget of the handle (0: none), checked by dev_alloc
  ~Handle();
};

// kinds of SpMM launches for the per-kernel statistics
enum {
  KIND_S_CHAIN = 0, KIND_FINAL_LEFT = 1, KIND_XFER_LEFT = 2, KIND_XFER_RIGHT = 3,
  KIND_FUSED_A = 4, KIND_CHAIN_B = 5, KIND_RESERVED = 6, KIND_FINAL_RIGHT = 7, KIND_COUNT = 8
};

// allocation helper that records bytes and reports ENOMEM
cudaError_t dev_alloc(Handle& h, void** p, size_t bytes);

// ELL (width w) copies of a CSR matrix: row r's entries at [r w, r w + len);
// padded columns repeat the row's first column, padded values are zero.
std::vector<int> ell_columns(const std::vector<int>& rowptr, const std::vector<int>& col, int w);
std::vector<double> ell_values(const std::vector<int>& rowptr, const std::vector<double>& val, int w);
// Values of factor f's products with the transfers (R_l F_{l+1}, F_l E_{l-1})
// from its per-level matrices X, uploaded in ELL form (allocated on first use).
Status upload_factor_products(Handle& h, const Hierarchy& hi, SideDev& sd, int f, const std::vector<Csr>& X);
// The same in two steps: host values of the products (no device work; safe
// to run concurrently for different factors), then their upload.
struct FactorProducts { std::vector<std::vector<double>> rf, fp; };
void factor_products(const Hierarchy& hi, const SideDev& sd, const std::vector<Csr>& X, FactorProducts& out);
Status upload_products(Handle& h, SideDev& sd, int f, const FactorProducts& pr);
// Uploads the FP64 and FP32 ELL values; allocates when *d64 is null, else overwrites.
Status upload_ell_vals(Handle& h, const std::vector<int>& rowptr, const std::vector<double>& val, int w,
                       double** d64, float** d32);
// The ELL columns of level l's pattern P as the device holds them (slot order
// on lattice levels), and the upload of a factor's values on that pattern.
std::vector<int> pattern_ell_columns(const SideDev& sd, const Csr& P, int l);
Status upload_pattern_vals(Handle& h, const SideDev& sd, const Csr& P, int l, const std::vector<double>& val,
                           double** d64, float** d32);

// Optional per-grid synchronisation of an apply: before grid i's input U_i
// is first read the stream waits for ready[i]; once Y_i is final, done(i)
// is called (it may enqueue work that reads Y_i on another stream).
struct ApplyHooks {
  const cudaEvent_t* ready = nullptr;
  Status (*done)(void* ctx, int grid) = nullptr;
  void* ctx = nullptr;
};

template <typename T>
Status apply_plan(Handle& h, const Plan& p, const Store<T>* u, Store<T>* y, cudaStream_t s,
                  const ApplyHooks* hooks = nullptr);
template <typename T>
Status apply_diag_grids(Handle& h, int ng, const int* l1, const int* l2, const Store<T>* const* u,
                        Store<T>* const* y, cudaStream_t s);
Status nodal_eval(Handle& h, const double* u, double* out, cudaStream_t s);

// Time candidate rows-per-thread settings of every sweep launch site on live
// applies of u and keep the fastest per site.
template <typename T>
Status autotune(Handle& h, const Store<T>* u, Store<T>* y, cudaStream_t s);

// Vlasov-Poisson coupling (field.cu)
Status field_setup(Handle& h, const sgdg_coeffs& c, const Hierarchy& hx, const Hierarchy& hv, const SideFns& fx);
// Fused branch-A plan of grid i for S pairs of pair_bytes bytes and nchains
// chains (sweep_fused_plan.cu); *out is null when no tile shape fits.
Status fused_plan(Handle& h, int i, int pair_bytes, int nchains, int nterms, const Handle::FusedGrid** out);
Status field_update(Handle& h, int source, double* energy);
Status field_reassemble(Handle& h);
// caller-supplied field: E[k * n_cells + e] = component k on finest x cell e
Status field_set(Handle& h, const double* E, int n_cells);
Status field_get(const Handle& h, double* E, int n_cells);

// coarse full-grid views (coarse.cu)
Status coarse_values(Handle& h, const double* u, int R, int lx, int lv, double* out, cudaStream_t s);
Status add_coarse(Handle& h, const double* c, int lx, int lv, double* u, cudaStream_t s);
Status coarse_diff(Handle& h, const double* a, const double* b, int R, int lx, int lv, double* out,
                   cudaStream_t s);

Status solver_init(Handle& h);
// ||u||_{H^1(I_j x Omega)} of a strip vector (FP64, device): u . (G u) with
// the Gram plan h.h1 (deterministic reduction); tmp: n_coeffs doubles.
Status h1_norm(Handle& h, const double* u, double* tmp, double* out, cudaStream_t s);
// dst = (U, 0): a spatial vector as the strip function constant in time
Status constant_in_time(Handle& h, const double* U, double* dst, cudaStream_t s);
Status ct_precondition(Handle& h, const double* r, double* z, cudaStream_t s, int* inner_its);
Status advance_strip(Handle& h, cudaStream_t s, sgdg_strip_stats* st, bool resolve = false);
// With time factors of beta or sigma: the time couplings of the operator for
// the strip (t0, t0 + dt) (Sect. 4.2 quadrature); nothing otherwise.
Status set_strip_time(Handle& h, double t0);
void solver_free(Handle& h);

}  // namespace sgdg
