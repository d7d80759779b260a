// Internal data structures of the sgdg library (host side).
#pragma once

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/sgdg.h"

namespace sgdg {

constexpr int kMaxLevels = 12;   // 0..11
constexpr int kR = 2;            // time-DG degree 1: two Legendre coefficients
constexpr int kMaxDim = 3;       // d = 1, 2, 3 (phase space of dimension 2d)
// coefficient function ids of a side: beta components 0 .. 2 kMaxDim - 1, then sigma
constexpr int kSigmaFn = 2 * kMaxDim;

struct Status {
  sgdg_status code = SGDG_OK;
  std::string msg;
};

// The message sgdg_last_error(NULL) returns (calls without a handle).
void set_last_error(const std::string& msg);

// Host CSR (rows sorted, columns sorted within a row).
struct Csr {
  int nrows = 0, ncols = 0;
  std::vector<int> rowptr, col;
  std::vector<double> val;
  int nnz() const { return (int)col.size(); }
};

// One refinement level of a mesh, canonical (lexicographic) vertex order.
struct MeshLevel {
  int n = 0;                          // vertices (periodic masters only)
  std::vector<double> coords;         // n * d
  std::vector<int> cells;             // nc * (d+1), canonical vertex ids
  std::vector<double> cell_coords;    // nc * (d+1) * d, geometric coords
  std::vector<int> bfaces;            // nf * d, canonical vertex ids
  std::vector<double> bface_coords;   // nf * d * d
  std::vector<int> bface_axis, bface_side;
  Csr pattern;                        // P1 adjacency (vertices sharing a cell)
  int ncells(int d) const { return (int)cells.size() / (d + 1); }
  int nbfaces(int d) const { return (int)bfaces.size() / d; }
};

struct Hierarchy {
  int d = 0, L = 0;
  std::vector<MeshLevel> lev;         // 0..L
  std::vector<Csr> E;                 // E[l]: prolongation level l -> l+1 (n_{l+1} x n_l)
  std::vector<Csr> Rt;                // Rt[l] = E[l]^T (n_l x n_{l+1})
  std::vector<std::vector<int>> inj;  // inj[l][k]: level-(l+1) index of level-l vertex k
};

// Host checks of a coarse mesh: box, vertices inside it and distinct, cells
// of positive volume tiling the box, conforming faces (at most two cells;
// one-cell faces on a box side), matching vertices on periodic sides.
Status validate_mesh(const sgdg_mesh& m);
Status build_hierarchy(const sgdg_mesh& m, int L, Hierarchy& h);

// q-point Gauss-Legendre rule on [0, 1] (nodes by Newton's method on P_q).
void gauss_rule01(int q, std::vector<double>& x, std::vector<double>& w);

// ---------------------------------------------------------------------------
// Factors of the Kronecker terms (Sect. 4.2)
// ---------------------------------------------------------------------------

// Coefficient functions on one side: ids into a table of callbacks.
struct SideFns {
  std::vector<sgdg_fn> fn;
  std::vector<void*> user;
  // optional piecewise-constant replacement of function id k: one value per
  // cell of the finest level (nullptr: use fn[k])
  std::vector<const std::vector<double>*> cell;
  const std::vector<double>* cell_field(int id) const {
    return id < (int)cell.size() ? cell[id] : nullptr;
  }
};

// X[i,j] = int w (D_trial phi_j)(D_test phi_i), w = product of fns (no
// scalar); over the domain (kind 0) or the boundary faces of one box side
// (kind 1); restricted to cells whose centroid has sign(fn) == sign.
struct FactorSpec {
  int kind = 0;
  std::vector<int> wfn;                         // sorted function ids
  int test = 0, trial = 0;                      // 0 value, p >= 1: d/dy_p
  std::vector<std::pair<int, int>> restrict_;   // (fn id, sign), sorted
  int face_axis = -1, face_side = 0;
  bool operator<(const FactorSpec& o) const;
  bool operator==(const FactorSpec& o) const;
};

// Volume factors (kind 0) of one hierarchy assembled together on the finest
// level and projected to every coarser level: one pass over the cells in
// chunks evaluates each coefficient function once per quadrature point and
// forms every factor's element matrices, scattered in cell order (values
// independent of the chunking and the thread count).  X[f][l] on
// lev[l].pattern.
Status assemble_volume(const Hierarchy& h, const SideFns& fns, const std::vector<FactorSpec>& specs,
                       std::vector<std::vector<Csr>>& X);

Status assemble_factor(const Hierarchy& h, const SideFns& fns, const FactorSpec& f,
                       std::vector<Csr>& per_level);   // per_level[l] on lev[l].pattern

struct Term {
  double tau[kR][kR];  // time coupling [s][s']
  int x, v;            // factor ids
};

// One contribution to a term's time coupling (Sect. 4.2):
//   scale * sum_mu w_mu g(tau_mu) B_mu      (base M, T, T^T or C)
//   scale * G^(t)                           (base G, the jump at t_{j-1})
// with B_mu the time basis products at the Gauss point tau_mu (M: eta_s'
// eta_s, T: eta'_s' eta_s, C: eta'_s' eta'_s; [s][s'], s the test index),
// g the product of the time factors of the coefficients f1, f2 (function
// ids, -1: none) and, for inflow parts, the indicator that the time factor
// of component gate_fn has the sign gate_sign (times its coefficient).
// Without time factors the sum is the exact time matrix.
struct TauPart {
  enum Base { M = 0, T = 1, TT = 2, C = 3, G = 4 };
  int base = M;
  double scale = 0.0;
  int f1 = -1, f2 = -1;
  int gate_fn = -1, gate_sign = 0;
  double gate_coef = 1.0;
};

struct TermTable {
  std::vector<FactorSpec> xf, vf;
  std::vector<Term> terms;
  std::vector<std::vector<TauPart>> parts;   // per term: its time coupling
  bool time_dep = false;                     // some coefficient has a time factor
};

// The time coupling of every term for the strip (t0, t0 + dt) from its
// parts: an m-point Gauss rule per strip with time factors (ft[id] = the
// callback of function id, NULL: constant 1), the exact time matrices
// without.  Writes terms[k].tau.
Status strip_time_couplings(TermTable& tt, double t0, double dt, int m,
                            const std::vector<std::pair<sgdg_tfn, void*>>& ft);

Status build_terms(const sgdg_coeffs& c, int d, const sgdg_mesh& mx, const sgdg_mesh& mv,
                   double dt, double delta, TermTable& out);

// The inflow boundary Gamma^- of Sect. 2 split into Kronecker pairs (Sect.
// 5.2): <u, w>_{Gamma^-} = sum over parts of scale (x factor) (x) (v factor),
// one part per beta component, box side and sign pair of its two factors
// (function ids 0..2d-1 are the beta components).
struct InflowPart {
  FactorSpec x, v;
  double scale = 0.0;
  int gate_fn = -1, gate_sign = 0;   // time factor of beta[gate_fn]: part active when
                                     // sign(coef * factor(t)) == gate_sign
};
std::vector<InflowPart> inflow_parts(const sgdg_coeffs& c, int d, const sgdg_mesh& mx, const sgdg_mesh& mv,
                                     bool with_time = false);

// C = A B: the structural pattern (sorted rows, no values) and the values of
// A B on that pattern (aval, bval: values of A and B on their patterns).
Csr product_pattern(const Csr& A, const Csr& B);
void product_values(const Csr& A, const std::vector<double>& aval, const Csr& B, const std::vector<double>& bval,
                    const Csr& C, std::vector<double>& cval);

// Load vector F[i] = int fn phi_i on the finest level, restricted to all levels.
Status load_vectors(const Hierarchy& h, sgdg_fn fn, void* user, std::vector<std::vector<double>>& per_level);
// F[i] = int (prod_k fns[k]) D phi_i, D = identity (deriv 0) or d/dy_p (deriv
// p + 1), on the finest level and restricted to all levels; NULL functions
// are the constant 1.
Status load_vectors_w(const Hierarchy& h, const std::vector<std::pair<sgdg_fn, void*>>& fns, int deriv,
                      std::vector<std::vector<double>>& per_level);

}  // namespace sgdg
