/*
 * sgdg.h - C ABI of the GB300 sparse-grid time-DG streamline-diffusion
 * transport library (sm_103a CUDA + C++).
 *
 * Problem (Sect. 1, Eqs. 1-2): d_t u + beta . grad u + sigma u = f on
 * (0,T) x Omega, Omega = Omega_x x Omega_v (both d-dimensional, d = 1, 2, 3),
 * u(0) = u0, inflow u = g on Gamma^- = {beta . n < 0}, with f and g sums of
 * separable terms.
 *
 * Discretisation (Sect. 2): sparse grid V_L = sum_{l=0..L} V^(1)_l (x) V^(2)_{L-l}
 * of nested continuous P1 spaces on simplicial meshes (levels 0-based: the
 * paper's level is L+1), time-DG of degree r = 1 on strips, streamline
 * diffusion with parameter delta; the strip problem a_j(U_j, w) = b_j(w) of
 * Eq. 5 is solved strip by strip.  (P2 and tensor-product Q_r elements on
 * d-cubes, which Sect. 5.1 also uses, are not built.)
 *
 * Storage (Sect. 4.1): a sparse-grid coefficient vector is the concatenation
 * over grids l = 0..L of arrays u_l[k1][k2][s] (row-major, s fastest), k1 over
 * the vertices of level l of Omega_x, k2 over level L-l of Omega_v, s = 0, 1
 * the Legendre time basis eta_s(t) = P_s(2 (t - t_{j-1}) / dt - 1).  Vertices
 * of every level are ordered lexicographically by coordinates (last axis
 * slowest).  A spatial vector (no time index) has the same layout without s.
 * These coefficients belong to a spanning set: they are not unique
 * (Sect. 4.1); operator outputs are unique (rows are test functions).
 *
 * Conventions:
 *  - Every call returns an sgdg_status; on error, outputs are untouched and
 *    sgdg_last_error() describes the failure.
 *  - The caller owns every array it passes.  Mesh arrays and callbacks are
 *    read during sgdg_create only.  The library owns all memory it allocates
 *    (device and host) and frees it in sgdg_destroy.
 *  - Device pointers passed in (u, y, r, z) must be allocations on the
 *    handle's device, 16-byte aligned, and are not retained after the call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream); calls taking a
 *    stream enqueue work on it and may synchronise it to read Krylov scalars.
 *  - A handle is thread-compatible, not thread-safe.
 */
#ifndef SGDG_H
#define SGDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SGDG_OK = 0,
  SGDG_EINVAL = 1,     /* bad argument or unsupported configuration */
  SGDG_ENOMEM = 2,     /* device or host allocation failed / over budget */
  SGDG_ECUDA = 3,      /* a CUDA call failed */
  SGDG_ENOCONV = 4,    /* Krylov solve hit its iteration cap (stats filled) */
  SGDG_ENAN = 5,       /* NaN or Inf met in a residual */
  SGDG_ETIMEOUT = 6,   /* a bounded device wait gave up */
  SGDG_EIO = 7
} sgdg_status;

typedef enum {
  SGDG_FP64 = 0,        /* every apply, transfer and Krylov vector in FP64 */
  SGDG_MIXED_FP32 = 1,  /* FP32 apply / transfers / component solves, FP64
                           Krylov scalars and FP64 outer residual
                           (iterative refinement) */
  SGDG_BF16_STORE = 2   /* applies only (operator, mass, diagonal blocks,
                           autotune, batch): every grid array - input,
                           chain states, output - stored in bfloat16
                           (round to nearest even), FP32 matrix values and
                           FP32 arithmetic.  Half the bytes per element of
                           FP32; about 2^-8 relative rounding per stored
                           intermediate.  Not a solver precision. */
} sgdg_precision;

/* Outer iteration of a strip solve; both stop on the FP64 true residual
 * ||b - A u||_2 <= rtol ||b||_2. */
typedef enum {
  SGDG_OUTER_FGMRES = 0,      /* right-preconditioned FGMRES with the CT
                                 preconditioner (restart, max_outer) */
  SGDG_OUTER_RICHARDSON = 1   /* Algorithm 1 (Sect. 4.3): u <- u + P_CT(b - A u),
                                 one CT preconditioner step and one FP64
                                 apply per iteration, up to max_outer */
} sgdg_outer;

/* A coarse simplicial mesh of an axis-aligned box (one of Omega_x, Omega_v).
 * coords: [n_vertices][dim]; cells: [n_cells][dim+1] vertex indices.
 * lo/hi: box bounds per axis; periodic: per-axis flag (0/1; NULL: none).
 * Uniform refinement (1D bisection, 2D red refinement, 3D regular
 * refinement after Bey, which keeps a Kuhn mesh a Kuhn mesh when its
 * tetrahedra list their vertices along a monotone lattice path) builds the
 * levels (Sect. 2).  sgdg_create checks each mesh on the host before it
 * touches a device and returns SGDG_EINVAL when: lo < hi fails on an axis;
 * a vertex lies outside the box or two share their coordinates; a cell
 * index is out of range or a cell has zero volume; the cell volumes do not
 * add up to the box volume; a face lies in more than two cells, or a face of
 * one cell is not on a side of the box; or the vertices on the two sides of
 * a periodic axis do not match. */
typedef struct {
  int dim;
  int n_vertices;
  const double* coords;
  int n_cells;
  const int* cells;
  const double* lo;
  const double* hi;
  const int* periodic;
} sgdg_mesh;

/* Batched coefficient callback: out[i] = f(pts[i*dim .. i*dim+dim-1]),
 * i < npts.  Called on the host during sgdg_create / sgdg_set_initial. */
typedef void (*sgdg_fn)(int npts, const double* pts, double* out, void* user);

/* coef * fx(x) * fv(v); a NULL function is the constant 1 (Sect. 4.2). */
typedef struct {
  double coef;
  sgdg_fn fx;
  void* ux;
  sgdg_fn fv;
  void* uv;
} sgdg_product;

/* Batched time callback: out[i] = g(t[i]), i < npts.  Called on the host
 * when a strip's right-hand side is formed. */
typedef void (*sgdg_tfn)(int npts, const double* t, double* out, void* user);

/* One separable term coef * ft(t) * fx(x) * fv(v) of the source f; a NULL
 * function is the constant 1. */
typedef struct {
  double coef;
  sgdg_fn fx;
  void* ux;
  sgdg_fn fv;
  void* uv;
  sgdg_tfn ft;
  void* ut;
} sgdg_source;

/* beta_p = beta[p] for p < 2d (x-components first), sigma,
 * u0 = sum_k u0[k], the source f = sum_k f[k] (n_f may be 0) and the inflow
 * data g = sum_k g[k] on Gamma^- (n_g may be 0: g = 0).  Every component of
 * beta is ONE product (the tensor structure of Sect. 4.2); inflow splitting
 * (Sect. 5.2) assumes the sign of each factor changes only on mesh lines.
 * The strip right-hand side b_j of Sect. 2 pairs f with
 * w + delta (d_t w + beta . grad w) and takes -int_{I_j} <g, w>_{Gamma^-} dt,
 * <u, w>_Gamma = int_Gamma (beta . n) u w, split like the inflow term of the
 * operator; its time integrals use 3-point Gauss-Legendre on every strip.
 * Sources and inflow data are not combined with vlasov_poisson (EINVAL). */
typedef struct {
  sgdg_product beta[6];   /* 2d used; the rest are ignored */
  sgdg_product sigma;
  int n_u0;
  const sgdg_product* u0;
  int n_f;
  const sgdg_source* f;
  int n_g;
  const sgdg_source* g;
  /* Time factors (Sect. 4.2 lets beta and sigma depend on t inside the
   * tensor form): beta_p(t, x, v) = beta[p].coef * beta_t[p](t) * fx(x) *
   * fv(v), sigma likewise with sigma_t; a NULL factor is the constant 1.
   * With any time factor the strip operator is the quadrature sum of
   * Sect. 4.2 over time_quad Gauss-Legendre points per strip (0: 3 points;
   * at most 8): the Kronecker factors stay as assembled at create, the 2 x 2
   * time couplings are recomputed per strip (time callbacks on the host),
   * and the inflow part of each beta component follows the sign of its time
   * factor at every point.  Applies (operator, diagonal blocks, batch) use
   * the operator of the strip that starts at the handle's current time: 0
   * after sgdg_create and sgdg_set_initial, advanced by dt with every
   * sgdg_advance_strip, restored by sgdg_restore.  In the right-hand side
   * the streamline-diffusion part of a source and the inflow data carry the
   * time factor of the beta component they involve (inflow parts gated by
   * its sign), integrated by the 3-point Gauss rule of the sources.  Time
   * factors are not combined with vlasov_poisson (EINVAL). */
  sgdg_tfn beta_t[6];
  void* beta_ut[6];
  sgdg_tfn sigma_t;
  void* sigma_ut;
  int time_quad;
} sgdg_coeffs;

typedef struct {
  sgdg_mesh mesh_x, mesh_v;
  int level_L;          /* sparse level, 0-based, 0..11 */
  int time_degree;      /* r; must be 1 */
  double dt;            /* strip length */
  double delta;         /* streamline-diffusion parameter (> 0) */
  sgdg_precision precision;
  double rtol;          /* outer stop: ||b - A u||_2 <= rtol ||b||_2 */
  int max_outer;        /* outer iteration cap (FGMRES or Richardson steps) */
  int restart;          /* outer FGMRES restart length (<= 64) */
  int inner_its;        /* GMRES iterations per component solve (<= 64) */
  double inner_rtol;    /* early stop of a component solve */
  int cheb_steps;       /* Chebyshev-Jacobi steps per mass inverse */
  int device;           /* CUDA device ordinal */
  int vlasov_poisson;   /* 1: beta_v = -E(x) with E from a Poisson solve of the
                           density (Sect. 5.3); needs a periodic Omega_x and
                           beta[d+i] = {coef -1, fx = initial E_i, fv = NULL} */
  int outer_method;     /* sgdg_outer; 0 (zero-initialised): FGMRES */
  size_t hbm_budget_bytes; /* device memory the handle may hold (factors, state,
                              sweep and solver buffers); 0: no limit.  An
                              allocation that would pass it fails with
                              SGDG_ENOMEM (at create or on first use). */
} sgdg_config;

typedef struct {
  int L, d, R;                 /* R = r + 1 time coefficients */
  int n_grids;                 /* L + 1 */
  long long n_spatial;         /* sum_l n1(l) n2(L-l) */
  long long n_coeffs;          /* R * n_spatial: length of a strip vector */
  int n_terms;                 /* Kronecker terms after merging */
  int n_x_factors, n_v_factors;
  double device_bytes;         /* device memory held by the handle */
  long long nnz_x, nnz_v;      /* P1 pattern entries summed over the levels of each side */
  long long rows_x, rows_v;    /* pattern rows (vertices) summed over the levels of each side */
  int lattice_x_levels;        /* x levels held as 2-D structured lattices (slot-ordered rows) */
} sgdg_info;

typedef struct {
  int outer_its;
  int inner_its_total;
  int applies;                 /* full sparse-grid operator applies */
  double rel_residual;         /* true ||b - A u|| / ||b|| (FP64) */
  double initial_rel_residual; /* the same for the initial guess */
  double seconds;
  int status;
} sgdg_strip_stats;

/* Build the level hierarchies, assemble the finest-level factor matrices in
 * FP64 (Sect. 4.2), project them to every level with the embeddings
 * (X_l = E^T X_{l+1} E), compile the Kronecker term table of the block
 * formula (Sect. 4.2; delta on K~ per the weak form of Sect. 2), upload
 * everything to the device.  EINVAL for unsupported input (including a
 * coefficient function of beta, sigma or g that returns NaN or Inf at a
 * quadrature point or centroid; NaN in u0 or f is left to the solver's
 * SGDG_ENAN), ENOMEM, ECUDA. */
sgdg_status sgdg_create(const sgdg_config* cfg, const sgdg_coeffs* coeffs, void** out_handle);
/* The mesh checks of sgdg_create on one coarse mesh (host only, no device
 * call; the list is at sgdg_mesh): SGDG_OK or SGDG_EINVAL, with
 * sgdg_last_error(NULL) naming the failed check. */
sgdg_status sgdg_validate_mesh(const sgdg_mesh* mesh);

/* Host-only views of what sgdg_create builds from one coarse mesh, with no
 * handle and no device: the nested levels of Sect. 2 (uniform refinement up
 * to level L, vertices in the canonical order of the storage layout), the
 * embedding E_{l+1 <- l} of Sect. 4.2, and one Kronecker factor assembled in
 * FP64 on level L and carried to level l by the Galerkin projection
 * X_l = E^T X_{l+1} E (Sect. 4.2).  For checking the library's spaces and
 * factors against another implementation.  Errors: SGDG_EINVAL (mesh checks
 * of sgdg_validate_mesh, levels outside 0 <= l <= L < 12, a spec naming
 * no function of the side), with sgdg_last_error(NULL) saying why.
 *
 * A factor is X[i][j] = int w (D_trial phi_j)(D_test phi_i) over the domain
 * (kind 0) or over the boundary faces on one box side (kind 1: face_axis
 * 0-based, face_side -1 lower / +1 upper), D_0 = value and D_p = d/dy_p
 * (1-based axis p); w is the product of n_weight coefficient functions of
 * the side (ids 0 .. 5: the fx (side 0) or fv (side 1) factor of beta
 * component id, 6: of sigma, as given in the sgdg_coeffs); n_restrict
 * restrictions keep the cells (faces) whose centroid has sign(function) ==
 * sign.  Only the coefficient callbacks of the sgdg_coeffs are read. */
typedef struct {
  int kind;
  int test, trial;
  int n_weight;
  int weight[4];
  int n_restrict;
  int restrict_fn[2];
  int restrict_sign[2];
  int face_axis, face_side;
} sgdg_factor_spec;
/* Level `level` of the hierarchy refined to L: its vertex count and (coords
 * not NULL) its vertex coordinates [n][dim]. */
sgdg_status sgdg_inspect_level(const sgdg_mesh* mesh, int L, int level, int* n_vertices, double* coords);
/* E_{level+1 <- level} of the hierarchy refined to L (level < L) as CSR
 * (rows: level+1 vertices): *nrows and *nnz always; rowptr[nrows+1],
 * col[nnz], val[nnz] when all three are given (call once for the sizes). */
sgdg_status sgdg_inspect_embedding(const sgdg_mesh* mesh, int L, int level, int* nrows, int* nnz, int* rowptr,
                                   int* col, double* val);
/* The factor `spec` of side 0 (x) or 1 (v), assembled on level L and
 * projected to `level`, as CSR on that level's P1 pattern (square, rows =
 * test functions); sizes and arrays as for sgdg_inspect_embedding. */
sgdg_status sgdg_inspect_factor(const sgdg_mesh* mesh, const sgdg_coeffs* coeffs, int side, int L, int level,
                                const sgdg_factor_spec* spec, int* nrows, int* nnz, int* rowptr, int* col,
                                double* val);
/* The products of a factor with the transfers that the sweep applies
 * (Sect. 4.2, X_{l,l'} through E): which 0, R_level X_{level+1} = E^T X
 * (rows: level, columns: level + 1; level < L); which 1, X_level E_{level-1}
 * (rows: level, columns: level - 1; level >= 1).  Factor, sizes and arrays
 * as for sgdg_inspect_factor. */
sgdg_status sgdg_inspect_product(const sgdg_mesh* mesh, const sgdg_coeffs* coeffs, int side, int L, int level,
                                 const sgdg_factor_spec* spec, int which, int* nrows, int* nnz, int* rowptr,
                                 int* col, double* val);
/* The load vector F[i] = int (f_1 ... f_n)(y) D phi_i(y) dy of the n_fn
 * (0..4) functions fns (users: their user pointers, may be NULL; no
 * functions: f = 1), D = the value (deriv 0) or d/dy_deriv (1-based axis),
 * assembled on level L and restricted to `level` (E^T, Sect. 4.2) - the
 * spatial factors of the source terms of b_j (Sect. 2) as sgdg_create forms
 * them; out[n_vertices of level]. */
sgdg_status sgdg_inspect_load(const sgdg_mesh* mesh, int L, int level, int n_fn, const sgdg_fn* fns,
                              void* const* users, int deriv, double* out);
/* The Kronecker terms of A^(delta) (Sect. 4.2, the block formula) that
 * sgdg_create forms for these meshes and coefficients, with the time
 * couplings of the strip (t0, t0 + dt) (with time factors: the Gauss sum of
 * Sect. 4.2 over time_quad points; without: the exact time matrices, and t0
 * is ignored): *n_terms always; when tau, xspec and vspec are given and
 * capacity >= *n_terms, term k's coupling tau[4k + 2s + s'] (s the test
 * index, as in the block formula) and its x and v factors.  The operator's
 * full-grid form is sum_k tau_k (x) X_k (x) V_k with X_k, V_k from
 * sgdg_inspect_factor.  Only coefficient callbacks and time factors of the
 * sgdg_coeffs are read (u0, f, g are not). */
sgdg_status sgdg_inspect_terms(const sgdg_mesh* mesh_x, const sgdg_mesh* mesh_v, const sgdg_coeffs* coeffs,
                               double dt, double delta, double t0, int capacity, int* n_terms, double* tau,
                               sgdg_factor_spec* xspec, sgdg_factor_spec* vspec);
void sgdg_destroy(void* h);
const char* sgdg_last_error(const void* h);
sgdg_status sgdg_get_info(const void* h, sgdg_info* out);
/* Shape and element offset (in elements of a strip vector of any precision,
 * i.e. with the time index) of grid l = (l, L-l). */
sgdg_status sgdg_grid_shape(const void* h, int l, int* n1, int* n2, long long* offset);

/* y = A^(delta) u: the strip operator of Eq. 5 on the sparse grid,
 * [A u]_l = sum_l' A_{l,l'} u_l' (Sect. 4.2), evaluated by a linear-cost
 * sweep over the grids.  u, y: device arrays of n_coeffs elements of type
 * double (SGDG_FP64), float (SGDG_MIXED_FP32) or bfloat16 (SGDG_BF16_STORE);
 * y is overwritten; u and y must not overlap.  Any other precision:
 * SGDG_EINVAL. */
sgdg_status sgdg_apply_operator(void* h, const void* u, void* y, int precision, void* stream);
/* Same operator with host arrays (double): copies u to the device, rounds
 * it to the precision's element type there, applies, and copies y back as
 * double.  Synchronous; pinned host memory gives the full copy rate. */
sgdg_status sgdg_apply_operator_host(void* h, const double* u, double* y, int precision);
/* y = (Id_t (x) M_sg) u, the sparse-grid mass matrix on both time slots;
 * u, y as for sgdg_apply_operator. */
sgdg_status sgdg_apply_mass(void* h, const void* u, void* y, int precision, void* stream);
/* y = A_{l,l} u on one anisotropic full grid (l1, l2) with l1 + l2 in {L-1, L}
 * (the component systems of Eq. 22); arrays [n1][n2][2] of the precision's
 * element type on the device. */
sgdg_status sgdg_apply_diag(void* h, int l1, int l2, const void* u, void* y, int precision, void* stream);

/* The same y = A_{l,l} u as sgdg_apply_diag, from an entry point that
 * allocates nothing.  The paper has no counterpart: this exists for callers
 * that may not allocate device memory when they apply the operator - loops
 * that must not pay the allocator's device-wide synchronisation, processes
 * (plugins, embedded solvers) whose device memory belongs to a pool another
 * component owns.  Its scratch is a static
 * device array of SGDG_NOALLOC_SCRATCH_BYTES held by every GPU that loads the
 * library until the process exits; grids whose intermediates
 * (distinct v factors x n1 x n2 x 2 elements) do not fit are rejected with
 * SGDG_EINVAL and a message naming the size and the limit.  Every call looks
 * up the array's device address (a host query, so a device reset cannot leave
 * a stale address); the first call on a device also loads the library's
 * device code there, so make that first call before any stream capture.  All
 * calls share the array: calls that overlap on the GPU race.  u, y as for sgdg_apply_diag; precision SGDG_FP64 or
 * SGDG_MIXED_FP32 (others: SGDG_EINVAL). */
#define SGDG_NOALLOC_SCRATCH_BYTES (64u << 20)
sgdg_status sgdg_apply_diag_noalloc(void* h, int l1, int l2, const void* u, void* y, int precision,
                                    void* stream);
/* z = P_CT(r): Algorithm 1's preconditioner step (component solves with the
 * configured inner iterations, restriction of the residual, combination).
 * r, z: device arrays of n_coeffs doubles. */
sgdg_status sgdg_ct_precondition(void* h, const double* r, double* z, void* stream);

/* Checkpoint and restore at a strip boundary (the strip scheme of Sect. 2
 * carries only U^-_j from strip to strip; the file also holds what the
 * library's warm starts and the Vlasov-Poisson field need to continue
 * bit for bit).  sgdg_checkpoint writes, to the file at `path`: the strip
 * count j and start time t_j, U^-_j, the last strip solution u_j, the one
 * before it (extrapolated warm start), the next right-hand side, the
 * warm-start mode and guess, and for vlasov_poisson handles the field E per
 * finest cell with the density and potential; plus a 64-bit hash of the
 * discrete problem (meshes, levels, dt, delta, term table, finest-level
 * factor values at creation).  sgdg_restore reads such a file into a handle
 * created with the same problem (hash mismatch: SGDG_EINVAL) and replaces
 * its strip state; later sgdg_advance_strip calls then give the results an
 * uninterrupted run gives, bit for bit (the solver's reductions are
 * deterministic).  Both synchronise the device.  File errors: SGDG_EIO.
 * sgdg_checkpoint needs sgdg_set_initial first (else SGDG_EINVAL).  The
 * file ends with an FNV-1a 64 checksum of all bytes before it; sgdg_restore
 * reads and checks the whole file on the host first (magic, sizes against
 * the file length, checksum, nothing after it), so a truncated or corrupted
 * file returns SGDG_EIO and leaves the handle's state unchanged. */
sgdg_status sgdg_checkpoint(void* h, const char* path);
sgdg_status sgdg_restore(void* h, const char* path);

/* What a checkpoint file holds, read without a handle or a device. */
typedef struct {
  unsigned long long problem_hash;   /* identity of the discrete problem */
  long long n_coeffs, n_spatial;
  double t_now;                      /* start time of the next strip */
  int strips_solved;
  int has_field;                     /* 1: Vlasov-Poisson state included */
} sgdg_checkpoint_info;
/* The checks of sgdg_restore on the file at `path` alone (host only, no
 * device call): SGDG_OK and *info filled (info may be NULL) when the file
 * is a complete, uncorrupted checkpoint; SGDG_EIO otherwise; SGDG_EINVAL
 * for a NULL path. */
sgdg_status sgdg_checkpoint_verify(const char* path, sgdg_checkpoint_info* info);

/* U^-_0 := u0 (the first right-hand side uses (u0, w^+) directly). */
sgdg_status sgdg_set_initial(void* h);
/* Solve one strip (Eq. 5) with right-preconditioned FGMRES + CT (Algorithm 1
 * as preconditioner), starting from u = 0; advance U^-_j.  ENOCONV when
 * max_outer is reached (stats still filled). */
sgdg_status sgdg_advance_strip(void* h, void* stream, sgdg_strip_stats* stats);
/* Copy out the last strip solution u (n_coeffs doubles) or the end value
 * U^-_j (n_spatial doubles); dst is device (on_device=1) or host memory. */
sgdg_status sgdg_get_solution(const void* h, double* dst, int on_device);
sgdg_status sgdg_get_end_value(const void* h, double* dst, int on_device);
/* Unique representation of a spatial sparse-grid function: its values at the
 * nodes of every component grid (prolongation from coarser grids, injection
 * from finer ones).  u, out: device arrays of n_spatial doubles. */
sgdg_status sgdg_eval_nodal(void* h, const double* u, double* out, void* stream);

/* Vlasov-Poisson field update (Sect. 5.3: "-Delta phi = -int f dv + 1",
 * E = -grad phi; one update per strip, from U^-_{j-1}; midpoint rule).
 * Computes rho(x) = int U^- dv as a P1 function on the finest level of
 * Omega_x (rho of u0 before the first strip), solves the periodic P1 Poisson
 * problem (mean of the source removed, phi of zero mean) by CG in FP64,
 * takes E = -grad phi per finest cell, re-assembles every x factor that
 * depends on E (finest level + Galerkin projection) and uploads it.
 * source 0: rho from the end value of the last strip (u0 before the first
 * strip); source 1: rho from the last strip solution at the strip midpoint
 * (the fixed point of Sect. 5.3, with sgdg_resolve_strip).
 * field_energy (may be NULL): 1/2 int |E|^2 dx of the new field.  Only for
 * handles created with vlasov_poisson = 1 (else EINVAL). */
sgdg_status sgdg_field_update(void* h, int source, double* field_energy);
/* A field given by the caller instead of the Poisson solve (Sect. 5.3 with
 * E from elsewhere, e.g. an external field solver): E[k * n_cells + e] is
 * component k (< d) of E on cell e of the finest level of Omega_x, in the
 * order of sgdg_get_field, n_cells the count sgdg_finest_x reports (host
 * array, copied).  Re-assembles every x factor that depends on E, like
 * sgdg_field_update; later strips use it until the next field update.
 * sgdg_get_field copies the current field out (host array of d n_cells).
 * Only for vlasov_poisson handles; a wrong n_cells or a NaN/Inf value:
 * SGDG_EINVAL. */
sgdg_status sgdg_set_field(void* h, const double* E, int n_cells);
sgdg_status sgdg_get_field(const void* h, double* E, int n_cells);
/* Re-solve the last strip with the current coefficients (same right-hand
 * side), starting from its last solution; replaces the solution and the end
 * value.  One step of the per-strip fixed point of Sect. 5.3. */
sgdg_status sgdg_resolve_strip(void* h, void* stream, sgdg_strip_stats* stats);
/* One strip of the Vlasov-Poisson system with the field iterated to
 * consistency (Sect. 5.3 iterates E and f within a strip): the field from
 * U^-_{j-1} (sgdg_field_update source 0), a strip solve, then up to max_fp
 * times: the field from the strip solution at the midpoint (source 1) and,
 * while the potential changed by more than tol (relative l2 against the
 * previous field), a re-solve of the strip with it.  stats: the last solve;
 * fp_steps: the re-solves made; phi_change: the last relative change (may be
 * NULL).  Handles without vlasov_poisson, tol < 0 or max_fp < 0: SGDG_EINVAL;
 * SGDG_ENOCONV when a solve hits max_outer. */
sgdg_status sgdg_advance_strip_vp(void* h, void* stream, double tol, int max_fp, sgdg_strip_stats* stats,
                                  int* fp_steps, double* phi_change);
/* Stop test of sgdg_advance_strip_vp's fixed point: 0 (default) the relative
 * l2 change of the potential phi between field updates; 1 the test of
 * Sect. 5.3, ||E^(k+1) - E^(k)||_{L^inf(I_j x Omega_x)} +
 * ||f^(k+1) - f^(k)||_{H^1(I_j x Omega)}, with f^(0) = U^-_{j-1} constant in
 * time on the strip and E constant in time on the strip (midpoint rule);
 * phi_change then reports that sum.  Other values: SGDG_EINVAL. */
sgdg_status sgdg_set_vp_stop(void* h, int criterion);
/* *out = ||U||_{H^1(I_j x Omega)}, the norm of Algorithm 1's stop test
 * (Sect. 4.3): int_{I_j} ||U||^2 + ||d_t U||^2 + ||grad_x U||^2 +
 * ||grad_v U||^2 dt for the strip function with coefficients u (device
 * array of n_coeffs doubles), from the Gram form applied blockwise in FP64.
 * Synchronises `stream`. */
sgdg_status sgdg_h1_norm(void* h, const double* u, double* out, void* stream);
/* Initial guess of the next sgdg_advance_strip: 0 zero (default), 1 the
 * previous strip's solution, 2 the array last given to sgdg_set_guess, 3 the
 * linear extrapolation 2 u_{j-1} - u_{j-2} of the last two strip solutions
 * (the previous solution while fewer than two strips are solved). */
sgdg_status sgdg_set_warm_start(void* h, int mode);
/* dst (device, n_coeffs doubles) = the mode-3 guess for the next strip. */
sgdg_status sgdg_extrapolated_guess(const void* h, double* dst);
/* Copy an initial guess (device array of n_coeffs doubles) for warm-start mode 2. */
sgdg_status sgdg_set_guess(void* h, const double* u);
/* Number of vertices / cells of the finest level of Omega_x. */
sgdg_status sgdg_finest_x(const void* h, int* n_vertices, int* n_cells);
/* Last computed density rho and potential phi at the finest x vertices
 * (lexicographic order), host arrays of n_vertices doubles. */
sgdg_status sgdg_get_density_potential(const void* h, double* rho, double* phi);

/* Learned warm start (no counterpart in the paper: an extension of the solver).
 *
 * sgdg_coarse_values: the values of a sparse-grid function at the nodes of
 * the full grid (lx, lv): u is a strip vector (R = 2) or a spatial vector
 * (R = 1); out [n_x(lx)][n_v(lv)][R] on the device.  Finer component grids are
 * injected, coarser ones prolonged (unique, unlike the coefficients).
 * sgdg_coarse_diff: out = the same view of a - b (both strip vectors for
 * R = 2, spatial for R = 1); the warm start's features and targets.
 * sgdg_add_coarse: adds the P1 function c ([n_x(lx)][n_v(lv)][2], device) to
 * the strip vector u, represented on component grid (lx, L-lx) by
 * prolongation in v; needs lv <= L - lx. */
sgdg_status sgdg_coarse_values(void* h, const double* u, int R, int lx, int lv, double* out, void* stream);
sgdg_status sgdg_coarse_diff(void* h, const double* a, const double* b, int R, int lx, int lv, double* out,
                             void* stream);
sgdg_status sgdg_add_coarse(void* h, const double* c, int lx, int lv, double* u, void* stream);

/* A 3-layer MLP y = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3 trained and
 * evaluated by the library's own BF16 tensor-core GEMMs (FP32 accumulation,
 * FP32 master weights, Adam).  Sizes must be multiples of 16; batches are
 * row-major [batch][n] FP64 device arrays (scaled by in_scale / out_scale
 * inside); at most max_batch rows.  Loss: 1/(2 batch) sum (y - t)^2. */
sgdg_status sgdg_mlp_create(int n_in, int width, int n_out, int max_batch, unsigned long long seed, void** mlp);
void sgdg_mlp_destroy(void* mlp);
sgdg_status sgdg_mlp_set_scaling(void* mlp, double in_scale, double out_scale);
sgdg_status sgdg_mlp_forward(void* mlp, const double* x, int batch, double* y, void* stream);
sgdg_status sgdg_mlp_train_step(void* mlp, const double* x, const double* t, int batch, double lr, double* loss,
                                void* stream);
/* Gradients of the loss (host, layout W1, b1, W2, b2, W3, b3 with W_k
 * [fan_in][fan_out]) without an update; loss to *loss. */
sgdg_status sgdg_mlp_gradients(void* mlp, const double* x, const double* t, int batch, float* grads, double* loss);
long long sgdg_mlp_num_params(const void* mlp);
sgdg_status sgdg_mlp_get_params(const void* mlp, float* params);
sgdg_status sgdg_mlp_set_params(void* mlp, const float* params);

/* Autotuner (no counterpart in the paper): times candidate launch shapes
 * (rows per thread in {1,2,4,8} x row-major or column-tiled block order x one
 * or two outputs per thread x with or without L2 prefetch hints) of
 * every sweep launch site on live applies y = A u (device arrays as for
 * sgdg_apply_operator, overwritten) and keeps the fastest per site for all
 * later applies of this handle. */
sgdg_status sgdg_autotune(void* h, const void* u, void* y, int precision, void* stream);
/* Which kernels run the sweep's branch A (no counterpart in the paper; both
 * compute the same operator with the same FP32/FP64 sums, bit for bit; in BF16
 * storage the fused kernel keeps S_b in FP32):
 * 0: one fused launch per grid where a tile plan fits - the states
 *   S_b = U V_b^T + P1 Z_b are formed per tile in shared memory, folded into
 *   y and restricted there, and never written to device memory (about a
 *   tenth of the unfused DRAM traffic, but slower on GB300: the kernels are
 *   bound by L1/shared-memory throughput and latency, and the tiles cost
 *   occupancy, barriers and halo recomputation);
 * 1 (default): the unfused kernels (S_b written per grid, then final update
 *   and restriction); on x levels that are 2-D structured lattices (cells
 *   cut along the (1, 1) diagonal) the autotuner may also pick lattice
 *   kernels for the final update along dim 1 and the mode-A chain step
 *   (runs along the lattice rows with register windows);
 * 2: the unfused generic kernels only (the same sums).  Other values:
 *   SGDG_EINVAL. */
sgdg_status sgdg_set_sweep_variant(void* h, int variant);
/* The fused branch-A plan of grid l for S pairs of pair_bytes bytes in shared
 * memory (FP32 and BF16 storage: 8; FP64: 16), built if needed (measurement; no counterpart in the paper): iout[0..3] = tiles,
 * chains per group, ELL width, shared-memory bytes per block; dout[0..1] =
 * S_b entries formed per chain (interior and halo), restricted outputs per
 * chain.  All zero when no tile shape fits (the unfused kernels run). */
sgdg_status sgdg_fused_plan_info(void* h, int l, int pair_bytes, int* iout, double* dout);
/* Copies the autotuner's per-site choices of `src` into `dst` (sites are keyed
 * by kernel kind, grid shape, chain count and element size, so handles of the
 * same problem size share them; sites `dst` never meets are ignored) and
 * clears any pinned shape of `dst`.  Host only. */
sgdg_status sgdg_copy_tuning(void* dst, const void* src);
/* Pins every sweep launch site of later applies to one launch shape,
 * code = rows per thread (1..15) | block order << 4 (0 row-major, 1 column
 * tiles) | two outputs per thread (final kernels, short-row chain steps) << 5
 * | L2 prefetch hints for operands a step ahead (final and chain kernels)
 * << 6 | the lattice kernels where a level allows them (runs of 4 or 8
 * vertices for the final, 2 or 4 for the chain step, from the rows per
 * thread) << 7; code 0 returns to the tuned or default shapes (sgdg_autotune also
 * clears the pin).  For tests and measurements: a shape changes the thread
 * mapping and the prefetching, never the values.  Other codes: SGDG_EINVAL. */
sgdg_status sgdg_set_launch_shape(void* h, int code);

/* Batches of independent problems (many instances of uneven L, Sect. 5's
 * experiments run one after another; here they share the GPU).  A batch
 * references n >= 1 member handles (not owned; they must outlive it). */
sgdg_status sgdg_batch_create(int n, void* const* members, void** out_batch);
void sgdg_batch_destroy(void* batch);
/* y_k = A_k u_k for every member k (u, y: arrays of n device pointers, the
 * precision's element type).  The whole batch is one CUDA graph: captured on
 * the first call for a given pointer set and precision, replayed on `stream`
 * afterwards.  The first call also runs one eager apply per member. */
sgdg_status sgdg_batch_apply(void* batch, const void* const* u, void* const* y, int precision, void* stream);
/* Advance every member by one strip, members concurrently (one stream and one
 * host thread each).  per_member: n stats (may be NULL).  Returns the first
 * non-OK member status. */
sgdg_status sgdg_batch_advance(void* batch, sgdg_strip_stats* per_member);

/* Kernel accounting (measurement; no counterpart in the paper).  Kinds:
 * 0 = per-grid states S_b = u V_b^T (+ P1 Z_b) of the sweep's branch A and of
 *     the diagonal blocks, 1 = final updates y (+)= tau X S_b along dim 1,
 * 2 / 3 = restriction of sweep chain states along dim 1 / dim 2,
 * 4 = fused branch-A launches (S_b per tile in shared memory, final update
 *     and restriction in one kernel), 5 = sweep chain steps of branch B,
 * 6 = reserved (no launches),
 * 7 = final updates of branch B along dim 2.
 * n_kinds must be >= 8. */
typedef struct {
  long long launches;
  double ms;        /* summed CUDA-event duration of the launches */
  double bytes;     /* summed algorithmic bytes: inputs + outputs (read and
                       written when accumulating) + matrix rows (ELL columns
                       and values) */
  double flops;     /* summed floating-point operations executed: 2 per
                       multiply-add, padded ELL entries included */
} sgdg_kernel_stat;
/* enable != 0: bracket every subsequent SpMM launch with CUDA events and
 * record its algorithmic bytes (clears earlier records); 0: stop. */
sgdg_status sgdg_profile(void* h, int enable);
/* Synchronise the device, fill out[0..7] (one per kind) and clear the records. */
sgdg_status sgdg_kernel_stats(void* h, sgdg_kernel_stat* out, int n_kinds);
/* Sizes in bytes of the ABI structs, for bindings to check their layouts
 * (host only; no device is touched): out[0..8] = sgdg_mesh, sgdg_product,
 * sgdg_source, sgdg_coeffs, sgdg_config, sgdg_info, sgdg_strip_stats,
 * sgdg_kernel_stat, sgdg_checkpoint_info, sgdg_factor_spec.  Writes
 * min(n, 10) entries and returns 10. */
int sgdg_struct_sizes(int* out, int n);
/* Number of SpMM kernels this handle has launched so far. */
long long sgdg_launch_count(const void* h);
/* Measured multiply-add peak of device `device` (measurement; no counterpart
 * in the paper): a register-only kernel runs 8 independent multiply-add
 * chains per thread, `iters` steps each, on every SM (as many 256-thread
 * blocks as fit), timed with CUDA events, best of 3 after a warm-up.
 * precision SGDG_MIXED_FP32 (FP32 FFMA) or SGDG_FP64 (DFMA); others EINVAL.
 * gflops: 2 flops per multiply-add / the best time; ms (may be NULL): that
 * time.  Allocates one small device buffer and frees it. */
sgdg_status sgdg_alu_peak(int device, int precision, int iters, double* gflops, double* ms);

#ifdef __cplusplus
}
#endif
#endif /* SGDG_H */
