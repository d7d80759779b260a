/* A C99 caller of the library: compiles against include/sgdg.h alone (no C++,
 * no CUDA headers), links libsgdg.so and prints, for each ABI struct, the size
 * this C compiler gives it next to the size the library was built with
 * (sgdg_struct_sizes).  It then calls the host-only entry points from C on a
 * 4-cell interval mesh (mesh check, levels, embedding, a factor with a C
 * coefficient callback) and checks what they return.  It calls no entry
 * point that touches a device. */
#include <stdio.h>
#include <math.h>
#include <stddef.h>
#include <string.h>

#include "sgdg.h"

/* beta's v factor: v itself */
static void vfun(int n, const double* pts, double* out, void* user) {
  (void)user;
  for (int i = 0; i < n; ++i) out[i] = pts[i];
}

/* Host-only calls from C on the interval [0, 1] with 4 cells; 0 when every
 * result is as expected. */
static int host_calls(void) {
  const double coords[5] = {0.0, 0.25, 0.5, 0.75, 1.0};
  const int cells[8] = {0, 1, 1, 2, 2, 3, 3, 4};
  const double lo[1] = {0.0}, hi[1] = {1.0};
  const int periodic[1] = {0};
  sgdg_mesh m = {1, 5, coords, 4, cells, lo, hi, periodic};
  int bad = 0, n = 0, nrows = 0, nnz = 0;
  bad |= sgdg_validate_mesh(&m) != SGDG_OK;
  /* refinement doubles the cells: 5, 9, 17 vertices */
  for (int l = 0; l <= 2; ++l) {
    bad |= sgdg_inspect_level(&m, 2, l, &n, NULL) != SGDG_OK;
    bad |= n != (4 << l) + 1;
  }
  /* E_{1 <- 0}: 9 rows; 5 copies and 4 midpoints of two entries */
  bad |= sgdg_inspect_embedding(&m, 2, 0, &nrows, &nnz, NULL, NULL, NULL) != SGDG_OK;
  bad |= nrows != 9 || nnz != 13;
  /* the mass on level 0 (h = 1/4): diagonal 2h/3 inside, h/3 at the ends,
   * off-diagonal h/6, total 1; the weighted factor int v phi_j phi_i on
   * level 0 sums to int v = 1/2 */
  sgdg_coeffs c;
  memset(&c, 0, sizeof(c));
  c.beta[0].coef = 1.0;
  c.beta[0].fv = vfun;
  sgdg_factor_spec spec;
  memset(&spec, 0, sizeof(spec));
  int rowptr[6], col[13];
  double val[13];
  bad |= sgdg_inspect_factor(&m, &c, 1, 2, 0, &spec, &nrows, &nnz, rowptr, col, val) != SGDG_OK;
  bad |= nrows != 5 || nnz != 13;
  double sum = 0.0, diag1 = 0.0;
  for (int r = 0; r < nrows; ++r)
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      sum += val[p];
      if (r == 1 && col[p] == 1) diag1 = val[p];
    }
  bad |= fabs(sum - 1.0) > 1e-15 || fabs(diag1 - 0.5 / 3.0) > 1e-15;
  spec.n_weight = 1;
  spec.weight[0] = 0;
  bad |= sgdg_inspect_factor(&m, &c, 1, 2, 0, &spec, &nrows, &nnz, rowptr, col, val) != SGDG_OK;
  sum = 0.0;
  for (int p = 0; p < nnz; ++p) sum += val[p];
  bad |= fabs(sum - 0.5) > 1e-14;
  /* a mesh with a hole is refused */
  sgdg_mesh holed = {1, 5, coords, 3, cells, lo, hi, periodic};
  bad |= sgdg_validate_mesh(&holed) != SGDG_EINVAL;
  printf("host calls %s\n", bad ? "FAILED" : "ok");
  return bad;
}

int main(void) {
  const int c_sizes[10] = {(int)sizeof(sgdg_mesh),   (int)sizeof(sgdg_product), (int)sizeof(sgdg_source),
                           (int)sizeof(sgdg_coeffs), (int)sizeof(sgdg_config),  (int)sizeof(sgdg_info),
                           (int)sizeof(sgdg_strip_stats), (int)sizeof(sgdg_kernel_stat),
                           (int)sizeof(sgdg_checkpoint_info), (int)sizeof(sgdg_factor_spec)};
  int lib_sizes[10] = {0};
  const int n = sgdg_struct_sizes(lib_sizes, 10);
  int bad = n != 10;
  for (int i = 0; i < 10; ++i) {
    printf("%d %d %d\n", i, c_sizes[i], lib_sizes[i]);
    bad |= c_sizes[i] != lib_sizes[i];
  }
  /* offsets a C caller relies on: the fields after the ones added over time */
  printf("offset time_quad %d\n", (int)offsetof(sgdg_coeffs, time_quad));
  printf("offset hbm_budget_bytes %d\n", (int)offsetof(sgdg_config, hbm_budget_bytes));
  printf("offset lattice_x_levels %d\n", (int)offsetof(sgdg_info, lattice_x_levels));
  bad |= host_calls();
  return bad;
}
