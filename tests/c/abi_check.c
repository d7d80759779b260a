/* A C99 caller of the library: compiles against include/sgdg.h alone (no C++,
 * no CUDA headers), links libsgdg.so and prints, for each ABI struct, the size
 * this C compiler gives it next to the size the library was built with
 * (sgdg_struct_sizes).  It calls no entry point that touches a device. */
#include <stdio.h>
#include <stddef.h>

#include "sgdg.h"

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
  return bad;
}
