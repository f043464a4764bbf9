/* Prints the layout of the structs include/vplbm.h passes by pointer, one
 * line per field ("struct field offset size") plus "struct sizeof N", so a
 * test can compare the Python binding's ctypes structures with what a C
 * compiler makes of the header. */
#include <stddef.h>
#include <stdio.h>

#include "vplbm.h"

#define FIELD(S, F) printf(#S " " #F " %zu %zu\n", offsetof(S, F), sizeof(((S*)0)->F))

int main(void) {
  FIELD(vplbm_body, cx);
  FIELD(vplbm_body, cy);
  FIELD(vplbm_body, radius);
  FIELD(vplbm_body, amp_x);
  FIELD(vplbm_body, amp_y);
  FIELD(vplbm_body, period);
  FIELD(vplbm_body, omega);
  FIELD(vplbm_body, outside);
  FIELD(vplbm_body, reserved);
  printf("vplbm_body sizeof %zu\n", sizeof(vplbm_body));
  FIELD(vplbm_config, nx);
  FIELD(vplbm_config, ny);
  FIELD(vplbm_config, collision);
  FIELD(vplbm_config, storage);
  FIELD(vplbm_config, bc_x);
  FIELD(vplbm_config, bc_y);
  FIELD(vplbm_config, use_rates);
  FIELD(vplbm_config, reduce_mass);
  FIELD(vplbm_config, tau);
  FIELD(vplbm_config, lambda);
  FIELD(vplbm_config, eta);
  FIELD(vplbm_config, u_in);
  FIELD(vplbm_config, rho0);
  FIELD(vplbm_config, u0);
  FIELD(vplbm_config, body_force);
  FIELD(vplbm_config, rates);
  FIELD(vplbm_config, force_ring_len);
  FIELD(vplbm_config, rounding);
  FIELD(vplbm_config, stream);
  FIELD(vplbm_config, u_conv);
  FIELD(vplbm_config, streaming);
  FIELD(vplbm_config, tile_rows);
  FIELD(vplbm_config, dev_alloc);
  FIELD(vplbm_config, dev_free);
  FIELD(vplbm_config, alloc_ctx);
  FIELD(vplbm_config, rounding_seed);
  FIELD(vplbm_config, reserved);
  printf("vplbm_config sizeof %zu\n", sizeof(vplbm_config));
  return 0;
}
