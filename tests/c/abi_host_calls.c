/* A C program against include/vplbm.h and libvplbm.so, using only the calls
 * that need no GPU: configuration defaults, the relaxation time from the
 * Reynolds number, footprints, and the refusal of invalid configurations
 * (including a device memory hook with only one of its two functions).
 * Prints one line per check and exits non-zero on the first failure. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "vplbm.h"

static int alloc_calls = 0;
static void* host_only_alloc(size_t bytes, void* ctx) {
  (void)bytes;
  (void)ctx;
  ++alloc_calls;
  return NULL;
}

static int fail(const char* what) {
  printf("FAIL %s\n", what);
  return 1;
}

int main(void) {
  vplbm_config c;
  vplbm_config_init(&c);
  if (c.collision != VPLBM_SRT || c.storage != VPLBM_F32 || c.bc_x != VPLBM_BC_PERIODIC ||
      c.streaming != VPLBM_STREAM_AB || c.rounding != VPLBM_ROUND_STOCHASTIC || c.nx != 0)
    return fail("config defaults");
  if (fabs(vplbm_tau_from_reynolds(0.05, 40.0, 100.0) - 0.56) > 1e-12) return fail("tau from Re");

  c.nx = 1024;
  c.ny = 256;
  c.collision = VPLBM_MRT;
  const size_t ab = vplbm_footprint_bytes(&c);
  c.streaming = VPLBM_STREAM_AA;
  const size_t aa = vplbm_footprint_bytes(&c);
  if (ab < 2u * 9u * 1024u * 256u * 4u || aa >= ab || ab - aa != 9u * 1024u * 256u * 4u)
    return fail("footprints");
  c.storage = VPLBM_F16_OFFSET;
  if (vplbm_footprint_bytes(&c) >= aa) return fail("16-bit footprint");

  /* invalid configurations are refused before any device work */
  vplbm_solver* s = (vplbm_solver*)1;
  c.tau = 0.5;
  if (vplbm_create(&c, &s) != VPLBM_ERR_INVALID || s != NULL) return fail("tau = 1/2 refused");
  vplbm_config_init(&c);
  c.nx = 64;
  c.ny = 32;
  c.bc_x = VPLBM_BC_INLET_CONVECTIVE;
  c.bc_y = VPLBM_BC_FREE_SLIP;
  c.u_conv = -1.0;
  if (vplbm_create(&c, &s) != VPLBM_ERR_INVALID) return fail("negative u_conv refused");
  c.u_conv = 0.05;
  c.streaming = 7;
  if (vplbm_create(&c, &s) != VPLBM_ERR_INVALID) return fail("unknown streaming refused");
  if (vplbm_create(NULL, &s) != VPLBM_ERR_INVALID) return fail("NULL config refused");
  /* the device memory hook: unset by default; one function without the other is refused */
  vplbm_config_init(&c);
  if (c.dev_alloc != NULL || c.dev_free != NULL || c.alloc_ctx != NULL) return fail("hook default");
  c.nx = 64;
  c.ny = 32;
  c.dev_alloc = host_only_alloc;
  if (vplbm_footprint_bytes(&c) != 0) return fail("half-set hook: no footprint");
  if (vplbm_create(&c, &s) != VPLBM_ERR_INVALID || s != NULL) return fail("half-set hook refused");
  if (alloc_calls != 0) return fail("refused before any allocation");
  if (vplbm_step_count(NULL) != -1 || vplbm_launch_count(NULL) != -1) return fail("NULL handle");
  if (strcmp(vplbm_status_string(VPLBM_ERR_DIVERGED), "diverged") != 0) return fail("status string");
  vplbm_destroy(NULL);
  printf("ok\n");
  return 0;
}
