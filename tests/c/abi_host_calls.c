/* A C program against include/vplbm.h and libvplbm.so, using only the calls
 * that need no GPU: configuration defaults, the relaxation time from the
 * Reynolds number, footprints, and the refusal of invalid configurations
 * (including a device memory hook with only one of its two functions), of a
 * NULL handle by every call that takes one, and of bad arguments to the
 * grouped and the allocation-free step.
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
  if (strstr(vplbm_create_error(), "tau") == NULL) return fail("creation error names tau");
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

  /* every call that takes a handle refuses NULL with a status (nothing crosses the ABI) */
  {
    double d[4] = {0, 0, 0, 0};
    int64_t cnt = 0;
    uint8_t chi[4] = {0, 0, 0, 0};
    char buf[64];
    vplbm_body body;
    memset(&body, 0, sizeof(body));
    const vplbm_status inv = VPLBM_ERR_INVALID;
    if (vplbm_set_initial_velocity(NULL, d) != inv ||
        vplbm_set_initial_perturbation(NULL, 0.0, 0.0, 0.0, 1) != inv ||
        vplbm_set_mask_and_solid_velocity(NULL, chi, NULL, 0) != inv ||
        vplbm_set_bodies(NULL, &body, 1) != inv || vplbm_step(NULL, 1) != inv ||
        vplbm_synchronize(NULL) != inv || vplbm_moments(NULL, d, d, d, 0) != inv ||
        vplbm_populations(NULL, d, 0) != inv || vplbm_set_populations(NULL, d, 0) != inv ||
        vplbm_mask(NULL, chi) != inv || vplbm_forces(NULL, d, d, d, 1, &cnt) != inv ||
        vplbm_forces_async(NULL, d, 1, &cnt) != inv ||
        vplbm_save_state(NULL, buf, sizeof(buf)) != inv ||
        vplbm_load_state(NULL, buf, sizeof(buf)) != inv || vplbm_momentum_exchange(NULL, d, d) != inv ||
        vplbm_enable_momentum_exchange(NULL, 1) != inv ||
        vplbm_momentum_exchange_forces(NULL, d, d, 1, &cnt) != inv ||
        vplbm_enable_timing(NULL, 1) != inv || vplbm_fused_timing(NULL, d, &cnt) != inv)
      return fail("NULL handle refused by every call");
    if (vplbm_state_bytes(NULL) != 0 || strcmp(vplbm_last_error(NULL), "no solver") != 0)
      return fail("NULL handle: state size and message");
    vplbm_solver* none[2] = {NULL, NULL};
    const int64_t steps[2] = {1, 1};
    if (vplbm_group_step(none, 2, steps) != inv || vplbm_group_step(NULL, 2, steps) != inv ||
        vplbm_group_step(none, -1, steps) != inv || vplbm_group_step(none, 0, steps) != VPLBM_OK)
      return fail("group step arguments");
  }

  /* the allocation-free step refuses bad arguments before any device work */
  {
    vplbm_config n;
    vplbm_config_init(&n);
    n.nx = 64;
    n.ny = 32;
    double rec[3];
    float* fa = (float*)16; /* never dereferenced: every call below is refused first */
    float* fb = (float*)32;
    const uint8_t* mk = (const uint8_t*)48;
    if (vplbm_step_noalloc(&n, NULL, 0, NULL, fb, mk, NULL, 64, 0, rec, NULL) != VPLBM_ERR_INVALID ||
        vplbm_step_noalloc(&n, NULL, 0, fa, fa, mk, NULL, 64, 0, rec, NULL) != VPLBM_ERR_INVALID ||
        vplbm_step_noalloc(&n, NULL, 0, fa, fb, mk, NULL, 60, 0, rec, NULL) != VPLBM_ERR_INVALID ||
        vplbm_step_noalloc(&n, NULL, 0, fa, fb, mk, NULL, 64, -1, rec, NULL) != VPLBM_ERR_INVALID ||
        vplbm_step_noalloc(&n, NULL, 1, fa, fb, mk, NULL, 64, 0, rec, NULL) != VPLBM_ERR_INVALID)
      return fail("allocation-free step arguments");
    n.streaming = VPLBM_STREAM_AA;
    if (vplbm_step_noalloc(&n, NULL, 0, fa, fb, mk, NULL, 64, 0, rec, NULL) != VPLBM_ERR_INVALID)
      return fail("allocation-free step refuses in-place streaming");
    n.streaming = VPLBM_STREAM_AB;
    n.bc_x = VPLBM_BC_INLET_CONVECTIVE;
    n.bc_y = VPLBM_BC_FREE_SLIP;
    n.u_conv = 0.05;
    if (vplbm_step_noalloc(&n, NULL, 0, fa, fb, mk, NULL, 64, 0, rec, NULL) != VPLBM_ERR_INVALID)
      return fail("allocation-free step refuses the convective outlet");
  }
  if (strcmp(vplbm_status_string(VPLBM_ERR_DIVERGED), "diverged") != 0) return fail("status string");
  vplbm_destroy(NULL);
  printf("ok\n");
  return 0;
}
