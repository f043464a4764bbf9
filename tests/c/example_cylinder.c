/* The C ABI end to end: a cylinder in a channel at Re = 100 (uniform inlet,
 * zero-gradient outlet, free-slip walls), MRT with FP32 storage, stepped on
 * the GPU; prints the mean drag coefficient of the second half of the run.
 * Usage: cylinder [nx ny diameter steps] (default 1024 256 40 20000). The CPU
 * tests build it against the header; a GPU test runs it on a small case and
 * compares its drag with the FP64 oracle's.
 *   gcc -std=c11 -I include tests/c/example_cylinder.c \
 *       -L paper_1812_05401_gb300 -lvplbm -Wl,-rpath,paper_1812_05401_gb300 -o cylinder
 */
#include <stdio.h>
#include <stdlib.h>

#include "vplbm.h"

static int check(vplbm_status st, const vplbm_solver* s, const char* what) {
  if (st == VPLBM_OK) return 0;
  fprintf(stderr, "%s: %s (%s)\n", what, vplbm_status_string(st),
          s ? vplbm_last_error(s) : vplbm_create_error());
  return 1;
}

int main(int argc, char** argv) {
  int nx = 1024, ny = 256, steps = 20000;
  double d = 40.0;
  const double u = 0.05, re = 100.0;
  if (argc == 5) {
    nx = atoi(argv[1]);
    ny = atoi(argv[2]);
    d = atof(argv[3]);
    steps = atoi(argv[4]);
  } else if (argc != 1) {
    fprintf(stderr, "usage: %s [nx ny diameter steps]\n", argv[0]);
    return 2;
  }
  if (nx < 1 || ny < 1 || steps < 2 || !(d > 0.0)) {
    fprintf(stderr, "need nx, ny >= 1, steps >= 2 and a positive diameter\n");
    return 2;
  }

  vplbm_config cfg;
  vplbm_config_init(&cfg);
  cfg.nx = nx;
  cfg.ny = ny;
  cfg.collision = VPLBM_MRT;
  cfg.storage = VPLBM_F32;
  cfg.bc_x = VPLBM_BC_INLET_OUTLET;
  cfg.bc_y = VPLBM_BC_FREE_SLIP;
  cfg.u_in[0] = u;
  cfg.u0[0] = u;
  cfg.tau = vplbm_tau_from_reynolds(u, d, re); /* nu = U D / Re, tau = 3 nu + 1/2 */
  cfg.force_ring_len = steps;

  vplbm_solver* s = NULL;
  if (check(vplbm_create(&cfg, &s), NULL, "vplbm_create")) return 1;

  vplbm_body cylinder = {0};
  cylinder.cx = nx / 4.0;
  cylinder.cy = (ny - 1) / 2.0;
  cylinder.radius = d / 2.0;
  if (check(vplbm_set_bodies(s, &cylinder, 1), s, "vplbm_set_bodies") ||
      check(vplbm_set_initial_perturbation(s, u, 0.0, 1e-4, 1), s, "perturbation") ||
      check(vplbm_step(s, steps), s, "vplbm_step")) {
    vplbm_destroy(s);
    return 1;
  }

  double* fx = malloc(sizeof(double) * steps);
  double* fy = malloc(sizeof(double) * steps);
  int64_t n = 0;
  int rc = 1;
  if (fx && fy && !check(vplbm_forces(s, fx, fy, NULL, steps, &n), s, "vplbm_forces")) {
    double sum = 0.0;
    for (int64_t k = n / 2; k < n; ++k) sum += fx[k];
    const double cd = sum / (double)(n - n / 2) / (0.5 * u * u * d); /* rho_ref = 1 */
    printf("mean C_D over steps %lld..%lld: %.9f\n", (long long)(n / 2), (long long)n, cd);
    rc = 0;
  }
  free(fx);
  free(fy);
  vplbm_destroy(s);
  return rc;
}
