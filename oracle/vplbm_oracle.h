/*
 * Plain FP64 CPU oracle of the volume-penalization lattice Boltzmann (VP-LBM)
 * time step (Benamour, Liberge, Beghein, arXiv 1812.05401).
 *
 * TEST INFRASTRUCTURE ONLY. This oracle is what the CUDA path is checked
 * against. Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load or call it; the product path never does. It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Pins (tests/test_oracle_pins.py): every function is checked against what
 * the paper and the mathematics fix (printed constants, exact rational
 * single-node collisions, invariants, closed forms, symmetries, limits).
 * Parity unpinned: the magnitude of the curved-wall (staircase) error, which
 * the paper gives only in figures (Section 3.2). It is pinned as nonzero and
 * falling with refinement, and the 128 x 128 circular Couette value is
 * locked as a regression of this oracle.
 *
 * Layout: populations f[alpha][y][x], alpha = 0..8, row length nx, no padding.
 * Node (i, j) sits at the point (x, y) = (i, j); lattice spacing and time step
 * are 1 (Section 2.1.1, after Eq. vecteurs_D2Q9).
 */
#ifndef VPLBM_ORACLE_H
#define VPLBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SRT = 0, ORC_MRT = 1 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_INLET_OUTLET = 1, ORC_BC_FREE_SLIP = 2,
       ORC_BC_INLET_CONVECTIVE = 3 };

/* Rigid circular body. Centre(t) = (cx, cy) + (amp_x, amp_y) sin(2 pi t / period)
 * (period <= 0: fixed). Solid velocity: translation d centre/dt plus rigid
 * rotation omega about the centre. outside = 0: solid where r <= radius;
 * outside = 1: solid where r >= radius (an enclosing cylinder wall). */
typedef struct {
  double cx, cy, radius;
  double amp_x, amp_y, period;
  double omega;
  int32_t outside;
  int32_t pad_;
} orc_body;

typedef struct {
  int32_t nx, ny;
  int32_t collision;        /* ORC_SRT | ORC_MRT */
  int32_t bc_x;             /* ORC_BC_PERIODIC | ORC_BC_INLET_OUTLET | ORC_BC_INLET_CONVECTIVE */
  int32_t bc_y;             /* ORC_BC_PERIODIC | ORC_BC_FREE_SLIP */
  int32_t use_rates;        /* 1: take the nine MRT rates from rates[] */
  double tau;               /* SRT relaxation time; MRT s_n = 1/tau */
  double lambda;            /* MRT magic parameter, Eq. lambda_parameter */
  double eta;               /* penalization parameter (paper: 1e-7) */
  double u_in[2];           /* inlet velocity (bc_x = INLET_OUTLET) */
  double g[2];              /* uniform body force per unit mass */
  double rates[9];          /* explicit S diagonal when use_rates = 1 */
  const uint8_t* chi;       /* static mask [ny][nx] (0 fluid, 1 solid) or NULL */
  const double* us;         /* static solid velocity [2][ny][nx] or NULL */
  const orc_body* bodies;   /* rigid bodies, may be NULL */
  int32_t n_bodies;
  int32_t pad_;
  /* Convective outlet (bc_x = ORC_BC_INLET_CONVECTIVE, Section 3.3 after
   * Yang): the ghost column x = nx of the three directions entering through
   * it (alpha = 3, 6, 7) carries its own state g, advanced once per step by
   * the implicit upwind form of dg/dt + U_c dg/dx = 0,
   *   g^t = (g^{t-1} + U_c f*_alpha(nx - 1, y; t)) / (1 + U_c),
   * before the last column pulls g^t. outlet holds g^{t-1} as [3][ny] (rows of
   * alpha = 3, 6, 7; values of f) and orc_run leaves g^{t+n-1} in it. */
  double u_conv;
  double* outlet;
} orc_config;

/* D2Q9 constants as the oracle derives them (for the pin tests). */
void orc_velocity_set(int32_t xi[9][2]);
void orc_weights(double w[9]);
void orc_moment_matrix(double M[9][9]);
void orc_moment_matrix_inverse(double Minv[9][9]);

/* Single-node building blocks. */
void orc_equilibrium(double rho, double ux, double uy, double feq[9]);
void orc_guo_force_srt(double tau, double ux, double uy, double fx, double fy, double F[9]);
void orc_guo_force_mrt(double ux, double uy, double fx, double fy, double F[9]);
void orc_mrt_equilibrium_moments(double rho, double ux, double uy, double meq[9]);

/* Macroscopic step of one node: density, implicit velocity (Eq. 18) and the
 * penalization force (Eq. 17) for mask value chi and solid velocity us. */
void orc_node_macros(const orc_config* c, const double f[9], int32_t chi,
                     double usx, double usy, double* rho, double* ux, double* uy,
                     double* fpx, double* fpy);
/* The same quantities from the literal Eqs. 18 and 17 (for the pin test of
 * the algebraically rearranged force). */
void orc_node_macros_literal(const orc_config* c, const double f[9], int32_t chi,
                             double usx, double usy, double* rho, double* ux,
                             double* uy, double* fpx, double* fpy);

/* Collision of one node (pulled populations f -> post-collision fout). */
void orc_collide_node(const orc_config* c, const double f[9], int32_t chi,
                      double usx, double usy, double fout[9],
                      double* fpx, double* fpy);

/* Mask and solid velocity at time step t: chi[ny][nx] in {0,1}, us[2][ny][nx]. */
int orc_mask(const orc_config* c, int64_t t, uint8_t* chi, double* us);

/* f[9][ny][nx] := f_eq(rho0, u) with u from u_init[2][ny][nx] (or zero). */
int orc_init_equilibrium(const orc_config* c, double rho0, const double* u_init, double* f);

/* Advance n steps from step index t0. f holds the post-collision store f*(t0)
 * on entry and f*(t0 + n) on return. fx, fy, mass (each n entries, may be NULL)
 * receive per step the force on the bodies (-sum of the penalization force over
 * solid nodes) and the total density of the pulled populations. */
int orc_run(const orc_config* c, double* f, int64_t t0, int64_t n,
            double* fx, double* fy, double* mass);

/* Density and implicit velocity that the next step (index t) computes from the
 * store f (post-collision f*(t)). */
int orc_moments(const orc_config* c, const double* f, int64_t t,
                double* rho, double* ux, double* uy);

/* One step (index t) of the listed nodes only, from the store f*(t): the pull
 * with the boundary rules of orc_run (convective state read, not advanced),
 * the mask of step t and the collision. fout [n][9] receives f*(t+1) of each
 * node, fpx/fpy its penalization force and chi its mask (any may be NULL
 * except fout). The same arithmetic as orc_run, node by node, so that a step
 * of a grid too large for the oracle can be checked at sampled nodes. */
int orc_step_nodes(const orc_config* c, const double* f, int64_t t, int64_t n,
                   const int32_t* xs, const int32_t* ys, double* fout, double* fpx, double* fpy,
                   uint8_t* chi);

/* Momentum-exchange force on the solids at step index t (the force measure of
 * Section 3.3, after Ladd): over every link from a fluid node x_f to a solid
 * node x_s = x_f + xi_alpha, the momentum xi_alpha [f*_alpha(x_f) +
 * f*_abar(x_s)] of the store f*(t) crosses into the solid (abar: the opposite
 * direction). Links that leave the grid through a non-periodic side are not
 * counted. */
int orc_momentum_exchange(const orc_config* c, const double* f, int64_t t, double* fx, double* fy);

/* Host threads of the row loop (OpenMP builds); n <= 0: all processors. */
void orc_set_num_threads(int n);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
