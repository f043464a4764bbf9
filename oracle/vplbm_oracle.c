/*
 * Plain FP64 CPU oracle of the VP-LBM time step (arXiv 1812.05401).
 *
 * TEST INFRASTRUCTURE ONLY: the CUDA path is checked against this file. Only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code with the CUDA library.
 *
 * Every function follows the paper's equations in the paper's order, written
 * out plainly: explicit velocity set (evaluated from its cos/sin formula),
 * weights, the printed moment matrix M and its numerically inverted M^-1, and
 * no fused or rearranged arithmetic beyond the one documented algebraic
 * rearrangement of the penalization force (orc_node_macros). Rows of the grid
 * are independent within a step; OpenMP (when compiled with -fopenmp) splits
 * them across host cores, and the per-row partial sums are added in row order
 * so that results do not depend on the thread count.
 */
#include "vplbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Speed of sound squared, c_s^2 = c^2/3 with c = 1 (Section 2.1.1). */
static const double CS2 = 1.0 / 3.0;

/* ---------------------------------------------------------------------------
 * D2Q9 model (Sections 2.1.1 and 2.1.2)
 * ------------------------------------------------------------------------- */

/* Velocity set, Eq. vecteurs_D2Q9: alpha = 1..4 at angles (alpha-1) pi/2 with
 * speed c; alpha = 5..8 at angles (2 alpha - 9) pi/4 with speed sqrt(2) c.
 * Evaluated from the formula and rounded to the integer lattice. */
void orc_velocity_set(int32_t xi[9][2]) {
  xi[0][0] = 0;
  xi[0][1] = 0;
  for (int a = 1; a <= 4; ++a) {
    double th = (double)(a - 1) * M_PI / 2.0;
    xi[a][0] = (int32_t)lround(cos(th));
    xi[a][1] = (int32_t)lround(sin(th));
  }
  for (int a = 5; a <= 8; ++a) {
    double th = (double)(2 * a - 9) * M_PI / 4.0;
    xi[a][0] = (int32_t)lround(sqrt(2.0) * cos(th));
    xi[a][1] = (int32_t)lround(sqrt(2.0) * sin(th));
  }
}

/* Weights, Eq. anex_eq19. */
void orc_weights(double w[9]) {
  w[0] = 4.0 / 9.0;
  for (int a = 1; a <= 4; ++a) w[a] = 1.0 / 9.0;
  for (int a = 5; a <= 8; ++a) w[a] = 1.0 / 36.0;
}

/* Transformation matrix M, Eq. eq1.7, rows (rho, e, eps, j_x, q_x, j_y, q_y,
 * p_xx, p_xy), columns alpha = 0..8. */
void orc_moment_matrix(double M[9][9]) {
  static const double Mp[9][9] = {
      {1, 1, 1, 1, 1, 1, 1, 1, 1},
      {-4, -1, -1, -1, -1, 2, 2, 2, 2},
      {4, -2, -2, -2, -2, 1, 1, 1, 1},
      {0, 1, 0, -1, 0, 1, -1, -1, 1},
      {0, -2, 0, 2, 0, 1, -1, -1, 1},
      {0, 0, 1, 0, -1, 1, 1, -1, -1},
      {0, 0, -2, 0, 2, 1, 1, -1, -1},
      {0, 1, -1, 1, -1, 0, 0, 0, 0},
      {0, 0, 0, 0, 0, 1, -1, 1, -1}};
  memcpy(M, Mp, sizeof(Mp));
}

/* M^-1 by Gauss-Jordan elimination with partial pivoting: the plain numerical
 * inverse, making no use of the orthogonality of M's rows. */
void orc_moment_matrix_inverse(double Minv[9][9]) {
  double A[9][18];
  double M[9][9];
  orc_moment_matrix(M);
  for (int i = 0; i < 9; ++i) {
    for (int j = 0; j < 9; ++j) {
      A[i][j] = M[i][j];
      A[i][9 + j] = (i == j) ? 1.0 : 0.0;
    }
  }
  for (int col = 0; col < 9; ++col) {
    int piv = col;
    for (int r = col + 1; r < 9; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (piv != col) {
      for (int j = 0; j < 18; ++j) {
        double t = A[col][j];
        A[col][j] = A[piv][j];
        A[piv][j] = t;
      }
    }
    double p = A[col][col];
    for (int j = 0; j < 18; ++j) A[col][j] /= p;
    for (int r = 0; r < 9; ++r) {
      if (r == col) continue;
      double fct = A[r][col];
      if (fct == 0.0) continue;
      for (int j = 0; j < 18; ++j) A[r][j] -= fct * A[col][j];
    }
  }
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) Minv[i][j] = A[i][9 + j];
}

/* Constants of the model, evaluated once per oracle call. */
typedef struct {
  int32_t xi[9][2];
  double w[9];
  double M[9][9];
  double Minv[9][9];
  double S[9];
  int mirror_y[9]; /* direction with the same xi_x and opposite xi_y */
  double feq_in[9]; /* f_eq(1, u_in): the inlet ghost column */
} orc_model;

/* Equilibrium distribution (Section 2.1.1):
 * f_eq = w rho [1 + xi.u / cs^2 + u u : (xi xi - cs^2 I) / (2 cs^4)],
 * with u u : (xi xi - cs^2 I) = (xi.u)^2 - cs^2 |u|^2. */
static void equilibrium(const orc_model* m, double rho, double ux, double uy,
                        double feq[9]) {
  double uu = ux * ux + uy * uy;
  for (int a = 0; a < 9; ++a) {
    double xu = m->xi[a][0] * ux + m->xi[a][1] * uy;
    double contraction = xu * xu - CS2 * uu;
    feq[a] = m->w[a] * rho * (1.0 + xu / CS2 + contraction / (2.0 * CS2 * CS2));
  }
}

/* Forcing term, Eq. Guo2 (no prefactor):
 * F_alpha = w [(xi - u)/cs^2 + (xi.u) xi / cs^4] . f. */
static void guo_force(const orc_model* m, double ux, double uy, double fx,
                      double fy, double F[9]) {
  for (int a = 0; a < 9; ++a) {
    double xu = m->xi[a][0] * ux + m->xi[a][1] * uy;
    double vx = (m->xi[a][0] - ux) / CS2 + xu * m->xi[a][0] / (CS2 * CS2);
    double vy = (m->xi[a][1] - uy) / CS2 + xu * m->xi[a][1] / (CS2 * CS2);
    F[a] = m->w[a] * (vx * fx + vy * fy);
  }
}

/* Equilibrium moments (Section 2.1.2):
 * m_eq = rho (1, -2 + 3|u|^2, 1 - 3|u|^2, u, -u, v, -v, u^2 - v^2, u v). */
void orc_mrt_equilibrium_moments(double rho, double ux, double uy, double meq[9]) {
  double uu = ux * ux + uy * uy;
  meq[0] = rho;
  meq[1] = rho * (-2.0 + 3.0 * uu);
  meq[2] = rho * (1.0 - 3.0 * uu);
  meq[3] = rho * ux;
  meq[4] = -rho * ux;
  meq[5] = rho * uy;
  meq[6] = -rho * uy;
  meq[7] = rho * (ux * ux - uy * uy);
  meq[8] = rho * ux * uy;
}

/* Relaxation rates S = diag(0, s_n, s_n, 0, s_q, 0, s_q, s_n, s_n) with
 * s_n = 1/tau and s_q from Lambda = (1/s_n - 1/2)(1/s_q - 1/2)
 * (Eq. lambda_parameter), unless explicit rates are given. */
static void mrt_rates(const orc_config* c, double S[9]) {
  if (c->use_rates) {
    for (int k = 0; k < 9; ++k) S[k] = c->rates[k];
    return;
  }
  double sn = 1.0 / c->tau;
  double sq = 1.0 / (0.5 + c->lambda / (1.0 / sn - 0.5));
  S[0] = 0.0;
  S[1] = sn;
  S[2] = sn;
  S[3] = 0.0;
  S[4] = sq;
  S[5] = 0.0;
  S[6] = sq;
  S[7] = sn;
  S[8] = sn;
}

static void model_init(const orc_config* c, orc_model* m) {
  orc_velocity_set(m->xi);
  orc_weights(m->w);
  orc_moment_matrix(m->M);
  orc_moment_matrix_inverse(m->Minv);
  mrt_rates(c, m->S);
  for (int a = 0; a < 9; ++a) {
    m->mirror_y[a] = a;
    for (int b = 0; b < 9; ++b)
      if (m->xi[b][0] == m->xi[a][0] && m->xi[b][1] == -m->xi[a][1]) m->mirror_y[a] = b;
  }
  equilibrium(m, 1.0, c->u_in[0], c->u_in[1], m->feq_in);
}

/* Public single-node entry points (for the pin tests). */
void orc_equilibrium(double rho, double ux, double uy, double feq[9]) {
  orc_model m;
  orc_config c;
  memset(&c, 0, sizeof(c));
  c.tau = 1.0;
  model_init(&c, &m);
  equilibrium(&m, rho, ux, uy, feq);
}

void orc_guo_force_mrt(double ux, double uy, double fx, double fy, double F[9]) {
  orc_model m;
  orc_config c;
  memset(&c, 0, sizeof(c));
  c.tau = 1.0;
  model_init(&c, &m);
  guo_force(&m, ux, uy, fx, fy, F);
}

/* Eq. Guo1: Eq. Guo2 times (1 - 1/(2 tau)). */
void orc_guo_force_srt(double tau, double ux, double uy, double fx, double fy,
                       double F[9]) {
  orc_guo_force_mrt(ux, uy, fx, fy, F);
  double pre = 1.0 - 1.0 / (2.0 * tau);
  for (int a = 0; a < 9; ++a) F[a] *= pre;
}

/* ---------------------------------------------------------------------------
 * Volume penalization (Section 2.2)
 * ------------------------------------------------------------------------- */

/* Density (Eq. density), implicit velocity (Eq. vitesse_fluide_penalisation_1)
 * and penalization force (Eq. 17) of one node.
 *
 * Velocity: rho u = sum xi f + (1/2) f_tot (Eq. velocity) with the total force
 * f_tot = f_pen + rho g and f_pen = -rho (chi/eta)(u - u_s). Solving for u gives
 * Eq. 18, extended by the uniform body force g:
 *   u = (j + rho g/2 + (chi/(2 eta)) rho u_s) / (rho + (chi/(2 eta)) rho).
 * Force: substituting that u into Eq. 17 gives, exactly,
 *   f_pen = -kappa (j + rho g/2 - rho u_s),  kappa = (chi/eta) / (1 + chi/(2 eta)),
 * which is Eq. 17 without the subtraction u - u_s of two nearly equal numbers
 * whose rounding error chi/eta = 1e7 would multiply. */
static void node_macros(const orc_model* m, const orc_config* c, const double f[9],
                        int32_t chi, double usx, double usy, double* rho,
                        double* ux, double* uy, double* fpx, double* fpy) {
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int a = 0; a < 9; ++a) {
    r += f[a];
    jx += m->xi[a][0] * f[a];
    jy += m->xi[a][1] * f[a];
  }
  double ce = (double)chi / c->eta;   /* chi / eta */
  double half = 0.5 * ce;             /* (Delta t / 2) chi / eta */
  double bx = jx + 0.5 * r * c->g[0]; /* j + rho g / 2 */
  double by = jy + 0.5 * r * c->g[1];
  *rho = r;
  *ux = (bx + half * r * usx) / (r + half * r);
  *uy = (by + half * r * usy) / (r + half * r);
  double kappa = ce / (1.0 + half);
  *fpx = -kappa * (bx - r * usx);
  *fpy = -kappa * (by - r * usy);
}

void orc_node_macros(const orc_config* c, const double f[9], int32_t chi,
                     double usx, double usy, double* rho, double* ux, double* uy,
                     double* fpx, double* fpy) {
  orc_model m;
  model_init(c, &m);
  node_macros(&m, c, f, chi, usx, usy, rho, ux, uy, fpx, fpy);
}

/* Literal Eqs. 18 and 17: the same u, then f_pen = -rho (chi/eta)(u - u_s). */
void orc_node_macros_literal(const orc_config* c, const double f[9], int32_t chi,
                             double usx, double usy, double* rho, double* ux,
                             double* uy, double* fpx, double* fpy) {
  orc_model m;
  model_init(c, &m);
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int a = 0; a < 9; ++a) {
    r += f[a];
    jx += m.xi[a][0] * f[a];
    jy += m.xi[a][1] * f[a];
  }
  double ce = (double)chi / c->eta;
  double half = 0.5 * ce;
  *rho = r;
  *ux = (jx + 0.5 * r * c->g[0] + half * r * usx) / (r + half * r);
  *uy = (jy + 0.5 * r * c->g[1] + half * r * usy) / (r + half * r);
  *fpx = -r * ce * (*ux - usx);
  *fpy = -r * ce * (*uy - usy);
}

/* ---------------------------------------------------------------------------
 * Collision (Eq. LatticeBoltz for SRT, Eq. equa_lbl_mrt for MRT)
 * ------------------------------------------------------------------------- */

static void collide(const orc_model* m, const orc_config* c, const double f[9],
                    int32_t chi, double usx, double usy, double fout[9],
                    double* fpx, double* fpy) {
  double rho, ux, uy, px, py;
  node_macros(m, c, f, chi, usx, usy, &rho, &ux, &uy, &px, &py);
  /* Total body force: penalization plus the uniform force rho g. */
  double ftx = px + rho * c->g[0];
  double fty = py + rho * c->g[1];
  if (fpx) *fpx = px;
  if (fpy) *fpy = py;

  double F[9];
  guo_force(m, ux, uy, ftx, fty, F);

  if (c->collision == ORC_SRT) {
    /* f* = f - (f - f_eq)/tau + (1 - 1/(2 tau)) F_alpha (Eqs. LatticeBoltz, Guo1). */
    double feq[9];
    equilibrium(m, rho, ux, uy, feq);
    double pre = 1.0 - 1.0 / (2.0 * c->tau);
    for (int a = 0; a < 9; ++a) fout[a] = f[a] - (f[a] - feq[a]) / c->tau + pre * F[a];
    return;
  }

  /* MRT: f* = f - M^-1 [S (m - m_eq) - (I - S/2) M F] (Eqs. equa_lbl_mrt, Guo2). */
  double mom[9], meq[9], MF[9], r[9];
  orc_mrt_equilibrium_moments(rho, ux, uy, meq);
  for (int k = 0; k < 9; ++k) {
    mom[k] = 0.0;
    MF[k] = 0.0;
    for (int a = 0; a < 9; ++a) {
      mom[k] += m->M[k][a] * f[a];
      MF[k] += m->M[k][a] * F[a];
    }
  }
  for (int k = 0; k < 9; ++k)
    r[k] = m->S[k] * (mom[k] - meq[k]) - (1.0 - m->S[k] / 2.0) * MF[k];
  for (int a = 0; a < 9; ++a) {
    double corr = 0.0;
    for (int k = 0; k < 9; ++k) corr += m->Minv[a][k] * r[k];
    fout[a] = f[a] - corr;
  }
}

void orc_collide_node(const orc_config* c, const double f[9], int32_t chi,
                      double usx, double usy, double fout[9], double* fpx,
                      double* fpy) {
  orc_model m;
  model_init(c, &m);
  collide(&m, c, f, chi, usx, usy, fout, fpx, fpy);
}

/* ---------------------------------------------------------------------------
 * Geometry: staircase mask chi and solid velocity u_s (Section 2.2; the
 * node-in-shape approximation of curved walls of Section 3.2)
 * ------------------------------------------------------------------------- */

static void body_state(const orc_body* b, int64_t t, double* cx, double* cy,
                       double* vx, double* vy) {
  if (b->period > 0.0) {
    double ph = 2.0 * M_PI * (double)t / b->period;
    double s = sin(ph), co = cos(ph);
    double rate = 2.0 * M_PI / b->period;
    *cx = b->cx + b->amp_x * s;
    *cy = b->cy + b->amp_y * s;
    *vx = b->amp_x * rate * co;
    *vy = b->amp_y * rate * co;
  } else {
    *cx = b->cx;
    *cy = b->cy;
    *vx = 0.0;
    *vy = 0.0;
  }
}

/* Mask and solid velocity of node (x, y), given the body states st (centre
 * x, y and velocity x, y of each body at the time of the step): the static
 * mask first, then the first body whose shape holds the node. */
static int node_mask(const orc_config* c, const double* st, int x, int y, double* usx,
                     double* usy) {
  const size_t plane = (size_t)c->nx * (size_t)c->ny;
  size_t i = (size_t)y * c->nx + x;
  int solid = 0;
  double sx = 0.0, sy = 0.0;
  if (c->chi && c->chi[i]) {
    solid = 1;
    if (c->us) {
      sx = c->us[i];
      sy = c->us[plane + i];
    }
  } else {
    for (int b = 0; b < c->n_bodies; ++b) {
      const orc_body* bd = &c->bodies[b];
      double dx = (double)x - st[4 * b];
      double dy = (double)y - st[4 * b + 1];
      double r2 = dx * dx + dy * dy;
      double R2 = bd->radius * bd->radius;
      int in = bd->outside ? (r2 >= R2) : (r2 <= R2);
      if (in) {
        solid = 1;
        sx = st[4 * b + 2] - bd->omega * dy;
        sy = st[4 * b + 3] + bd->omega * dx;
        break;
      }
    }
  }
  *usx = sx;
  *usy = sy;
  return solid;
}

/* Body states at step index t: [n_bodies][4] (centre x, y, velocity x, y). */
static double* body_states(const orc_config* c, int64_t t) {
  int nb = c->n_bodies;
  double* st = (double*)malloc(sizeof(double) * 4 * (size_t)(nb > 0 ? nb : 1));
  if (!st) return NULL;
  for (int b = 0; b < nb; ++b)
    body_state(&c->bodies[b], t, &st[4 * b], &st[4 * b + 1], &st[4 * b + 2],
               &st[4 * b + 3]);
  return st;
}

int orc_mask(const orc_config* c, int64_t t, uint8_t* chi, double* us) {
  const int nx = c->nx, ny = c->ny;
  const size_t plane = (size_t)nx * (size_t)ny;
  double* st = body_states(c, t);
  if (!st) return 2;
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      double sx, sy;
      chi[i] = (uint8_t)node_mask(c, st, x, y, &sx, &sy);
      if (us) {
        us[i] = sx;
        us[plane + i] = sy;
      }
    }
  }
  free(st);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Streaming with boundary conditions: f_alpha(x, t+1) = f*_alpha(x - xi_alpha, t),
 * the left-hand side of Eq. LatticeBoltz, realised as a pull.
 * y: periodic, or a specular (free-slip, "symmetry") wall half-way outside the
 *    first and last rows: a population arriving from beyond the wall is the
 *    mirror image (xi_y -> -xi_y) of the one that left the same row.
 * x: periodic, or a ghost column x = -1 held at f_eq(1, u_in) (uniform inlet)
 *    and a ghost column x = nx that copies column nx - 1 (zero-gradient outlet)
 *    or holds the convective outlet state of this step (ghost, [9][ny]).
 * ------------------------------------------------------------------------- */

static double pull_one(const orc_model* m, const orc_config* c, const double* src,
                       const double* ghost, int a, int x, int y) {
  const int nx = c->nx, ny = c->ny;
  const size_t plane = (size_t)nx * (size_t)ny;
  int as = a;
  int xs = x - m->xi[a][0];
  int ys = y - m->xi[a][1];
  if (ys < 0 || ys >= ny) {
    if (c->bc_y == ORC_BC_PERIODIC) {
      ys = (ys + ny) % ny;
    } else { /* free slip: mirror of the population leaving the same row */
      as = m->mirror_y[a];
      ys = y;
    }
  }
  if (xs < 0 || xs >= nx) {
    if (c->bc_x == ORC_BC_PERIODIC) {
      xs = (xs + nx) % nx;
    } else if (xs < 0) {
      return m->feq_in[as];
    } else if (c->bc_x == ORC_BC_INLET_CONVECTIVE) {
      return ghost[(size_t)as * ny + ys];
    } else {
      xs = nx - 1;
    }
  }
  return src[(size_t)as * plane + (size_t)ys * nx + xs];
}

/* The three directions entering through the outlet, in the order of the
 * outlet state's rows. */
static const int OUTLET_DIRS[3] = {3, 6, 7};

/* Convective outlet: ghost[as][y] := (g^{t-1} + U_c f*_as(nx - 1, y)) / (1 + U_c)
 * for the directions entering through the outlet (see vplbm_oracle.h). */
static int outlet_advance(const orc_config* c, const double* src, double* ghost) {
  if (c->bc_x != ORC_BC_INLET_CONVECTIVE) return 0;
  if (!c->outlet || !(c->u_conv >= 0.0)) return 1;
  const int nx = c->nx, ny = c->ny;
  const size_t plane = (size_t)nx * (size_t)ny;
  for (int k = 0; k < 3; ++k) {
    const int a = OUTLET_DIRS[k];
    for (int y = 0; y < ny; ++y) {
      const double g_old = c->outlet[(size_t)k * ny + y];
      const double f_last = src[(size_t)a * plane + (size_t)y * nx + (nx - 1)];
      ghost[(size_t)a * ny + y] = (g_old + c->u_conv * f_last) / (1.0 + c->u_conv);
    }
  }
  return 0;
}

int orc_init_equilibrium(const orc_config* c, double rho0, const double* u_init,
                         double* f) {
  orc_model m;
  model_init(c, &m);
  const size_t plane = (size_t)c->nx * (size_t)c->ny;
  for (size_t i = 0; i < plane; ++i) {
    double ux = u_init ? u_init[i] : 0.0;
    double uy = u_init ? u_init[plane + i] : 0.0;
    double feq[9];
    equilibrium(&m, rho0, ux, uy, feq);
    for (int a = 0; a < 9; ++a) f[(size_t)a * plane + i] = feq[a];
  }
  return 0;
}

int orc_run(const orc_config* c, double* f, int64_t t0, int64_t n, double* fx,
            double* fy, double* mass) {
  const int nx = c->nx, ny = c->ny;
  const size_t plane = (size_t)nx * (size_t)ny;
  if (nx < 1 || ny < 1 || n < 0) return 1;
  double* g = (double*)malloc(sizeof(double) * 9 * plane);
  uint8_t* chi = (uint8_t*)malloc(plane);
  double* us = (double*)malloc(sizeof(double) * 2 * plane);
  double* row_sum = (double*)malloc(sizeof(double) * 3 * (size_t)ny);
  double* ghost = (double*)calloc(9 * (size_t)ny, sizeof(double));
  if (!g || !chi || !us || !row_sum || !ghost) {
    free(g);
    free(chi);
    free(us);
    free(row_sum);
    free(ghost);
    return 2;
  }
  orc_model m;
  model_init(c, &m);

  double* src = f;
  double* dst = g;
  int rc = 0;
  for (int64_t s = 0; s < n; ++s) {
    int64_t t = t0 + s;
    orc_mask(c, t, chi, us);
    if ((rc = outlet_advance(c, src, ghost)) != 0) break;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
      double sfx = 0.0, sfy = 0.0, smass = 0.0;
      for (int x = 0; x < nx; ++x) {
        size_t i = (size_t)y * nx + x;
        double fl[9], fo[9], px, py;
        for (int a = 0; a < 9; ++a) fl[a] = pull_one(&m, c, src, ghost, a, x, y);
        for (int a = 0; a < 9; ++a) smass += fl[a];
        collide(&m, c, fl, chi[i], us[i], us[plane + i], fo, &px, &py);
        if (chi[i]) { /* reaction on the body: minus the penalization force */
          sfx -= px;
          sfy -= py;
        }
        for (int a = 0; a < 9; ++a) dst[(size_t)a * plane + i] = fo[a];
      }
      row_sum[3 * (size_t)y + 0] = sfx;
      row_sum[3 * (size_t)y + 1] = sfy;
      row_sum[3 * (size_t)y + 2] = smass;
    }
    double tfx = 0.0, tfy = 0.0, tm = 0.0;
    for (int y = 0; y < ny; ++y) {
      tfx += row_sum[3 * (size_t)y + 0];
      tfy += row_sum[3 * (size_t)y + 1];
      tm += row_sum[3 * (size_t)y + 2];
    }
    if (fx) fx[s] = tfx;
    if (fy) fy[s] = tfy;
    if (mass) mass[s] = tm;
    if (c->bc_x == ORC_BC_INLET_CONVECTIVE) /* the state moves on to g^t */
      for (int k = 0; k < 3; ++k)
        for (int y = 0; y < ny; ++y)
          c->outlet[(size_t)k * ny + y] = ghost[(size_t)OUTLET_DIRS[k] * ny + y];
    double* tmp = src;
    src = dst;
    dst = tmp;
  }
  if (src != f) memcpy(f, src, sizeof(double) * 9 * plane);
  free(g);
  free(chi);
  free(us);
  free(row_sum);
  free(ghost);
  return rc;
}

int orc_moments(const orc_config* c, const double* f, int64_t t, double* rho,
                double* ux, double* uy) {
  const int nx = c->nx, ny = c->ny;
  const size_t plane = (size_t)nx * (size_t)ny;
  uint8_t* chi = (uint8_t*)malloc(plane);
  double* us = (double*)malloc(sizeof(double) * 2 * plane);
  double* ghost = (double*)calloc(9 * (size_t)ny, sizeof(double));
  if (!chi || !us || !ghost) {
    free(chi);
    free(us);
    free(ghost);
    return 2;
  }
  orc_model m;
  model_init(c, &m);
  orc_mask(c, t, chi, us);
  if (outlet_advance(c, f, ghost) != 0) { /* the state itself is not advanced */
    free(chi);
    free(us);
    free(ghost);
    return 1;
  }
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      double fl[9], px, py;
      for (int a = 0; a < 9; ++a) fl[a] = pull_one(&m, c, f, ghost, a, x, y);
      node_macros(&m, c, fl, chi[i], us[i], us[plane + i], &rho[i], &ux[i], &uy[i],
                  &px, &py);
    }
  }
  free(chi);
  free(us);
  free(ghost);
  return 0;
}

int orc_step_nodes(const orc_config* c, const double* f, int64_t t, int64_t n,
                   const int32_t* xs, const int32_t* ys, double* fout, double* fpx, double* fpy,
                   uint8_t* chi) {
  const int ny = c->ny;
  double* st = body_states(c, t);
  double* ghost = (double*)calloc(9 * (size_t)ny, sizeof(double));
  if (!st || !ghost) {
    free(st);
    free(ghost);
    return 2;
  }
  orc_model m;
  model_init(c, &m);
  if (outlet_advance(c, f, ghost) != 0) { /* the state itself is not advanced */
    free(st);
    free(ghost);
    return 1;
  }
  for (int64_t k = 0; k < n; ++k) {
    const int x = xs[k], y = ys[k];
    if (x < 0 || x >= c->nx || y < 0 || y >= ny) {
      free(st);
      free(ghost);
      return 1;
    }
    double usx, usy, fl[9], px, py;
    const int solid = node_mask(c, st, x, y, &usx, &usy);
    for (int a = 0; a < 9; ++a) fl[a] = pull_one(&m, c, f, ghost, a, x, y);
    collide(&m, c, fl, solid, usx, usy, fout + 9 * (size_t)k, &px, &py);
    if (fpx) fpx[k] = px;
    if (fpy) fpy[k] = py;
    if (chi) chi[k] = (uint8_t)solid;
  }
  free(st);
  free(ghost);
  return 0;
}

int orc_momentum_exchange(const orc_config* c, const double* f, int64_t t, double* fx,
                          double* fy) {
  const int nx = c->nx, ny = c->ny;
  const size_t plane = (size_t)nx * (size_t)ny;
  uint8_t* chi = (uint8_t*)malloc(plane);
  if (!chi) return 2;
  orc_model m;
  model_init(c, &m);
  orc_mask(c, t, chi, NULL);
  double sx = 0.0, sy = 0.0;
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      if (chi[(size_t)y * nx + x]) continue; /* links start at fluid nodes */
      for (int a = 1; a < 9; ++a) {
        int xs = x + m.xi[a][0], ys = y + m.xi[a][1];
        if (xs < 0 || xs >= nx) {
          if (c->bc_x != ORC_BC_PERIODIC) continue;
          xs = (xs + nx) % nx;
        }
        if (ys < 0 || ys >= ny) {
          if (c->bc_y != ORC_BC_PERIODIC) continue;
          ys = (ys + ny) % ny;
        }
        if (!chi[(size_t)ys * nx + xs]) continue;
        int abar = 0;
        for (int b = 0; b < 9; ++b)
          if (m.xi[b][0] == -m.xi[a][0] && m.xi[b][1] == -m.xi[a][1]) abar = b;
        const double flow = f[(size_t)a * plane + (size_t)y * nx + x] +
                            f[(size_t)abar * plane + (size_t)ys * nx + xs];
        sx += m.xi[a][0] * flow;
        sy += m.xi[a][1] * flow;
      }
    }
  }
  free(chi);
  *fx = sx;
  *fy = sy;
  return 0;
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
  (void)n;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
