/*
 * weno_oracle.h -- plain CPU oracle of the WENO-ZA6 finite-difference scheme.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Method: Gu, Wang, Don, Jung, "A Family of Even-Order Central-Upwind WENO
 * Schemes with Averaged Downwind and Novel Global Smoothness Indicators"
 * (arXiv 2603.26272).  Section 2 gives the general framework, Section 3 the
 * sixth-order scheme (WENO-ZA6) and Section 4 the Euler experiments.
 *
 * Layout of every state array: [nbatch][ncomp][ny][nx], contiguous doubles,
 * x fastest.  ncomp = 1 (scalar equations), 3 (1D Euler: rho, rho*u, E) or
 * 4 (2D Euler: rho, rho*u, rho*v, E).  ny = 1 in 1D.
 *
 * Return codes: 0 = ok, 1 = bad argument, 2 = nonphysical state met
 * (rho <= 0, p <= 0, a non-positive Roe sound speed or a non-finite value).
 */
#ifndef WENO_ORACLE_H
#define WENO_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The oracle's own description of a problem (not the CUDA library's). */
typedef struct {
  int32_t system;   /* 0 = advection u_t + a u_x = 0, 1 = Euler, 2 = Burgers,    */
                    /* 3 = Buckley-Leverett (scalar systems are 1D)             */
  int32_t ndim;     /* 1 or 2                                                   */
  int64_t nbatch;   /* independent problems of the same shape                   */
  int64_t nx, ny;   /* cells per axis (ny = 1 in 1D)                            */
  double dx, dy;    /* cell sizes                                               */
  int32_t bc_x;     /* 0 = transmissive (zero-gradient ghosts), 1 = periodic    */
  int32_t bc_y;
  double gamma;     /* ratio of specific heats                                  */
  double eps;       /* sensitivity parameter epsilon of eq. (21)                */
  double mu0;       /* mu_0 of eq. (22)                                         */
  double p;         /* power parameter p of eq. (21)                            */
  int32_t ai;       /* 1: affine-invariant descaler mu[f] of eq. (22); 0: mu=1  */
  int32_t alpha_mode; /* 0: GLF alpha per characteristic field, 1: one alpha   */
  double adv_speed; /* a of the scalar advection equation                       */
  int32_t order;    /* 2r: 4, 6 (also 0), 8 or 10 -- the Appendix schemes        */
  int32_t pad;
} ora_grid;

/* WENO-ZA6 positive numerical flux at x_{i+1/2} from f = (f_{i-2}, ..., f_{i+3})
 * (Section 3, eqs. (11)-(22) with L = 1, q = 1).  If detail != NULL it receives
 * 16 values: fk[4] (candidate fluxes), beta[5] (beta_0, beta_1, beta_2, beta_d,
 * beta_3), tau, mu, omega[4], and the returned flux is also detail[15]. */
double ora_za6_flux(const double f[6], double eps, double mu0, double p, int ai,
                    double *detail);

/* The same flux in quadruple precision (f given as doubles; p in {1, 1.5, 2}). */
double ora_za6_flux_quad(const double f[6], double eps, double mu0, double p, int ai);

/* Central-upwind WENO flux of order 2r (r = 2..5; Section 2 with the tables of
 * Section 3 and the Appendix) from f_{i-r+1} .. f_{i+r}; NaN for a bad order. */
double ora_za_flux(int order, const double *f, double eps, double mu0, double p, int ai);

/* Tables of order 2r: c_2r[2r], c_k[(r+1) r], d[r+1], B_0..B_{r-1}, B_d
 * [(r+1) r r], c_tau[2r].  Returns 1 for a bad order. */
int ora_coefficients_r(int order, double *out);

/* Coefficient tables used by the oracle, for the pins: c6[6] (eq. (10)),
 * ck[4][3] (eq. (11)), d[4] (eq. (12)), B0, B1, B2, Bd [3][3] (eq. (15)),
 * ctau[6] (eq. (17)).  Writes 6 + 12 + 4 + 36 + 6 = 64 doubles. */
void ora_coefficients(double *out64);

/* L_inf error of (f_hat_{j+1/2} - f_hat_{j-1/2}) / dx against f'(x_j) for
 * f = x^(ncp+1) exp(0.75 x) on the nodes x_j = -1 + j dx, j = 0 .. 2/dx
 * (Section 3.1, Tables 3 and 4).  eps_variable = 1 uses eps = dx^(2(ncp-1)),
 * else eps = 1e-40; mu = 1 (no Ai).  use_quad = 1 evaluates everything in
 * quadruple precision.  p must be 1, 1.5 or 2 when use_quad = 1. */
double ora_operator_error(int ncp, int inv_dx, double p, int eps_variable, int use_quad);

/* Roe-averaged face state of two neighbouring cells UL, UR (nc = 3: 1D Euler,
 * nc = 4: 2D Euler; dir 0 = x, 1 = y) and the eigen-system of the flux
 * Jacobian there, the one the characteristic-wise splitting of Section 4.2
 * projects with (the face_flux routine uses exactly this).  out[40]:
 * u, v, H, c, R[4][4] (right eigenvectors as columns, row major), L[4][4]
 * (= R^{-1}), lam[4] (eigenvalues in the order of R's columns); rows and
 * columns beyond nc are 0.  Returns 0, 1 (bad argument) or 2 (nonphysical). */
int ora_roe_face(int nc, int dir, double gamma, const double *UL, const double *UR,
                 double *out);

/* Global Lax-Friedrichs speeds of eq. (6) for a stage input U:
 * alpha[b][dir][m] = max over all cells of |lambda_m| (dir 0 = x, 1 = y,
 * m = characteristic field, 4 slots, unused ones 0).  Returns a status code. */
int ora_alpha(const ora_grid *g, const double *U, double *alpha /* nbatch*8 */);

/* Right-hand side L(U) = -(F_{i+1/2}-F_{i-1/2})/dx [-(G_{j+1/2}-G_{j-1/2})/dy]
 * (eq. (5), applied dimension by dimension) using the speeds alpha. */
int ora_rhs(const ora_grid *g, const double *U, const double *alpha, double *L);

/* L(U) of one cell (b, j, i) only: out[ncomp]. */
int ora_rhs_cell(const ora_grid *g, const double *U, const double *alpha, int64_t b,
                 int64_t j, int64_t i, double *out);

/* CFL time step of each problem from U: 1D dt = cfl dx / max(|u|+c);
 * 2D dt = cfl / (max(|u|+c)/dx + max(|v|+c)/dy); advection dt = cfl dx / |a|. */
int ora_cfl_dt(const ora_grid *g, const double *U, double cfl, double *dt /* nbatch */);

/* One third-order SSP Runge-Kutta step (Shu-Osher form) of every problem with
 * its own dt[b] (dt[b] <= 0 leaves problem b unchanged). */
int ora_ssprk3_step(const ora_grid *g, double *U, const double *dt);

/* Advance every problem from t0 to t_final with CFL steps, the last step of
 * each clipped to land on t_final, at most max_steps steps.  t_out[b] and
 * steps_out[b] receive the reached time and step count of each problem.
 * Returns 3 if max_steps ran out first. */
int ora_solve(const ora_grid *g, double *U, double cfl, double t0, double t_final,
              int64_t max_steps, double *t_out, int64_t *steps_out);

/* Exact solution of the 1D Euler Riemann problem with states (rl,ul,pl) for
 * x < x0 and (rr,ur,pr) for x > x0 at time t > 0, sampled at n points x[].
 * star[0] = p*, star[1] = u*.  Returns 2 if a vacuum would form. */
int ora_riemann_exact(double rl, double ul, double pl, double rr, double ur, double pr,
                      double gamma, double x0, double t, int64_t n, const double *x,
                      double *rho, double *u, double *p, double *star);

#ifdef __cplusplus
}
#endif
#endif
