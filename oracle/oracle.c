/*
 * Oracle: the moment-chain LBM for non-linear solids, plain FP64 C.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  It follows Algorithm 1 of the
 * paper in its printed order, one whole-lattice pass per block:
 *   1. moments, equilibrium, forcing, collision, streaming   (Alg. 1, Sect. 3.2)
 *   2. bounce-back / anti-bounce-back boundaries             (Eq. bbcon, abbcon)
 *   3. displacement gradient and stresses                    (Eq. defgrad, Sect. 4)
 *   4. source term, moments, trapezoidal displacement update (Eq. source, Sect. 3.2)
 *
 * Readings where the paper is silent, garbled or inconsistent (each is listed
 * in the design notes of the repository):
 *   R1  collision uses the algorithm's form
 *       f - (dt/tau)(f - feq) + (1 - dt/(2 tau)) psi dt   (Eq. for the collision
 *       step in Sect. 2 has a misplaced bracket), with tau given in units of dt.
 *   R2  the trapezoidal update carries the time step:
 *       u(t+dt) = u(t) + dt/(2 rho0) (j(t+dt) + j(t)).
 *   R3  Pi(H) = -mu (H + H^T + tr(H) I): the constitutive momentum flux implied by
 *       the third line of the moment chain with Q = c_s^2 (j d + j d + j d),
 *       j = rho0 du/dt and c_s^2 rho0 = mu.
 *   R4  Lame constants are plane strain: mu = E/(2(1+nu)),
 *       lam = E nu/((1+nu)(1-2 nu)) (the only choice that reproduces the CFL
 *       bounds nu <= 1/4 and nu <= 5/11 quoted in Sect. 3.2).
 *   R5  finite differences are applied per axis: central in the interior of an
 *       axis, first-order one-sided on the first/last node of a walled axis,
 *       central with wrap-around on a periodic axis.
 *   R6  initial state: r0 = -rho0 tr(H0) (from d_t r + div j = 0), Pi0 = Pi(H0),
 *       f0 = feq(r0, rho0 v0 - dt/2 S0, Pi0), so that the first moment j
 *       evaluated by the algorithm equals rho0 v0.
 *   R7  r^bd of the Neumann rule is the node's own r from block 1; every tensor
 *       "extrapolated to the boundary" is the boundary node's own value; the
 *       (P + Pi(H)) used there is the array as it stands when block 2 runs,
 *       i.e. computed in block 3 of the previous iteration (or at initialisation).
 *       ORA_EXTRAP_LINEAR selects the other reading: v + (v - v_in)/2 for each
 *       wall the link crosses, v_in at the next node inwards (the wall lies half
 *       a spacing beyond the node).  Pinned through ora_wall_value: on a field
 *       that is linear across the wall the carried value is the field at the
 *       wall itself (x = -dX/2 from the boundary node), exactly.
 *   R8  corners: each outgoing link takes the rule of the wall it crosses,
 *       with the Pi* of that wall (its other diagonal entry from the node's
 *       own moment); a diagonal link crossing two walls is Dirichlet if either
 *       wall is (momentum: mean of the two walls' j* when both are), else its
 *       Pi* takes Pi*_xx from the x-wall, Pi*_yy from the y-wall and the mean
 *       of the two walls' shear entries.
 *   R9  a boundary value is evaluated at t_k = k dt of the iteration k that
 *       applies it.
 *
 * Parity status: the building blocks are pinned by the CPU tests (moment
 * identities, closed-form stresses, energy derivatives, FD exactness, rigid
 * motions, stationary homogeneous states, wave speeds, conservation).  The
 * paper's own error tables need its finite-element data, which is not
 * available, so full trajectories are pinned only through those properties.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- D2Q9 velocity set (Tab. 1): c_q = c (EX[q], EY[q]), weights w_q ---- */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* the direction opposite to q (q-bar) */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

typedef double mat2[2][2];

struct ora_sim {
  ora_config cfg;
  double mu, lam, cs, c, dt;
  long k;       /* iteration counter, t_k = k dt */
  long n;       /* number of nodes */
  int per_x, per_y;
  int order;
  double *f;     /* [9][n] distributions at t_k (before collision)        */
  double *fcoll; /* [9][n] post-collision distributions                   */
  double *fnew;  /* [9][n] distributions at t_k + dt                      */
  double *u;     /* [2][n] displacement                                   */
  double *j;     /* [2][n] momentum density j(t_k) (block 4 / init)       */
  double *jt;    /* [2][n] momentum density evaluated in block 1          */
  double *S;     /* [2][n] source term as it stands                       */
  double *P;     /* [4][n] P(H) as it stands                              */
  double *Ph;    /* [4][n] Pi(H) as it stands                             */
  double *r;     /* [n]    moment r from block 1                          */
  double *Pi;    /* [3][n] moment Pi (xx, xy, yy) from block 1            */
};

/* ------------------------------------------------------------------------ */
/* small 2x2 tensor helpers                                                  */

static void mat_mul(const mat2 A, const mat2 B, mat2 C) {
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) C[a][b] = A[a][0] * B[0][b] + A[a][1] * B[1][b];
}

static void mat_transpose(const mat2 A, mat2 T) {
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) T[a][b] = A[b][a];
}

static double mat_det(const mat2 A) { return A[0][0] * A[1][1] - A[0][1] * A[1][0]; }

static void mat_inverse(const mat2 A, mat2 Ai) {
  double d = mat_det(A);
  Ai[0][0] = A[1][1] / d;
  Ai[0][1] = -A[0][1] / d;
  Ai[1][0] = -A[1][0] / d;
  Ai[1][1] = A[0][0] / d;
}

static double delta(int a, int b) { return a == b ? 1.0 : 0.0; }

/* ------------------------------------------------------------------------ */
/* parameters (Sect. 3.1/3.2, reading R4)                                   */

void ora_params(const ora_config *cfg, double out[5]) {
  double E = cfg->E, nu = cfg->nu;
  double mu = E / (2.0 * (1.0 + nu));
  double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double cs = sqrt(mu / cfg->rho0); /* shear wave speed, Sect. 3.1 */
  double c = sqrt(3.0) * cs;        /* lattice speed, Sect. 3.2      */
  double dt = cfg->dx / c;          /* c = dX / dt, Sect. 2          */
  out[0] = mu;
  out[1] = lam;
  out[2] = cs;
  out[3] = c;
  out[4] = dt;
}

/* ------------------------------------------------------------------------ */
/* constitutive laws (Sect. 4): E, C, J from H, S(E) or S(C, J), P = (H + 1) S */

void ora_first_piola(int model, double lam, double mu, const double Hf[4], double Pf[4]) {
  mat2 H = {{Hf[0], Hf[1]}, {Hf[2], Hf[3]}};
  mat2 P;
  if (model == ORA_LE) {
    /* linear elastic comparison material: lam tr(H) I + mu (H + H^T) */
    double trH = H[0][0] + H[1][1];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) P[a][b] = lam * trH * delta(a, b) + mu * (H[a][b] + H[b][a]);
  } else {
    mat2 F, Ft, C, Ht, HtH, E, S;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) F[a][b] = H[a][b] + delta(a, b);
    mat_transpose(F, Ft);
    mat_mul(Ft, F, C); /* C = (H + 1)^T (H + 1) */
    mat_transpose(H, Ht);
    mat_mul(Ht, H, HtH);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) E[a][b] = 0.5 * (Ht[a][b] + H[a][b] + HtH[a][b]);
    double J = mat_det(F);
    if (model == ORA_SVK) {
      double trE = E[0][0] + E[1][1];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) S[a][b] = lam * trE * delta(a, b) + 2.0 * mu * E[a][b];
    } else { /* ORA_NH */
      mat2 Ci;
      mat_inverse(C, Ci);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          S[a][b] = 0.5 * lam * (J * J - 1.0) * Ci[a][b] + mu * (delta(a, b) - Ci[a][b]);
    }
    mat_mul(F, S, P); /* P = (H + 1) S */
  }
  Pf[0] = P[0][0];
  Pf[1] = P[0][1];
  Pf[2] = P[1][0];
  Pf[3] = P[1][1];
}

/* constitutive momentum flux Pi(H) (reading R3) */
void ora_pi_of_h(double mu, const double Hf[4], double Pif[4]) {
  double trH = Hf[0] + Hf[3];
  Pif[0] = -mu * (Hf[0] + Hf[0] + trH);
  Pif[1] = -mu * (Hf[1] + Hf[2]);
  Pif[2] = -mu * (Hf[2] + Hf[1]);
  Pif[3] = -mu * (Hf[3] + Hf[3] + trH);
}

/* ------------------------------------------------------------------------ */
/* equilibrium and forcing (Sect. 3.2)                                       */

static void equilibrium_full(double cs, double c, double r, const double j[2], const mat2 Pi,
                             double feq[9]) {
  double cs2 = cs * cs;
  for (int q = 0; q < 9; ++q) {
    double cq[2] = {c * EX[q], c * EY[q]};
    double cj = cq[0] * j[0] + cq[1] * j[1];
    double contr = 0.0; /* (Pi - r cs^2 I) : (c_q c_q - cs^2 I) */
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        contr += (Pi[a][b] - r * cs2 * delta(a, b)) * (cq[a] * cq[b] - cs2 * delta(a, b));
    feq[q] = W[q] * (r + cj / cs2 + contr / (2.0 * cs2 * cs2));
  }
}

void ora_equilibrium(double cs, double r, const double j[2], const double Pif[4], double feq[9]) {
  mat2 Pi = {{Pif[0], Pif[1]}, {Pif[2], Pif[3]}};
  equilibrium_full(cs, sqrt(3.0) * cs, r, j, Pi, feq);
}

static void forcing_full(double cs, double c, const double S[2], double psi[9]) {
  for (int q = 0; q < 9; ++q) psi[q] = W[q] * (c * EX[q] * S[0] + c * EY[q] * S[1]) / (cs * cs);
}

void ora_forcing(double cs, const double S[2], double psi[9]) {
  forcing_full(cs, sqrt(3.0) * cs, S, psi);
}

/* ------------------------------------------------------------------------ */
/* finite differences (Sect. 3.2, reading R5)                                */

static long node(const ora_sim *s, int x, int y) { return (long)y * s->cfg.nx + x; }

static double d_dx(const ora_sim *s, const double *a, int x, int y) {
  int nx = s->cfg.nx;
  double h = s->cfg.dx;
  if (s->per_x) {
    int xp = (x + 1) % nx, xm = (x - 1 + nx) % nx;
    return (a[node(s, xp, y)] - a[node(s, xm, y)]) / (2.0 * h);
  }
  if (x == 0) return (a[node(s, 1, y)] - a[node(s, 0, y)]) / h;
  if (x == nx - 1) return (a[node(s, nx - 1, y)] - a[node(s, nx - 2, y)]) / h;
  return (a[node(s, x + 1, y)] - a[node(s, x - 1, y)]) / (2.0 * h);
}

static double d_dy(const ora_sim *s, const double *a, int x, int y) {
  int ny = s->cfg.ny;
  double h = s->cfg.dx;
  if (s->per_y) {
    int yp = (y + 1) % ny, ym = (y - 1 + ny) % ny;
    return (a[node(s, x, yp)] - a[node(s, x, ym)]) / (2.0 * h);
  }
  if (y == 0) return (a[node(s, x, 1)] - a[node(s, x, 0)]) / h;
  if (y == ny - 1) return (a[node(s, x, ny - 1)] - a[node(s, x, ny - 2)]) / h;
  return (a[node(s, x, y + 1)] - a[node(s, x, y - 1)]) / (2.0 * h);
}

/* H_ab = d u_a / d X_b (Eq. defgrad) at every node; u is [2][n], H is [4][n] */
static void gradient_all(const ora_sim *s, const double *u, double *H) {
  long n = s->n;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < s->cfg.ny; ++y)
    for (int x = 0; x < s->cfg.nx; ++x) {
      long i = node(s, x, y);
      H[0 * n + i] = d_dx(s, u + 0 * n, x, y);
      H[1 * n + i] = d_dy(s, u + 0 * n, x, y);
      H[2 * n + i] = d_dx(s, u + 1 * n, x, y);
      H[3 * n + i] = d_dy(s, u + 1 * n, x, y);
    }
}

/* block 3: H from u, then P(H) and Pi(H) at every node */
static void stresses(ora_sim *s) {
  long n = s->n;
  double *H = malloc(sizeof(double) * 4 * n);
  gradient_all(s, s->u, H);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) {
    double Hi[4] = {H[i], H[n + i], H[2 * n + i], H[3 * n + i]}, Pi_[4], Ph_[4];
    ora_first_piola(s->cfg.model, s->lam, s->mu, Hi, Pi_);
    ora_pi_of_h(s->mu, Hi, Ph_);
    for (int m = 0; m < 4; ++m) {
      s->P[m * n + i] = Pi_[m];
      s->Ph[m * n + i] = Ph_[m];
    }
  }
  free(H);
}

/* S = rho0 b + div(P + Pi(H)), (div N)_a = d N_ab / d X_b (Eq. source) */
static void source(ora_sim *s) {
  long n = s->n;
  double *N = malloc(sizeof(double) * 4 * n);
  for (long m = 0; m < 4 * n; ++m) N[m] = s->P[m] + s->Ph[m];
#pragma omp parallel for schedule(static)
  for (int y = 0; y < s->cfg.ny; ++y)
    for (int x = 0; x < s->cfg.nx; ++x) {
      long i = node(s, x, y);
      s->S[0 * n + i] = s->cfg.rho0 * s->cfg.body[0] + d_dx(s, N + 0 * n, x, y) + d_dy(s, N + 1 * n, x, y);
      s->S[1 * n + i] = s->cfg.rho0 * s->cfg.body[1] + d_dx(s, N + 2 * n, x, y) + d_dy(s, N + 3 * n, x, y);
    }
  free(N);
}

/* ------------------------------------------------------------------------ */
/* prescribed boundary values (reading R9)                                   */

void ora_load(const ora_config *cfg, int edge, long k, double out[2]) {
  const ora_edge *e = &cfg->edge[edge];
  double p[5];
  ora_params(cfg, p);
  double t = e->time_unit ? (double)k * p[4] : (double)k, f = 0.0;
  double span = e->t1 - e->t0;
  switch (e->shape) {
    case ORA_CONST:
      f = 1.0;
      break;
    case ORA_LINEAR_RAMP: {
      double x = (t - e->t0) / span;
      f = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
      break;
    }
    case ORA_SIN2_RAMP: {
      double x = (t - e->t0) / span;
      x = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
      double sn = sin(0.5 * M_PI * x);
      f = sn * sn;
      break;
    }
    case ORA_HALF_SINE:
      f = (t >= e->t0 && t < e->t1) ? sin(M_PI * (t - e->t0) / span) : 0.0;
      break;
    case ORA_RICKER: {
      double d = t - e->t0;
      f = t < e->t1 ? (1.0 - d * d / e->s) * exp(-0.5 * d * d / e->s) : 0.0;
      break;
    }
    case ORA_DISP_RAMP: {
      double duration = e->time_unit ? span : span * p[4];
      f = (t >= e->t0 && t < e->t1) ? cfg->rho0 / duration : 0.0;
      break;
    }
    default:
      f = 0.0;
  }
  out[0] = e->amp[0] * f;
  out[1] = e->amp[1] * f;
}

/* ------------------------------------------------------------------------ */
/* Neumann momentum flux Pi* at a boundary node (Sect. 3.3, readings R7, R8) */

/* quasi-boundary traction on a wall with outward unit normal N:
 *   Pi* N = -T* + (P + Pi(H)) N  ->  first row and column of Pi* */
/* The value of a node field carried to the wall(s) a link crosses (reading
 * R7 and its linear variant): the node's own value, or under
 * ORA_EXTRAP_LINEAR v + (v - v_in)/2 for each crossed wall, v_in the value at
 * the next node inwards along that wall's normal. */
static double at_wall(const ora_sim *s, const double *a, int x, int y, int wx, int wy) {
  double v = a[node(s, x, y)];
  if (s->cfg.extrap != ORA_EXTRAP_LINEAR) return v;
  double e = v;
  if (wx >= 0) e += 0.5 * (v - a[node(s, wx == ORA_LEFT ? x + 1 : x - 1, y)]);
  if (wy >= 0) e += 0.5 * (v - a[node(s, x, wy == ORA_BOTTOM ? y + 1 : y - 1)]);
  return e;
}

/* the building block above on a caller's scalar field a[ny][nx], for the pin
 * tests; NAN if (x, y) does not lie on the named walls */
double ora_wall_value(const ora_config *cfg, const double *a, int x, int y, int wx, int wy) {
  if (x < 0 || x >= cfg->nx || y < 0 || y >= cfg->ny) return NAN;
  int okx = wx == -1 || (wx == ORA_LEFT && x == 0) || (wx == ORA_RIGHT && x == cfg->nx - 1);
  int oky = wy == -1 || (wy == ORA_BOTTOM && y == 0) || (wy == ORA_TOP && y == cfg->ny - 1);
  if (!okx || !oky) return NAN;
  ora_sim tmp;
  memset(&tmp, 0, sizeof(tmp));
  tmp.cfg = *cfg;
  tmp.n = (long)cfg->nx * cfg->ny;
  return at_wall(&tmp, a, x, y, wx, wy);
}

static void wall_flux_column(const ora_sim *s, int x, int y, int edge, int wx, int wy, double col[2]) {
  long n = s->n;
  double Nv[2] = {0.0, 0.0};
  if (edge == ORA_LEFT) Nv[0] = -1.0;
  if (edge == ORA_RIGHT) Nv[0] = 1.0;
  if (edge == ORA_BOTTOM) Nv[1] = -1.0;
  if (edge == ORA_TOP) Nv[1] = 1.0;
  double T[2];
  ora_load(&s->cfg, edge, s->k, T);
  mat2 NP;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      NP[a][b] = at_wall(s, s->P + (2 * a + b) * n, x, y, wx, wy) + at_wall(s, s->Ph + (2 * a + b) * n, x, y, wx, wy);
  int nd = (edge == ORA_LEFT || edge == ORA_RIGHT) ? 0 : 1;
  for (int a = 0; a < 2; ++a) {
    double q = -T[a] + NP[a][0] * Nv[0] + NP[a][1] * Nv[1];
    col[a] = q / Nv[nd]; /* Pi*_{a n} N_n = q_a */
  }
}

static void neumann_flux(const ora_sim *s, int x, int y, int xwall, int ywall, mat2 Pis) {
  long n = s->n;
  /* start from the node's own moment (extrapolated entries) */
  Pis[0][0] = at_wall(s, s->Pi + 0 * n, x, y, xwall, ywall);
  Pis[0][1] = Pis[1][0] = at_wall(s, s->Pi + 1 * n, x, y, xwall, ywall);
  Pis[1][1] = at_wall(s, s->Pi + 2 * n, x, y, xwall, ywall);
  double cx[2], cy[2];
  if (xwall >= 0) wall_flux_column(s, x, y, xwall, xwall, ywall, cx);
  if (ywall >= 0) wall_flux_column(s, x, y, ywall, xwall, ywall, cy);
  if (xwall >= 0 && ywall >= 0) {
    Pis[0][0] = cx[0];
    Pis[1][1] = cy[1];
    Pis[0][1] = Pis[1][0] = 0.5 * (cx[1] + cy[0]);
  } else if (xwall >= 0) {
    Pis[0][0] = cx[0];
    Pis[1][0] = Pis[0][1] = cx[1];
  } else if (ywall >= 0) {
    Pis[1][1] = cy[1];
    Pis[0][1] = Pis[1][0] = cy[0];
  }
}

/* ------------------------------------------------------------------------ */
/* creation and initialisation (Alg. 1 "Initialise", reading R6)             */

static int validate(const ora_config *c) {
  if (c->nx < 3 || c->ny < 3) return 0;
  if (!(c->tau > 0.5) || !(c->dx > 0.0) || !(c->rho0 > 0.0) || !(c->E > 0.0)) return 0;
  if (!(c->nu > -1.0 && c->nu < 0.5)) return 0;
  if (c->model < ORA_SVK || c->model > ORA_LE) return 0;
  for (int e = 0; e < 4; ++e) {
    const ora_edge *ed = &c->edge[e];
    if (ed->type < ORA_PERIODIC || ed->type > ORA_NEUMANN) return 0;
    if (ed->shape < ORA_CONST || ed->shape > ORA_DISP_RAMP) return 0;
    if ((ed->shape == ORA_LINEAR_RAMP || ed->shape == ORA_SIN2_RAMP || ed->shape == ORA_HALF_SINE ||
         ed->shape == ORA_DISP_RAMP) && !(ed->t1 > ed->t0))
      return 0;
    if (ed->shape == ORA_RICKER && !(ed->s > 0.0)) return 0;
    if (ed->shape == ORA_DISP_RAMP && ed->type != ORA_DIRICHLET) return 0;
    if (ed->time_unit != 0 && ed->time_unit != 1) return 0;
  }
  if (c->order != ORA_ORDER_TEXT && c->order != ORA_ORDER_LISTING) return 0;
  if (c->extrap != ORA_EXTRAP_OWN && c->extrap != ORA_EXTRAP_LINEAR) return 0;
  if ((c->edge[ORA_LEFT].type == ORA_PERIODIC) != (c->edge[ORA_RIGHT].type == ORA_PERIODIC)) return 0;
  if ((c->edge[ORA_BOTTOM].type == ORA_PERIODIC) != (c->edge[ORA_TOP].type == ORA_PERIODIC)) return 0;
  return 1;
}

ora_sim *ora_create(const ora_config *cfg, const double *u0, const double *v0) {
  if (!validate(cfg)) return NULL;
  ora_sim *s = calloc(1, sizeof(ora_sim));
  s->cfg = *cfg;
  double p[5];
  ora_params(cfg, p);
  s->mu = p[0];
  s->lam = p[1];
  s->cs = p[2];
  s->c = p[3];
  s->dt = p[4];
  s->n = (long)cfg->nx * cfg->ny;
  s->per_x = cfg->edge[ORA_LEFT].type == ORA_PERIODIC;
  s->per_y = cfg->edge[ORA_BOTTOM].type == ORA_PERIODIC;
  s->order = cfg->order;
  long n = s->n;
  s->f = calloc(9 * n, sizeof(double));
  s->fcoll = calloc(9 * n, sizeof(double));
  s->fnew = calloc(9 * n, sizeof(double));
  s->u = calloc(2 * n, sizeof(double));
  s->j = calloc(2 * n, sizeof(double));
  s->jt = calloc(2 * n, sizeof(double));
  s->S = calloc(2 * n, sizeof(double));
  s->P = calloc(4 * n, sizeof(double));
  s->Ph = calloc(4 * n, sizeof(double));
  s->r = calloc(n, sizeof(double));
  s->Pi = calloc(3 * n, sizeof(double));

  /* fields u, H, P, Pi(H) and the source S */
  for (long i = 0; i < n; ++i) {
    s->u[i] = u0 ? u0[2 * i] : 0.0;
    s->u[n + i] = u0 ? u0[2 * i + 1] : 0.0;
  }
  stresses(s);
  source(s);

  /* moments r0 = -rho0 tr(H0), j0 = rho0 v0, Pi0 = Pi(H0); f <- feq */
  double *H = malloc(sizeof(double) * 4 * n);
  gradient_all(s, s->u, H);
  for (long i = 0; i < n; ++i) {
    double r0 = -cfg->rho0 * (H[i] + H[3 * n + i]);
    double j0[2] = {cfg->rho0 * (v0 ? v0[2 * i] : 0.0), cfg->rho0 * (v0 ? v0[2 * i + 1] : 0.0)};
    mat2 Pi0 = {{s->Ph[i], s->Ph[n + i]}, {s->Ph[2 * n + i], s->Ph[3 * n + i]}};
    double jshift[2] = {j0[0] - 0.5 * s->dt * s->S[i], j0[1] - 0.5 * s->dt * s->S[n + i]};
    double feq[9];
    equilibrium_full(s->cs, s->c, r0, jshift, Pi0, feq);
    for (int q = 0; q < 9; ++q) s->f[q * n + i] = feq[q];
    s->j[i] = j0[0];
    s->j[n + i] = j0[1];
  }
  free(H);
  s->k = 0;
  return s;
}

void ora_destroy(ora_sim *s) {
  if (!s) return;
  free(s->f);
  free(s->fcoll);
  free(s->fnew);
  free(s->u);
  free(s->j);
  free(s->jt);
  free(s->S);
  free(s->P);
  free(s->Ph);
  free(s->r);
  free(s->Pi);
  free(s);
}

long ora_iteration(const ora_sim *s) { return s->k; }

int ora_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* one iteration of Algorithm 1                                              */

static void block1_collide_stream(ora_sim *s) {
  long n = s->n;
  int nx = s->cfg.nx, ny = s->cfg.ny;
  double c = s->c, cs = s->cs, dt = s->dt, tau = s->cfg.tau;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) {
    double fq[9], feq[9], psi[9];
    for (int q = 0; q < 9; ++q) fq[q] = s->f[q * n + i];
    double S[2] = {s->S[i], s->S[n + i]};
    /* moments: r, j (with dt/2 S), Pi */
    double r = 0.0, jsum[2] = {0.0, 0.0};
    mat2 Pi = {{0.0, 0.0}, {0.0, 0.0}};
    for (int q = 0; q < 9; ++q) {
      double cq[2] = {c * EX[q], c * EY[q]};
      r += fq[q];
      for (int a = 0; a < 2; ++a) {
        jsum[a] += cq[a] * fq[q];
        for (int b = 0; b < 2; ++b) Pi[a][b] += cq[a] * cq[b] * fq[q];
      }
    }
    double j[2] = {jsum[0] + 0.5 * dt * S[0], jsum[1] + 0.5 * dt * S[1]};
    s->r[i] = r;
    s->Pi[i] = Pi[0][0];
    s->Pi[n + i] = Pi[0][1];
    s->Pi[2 * n + i] = Pi[1][1];
    s->jt[i] = j[0];
    s->jt[n + i] = j[1];
    equilibrium_full(cs, c, r, j, Pi, feq);
    forcing_full(cs, c, S, psi);
    for (int q = 0; q < 9; ++q)
      s->fcoll[q * n + i] = fq[q] - (1.0 / tau) * (fq[q] - feq[q]) + (1.0 - 1.0 / (2.0 * tau)) * psi[q] * dt;
  }
  /* stream: f_q(X + c_q dt, t + dt) <- f_q^coll(X, t); unset entries stay NaN
   * until the boundary block writes them */
  for (long m = 0; m < 9 * n; ++m) s->fnew[m] = NAN;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x)
      for (int q = 0; q < 9; ++q) {
        int tx = x + EX[q], ty = y + EY[q];
        if (s->per_x) tx = (tx + nx) % nx;
        if (s->per_y) ty = (ty + ny) % ny;
        if (tx < 0 || tx >= nx || ty < 0 || ty >= ny) continue;
        s->fnew[q * n + node(s, tx, ty)] = s->fcoll[q * n + node(s, x, y)];
      }
}

static void block2_boundaries(ora_sim *s) {
  long n = s->n;
  int nx = s->cfg.nx, ny = s->cfg.ny;
  double c = s->c, cs = s->cs, cs2 = cs * cs;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int on_x = !s->per_x && (x == 0 || x == nx - 1);
      int on_y = !s->per_y && (y == 0 || y == ny - 1);
      if (!on_x && !on_y) continue;
      long i = node(s, x, y);
      for (int q = 1; q < 9; ++q) {
        int tx = x + EX[q], ty = y + EY[q];
        int ox = !s->per_x && (tx < 0 || tx >= nx);
        int oy = !s->per_y && (ty < 0 || ty >= ny);
        if (!ox && !oy) continue; /* link q stays inside the lattice */
        int wx = ox ? (tx < 0 ? ORA_LEFT : ORA_RIGHT) : -1;
        int wy = oy ? (ty < 0 ? ORA_BOTTOM : ORA_TOP) : -1;
        int dir_x = wx >= 0 && s->cfg.edge[wx].type == ORA_DIRICHLET;
        int dir_y = wy >= 0 && s->cfg.edge[wy].type == ORA_DIRICHLET;
        double cq[2] = {c * EX[q], c * EY[q]};
        double fc = s->fcoll[q * n + i];
        double out;
        if (dir_x || dir_y) {
          /* Eq. (bbcon): f_qbar = f_q^coll - 2/cs^2 w_q c_q . j* */
          double js[2] = {0.0, 0.0};
          if (dir_x && dir_y) {
            double a[2], b[2];
            ora_load(&s->cfg, wx, s->k, a);
            ora_load(&s->cfg, wy, s->k, b);
            js[0] = 0.5 * (a[0] + b[0]);
            js[1] = 0.5 * (a[1] + b[1]);
          } else {
            ora_load(&s->cfg, dir_x ? wx : wy, s->k, js);
          }
          out = fc - 2.0 / cs2 * W[q] * (cq[0] * js[0] + cq[1] * js[1]);
        } else {
          /* Eq. (abbcon): f_qbar = -f_q^coll + 2 w_q (r + (Pi* - r cs^2 I):(c c - cs^2 I)/(2 cs^4)) */
          /* Pi* from the wall(s) this link crosses */
          mat2 Pis;
          neumann_flux(s, x, y, wx, wy, Pis);
          double rbd = at_wall(s, s->r, x, y, wx, wy);
          double contr = 0.0;
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
              contr += (Pis[a][b] - rbd * cs2 * delta(a, b)) * (cq[a] * cq[b] - cs2 * delta(a, b));
          out = -fc + 2.0 * W[q] * (rbd + contr / (2.0 * cs2 * cs2));
        }
        s->fnew[OPP[q] * n + i] = out;
      }
    }
}

/* j(t + dt) and the trapezoidal displacement update; S is the array as it
 * stands (evaluated at t, Sect. 3.1 note on the source time level) */
static void update_displacement(ora_sim *s) {
  long n = s->n;
  double c = s->c, dt = s->dt, rho0 = s->cfg.rho0;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) {
    double jsum[2] = {0.0, 0.0};
    for (int q = 0; q < 9; ++q) {
      jsum[0] += c * EX[q] * s->fnew[q * n + i];
      jsum[1] += c * EY[q] * s->fnew[q * n + i];
    }
    for (int a = 0; a < 2; ++a) {
      double jn = jsum[a] + 0.5 * dt * s->S[a * n + i];
      s->u[a * n + i] = s->u[a * n + i] + dt / (2.0 * rho0) * (jn + s->jt[a * n + i]);
      s->j[a * n + i] = jn;
    }
  }
}

void ora_step(ora_sim *s, long nsteps) {
  for (long it = 0; it < nsteps; ++it) {
    block1_collide_stream(s);
    block2_boundaries(s);
    if (s->order == ORA_ORDER_LISTING) {
      stresses(s); /* H from u(t_k) */
      source(s);
      update_displacement(s);
    } else {
      update_displacement(s);
      stresses(s); /* H from u(t_k + dt): the next collision uses S(t_k + dt) */
      source(s);
    }
    double *tmp = s->f;
    s->f = s->fnew;
    s->fnew = tmp;
    s->k += 1;
  }
}

/* ------------------------------------------------------------------------ */
/* grid error norms (Sect. 4, Eq. griderror and the grid norms beside it)    */

/* ||a||_2 = sqrt(sum over nodes of a . a), a = [n][2] */
static double grid_norm2(long n, const double *a) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[2 * i] * a[2 * i] + a[2 * i + 1] * a[2 * i + 1];
  return sqrt(s);
}

/* ||a||_inf = max over nodes of max(|a_1|, |a_2|) (reading of max(u1, u2)) */
static double grid_norm_inf(long n, const double *a) {
  double m = 0.0;
  for (long i = 0; i < n; ++i) {
    double v = fabs(a[2 * i]) > fabs(a[2 * i + 1]) ? fabs(a[2 * i]) : fabs(a[2 * i + 1]);
    if (v > m) m = v;
  }
  return m;
}

void ora_grid_error(long n, const double *u, const double *u_ref, double out[2]) {
  double *du = malloc(sizeof(double) * 2 * n);
  for (long i = 0; i < 2 * n; ++i) du[i] = u[i] - u_ref[i];
  double r = grid_norm2(n, u_ref);
  out[0] = (1.0 / (double)n) * grid_norm2(n, du) / r;
  out[1] = grid_norm_inf(n, du) / r;
  free(du);
}

/* ------------------------------------------------------------------------ */
/* the carried state (for the stability analysis of the one-step map)       */

long ora_state_size(const ora_sim *s) { return 21 * s->n; }

/* f [9][n], u [2][n], P [4][n], Pi(H) [4][n], S [2][n], in that order */
void ora_get_state(const ora_sim *s, double *x) {
  long n = s->n;
  memcpy(x, s->f, sizeof(double) * 9 * n);
  memcpy(x + 9 * n, s->u, sizeof(double) * 2 * n);
  memcpy(x + 11 * n, s->P, sizeof(double) * 4 * n);
  memcpy(x + 15 * n, s->Ph, sizeof(double) * 4 * n);
  memcpy(x + 19 * n, s->S, sizeof(double) * 2 * n);
}

void ora_set_state(ora_sim *s, const double *x) {
  long n = s->n;
  memcpy(s->f, x, sizeof(double) * 9 * n);
  memcpy(s->u, x + 9 * n, sizeof(double) * 2 * n);
  memcpy(s->P, x + 11 * n, sizeof(double) * 4 * n);
  memcpy(s->Ph, x + 15 * n, sizeof(double) * 4 * n);
  memcpy(s->S, x + 19 * n, sizeof(double) * 2 * n);
}

/* ------------------------------------------------------------------------ */
/* outputs                                                                   */

void ora_gradient(const ora_config *cfg, const double *u_aos, double *H_aos) {
  ora_sim tmp;
  memset(&tmp, 0, sizeof(tmp));
  tmp.cfg = *cfg;
  tmp.n = (long)cfg->nx * cfg->ny;
  tmp.per_x = cfg->edge[ORA_LEFT].type == ORA_PERIODIC;
  tmp.per_y = cfg->edge[ORA_BOTTOM].type == ORA_PERIODIC;
  long n = tmp.n;
  double *u = malloc(sizeof(double) * 2 * n), *H = malloc(sizeof(double) * 4 * n);
  for (long i = 0; i < n; ++i) {
    u[i] = u_aos[2 * i];
    u[n + i] = u_aos[2 * i + 1];
  }
  gradient_all(&tmp, u, H);
  for (long i = 0; i < n; ++i)
    for (int m = 0; m < 4; ++m) H_aos[4 * i + m] = H[m * n + i];
  free(u);
  free(H);
}

void ora_fields(const ora_sim *s, double *u, double *v, double *P) {
  long n = s->n;
  if (u)
    for (long i = 0; i < n; ++i) {
      u[2 * i] = s->u[i];
      u[2 * i + 1] = s->u[n + i];
    }
  if (v)
    /* the momentum the collision at the current time uses (Alg. 1, first
     * block): j = sum_q c_q f_q + dt/2 S with S = S(u(t)) */
    for (long i = 0; i < n; ++i) {
      double jx = 0.0, jy = 0.0;
      for (int q = 0; q < 9; ++q) {
        jx += s->c * EX[q] * s->f[q * n + i];
        jy += s->c * EY[q] * s->f[q * n + i];
      }
      v[2 * i] = (jx + 0.5 * s->dt * s->S[i]) / s->cfg.rho0;
      v[2 * i + 1] = (jy + 0.5 * s->dt * s->S[n + i]) / s->cfg.rho0;
    }
  if (P) {
    double *H = malloc(sizeof(double) * 4 * n);
    gradient_all(s, s->u, H);
    for (long i = 0; i < n; ++i) {
      double Hi[4] = {H[i], H[n + i], H[2 * n + i], H[3 * n + i]};
      ora_first_piola(s->cfg.model, s->lam, s->mu, Hi, P + 4 * i);
    }
    free(H);
  }
}
