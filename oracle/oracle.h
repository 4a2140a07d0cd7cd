/*
 * Oracle for the moment-chain lattice Boltzmann method for geometrically and
 * constitutively non-linear solids (Mueller, Faust, Schlueter, Mueller,
 * "Extending the Lattice Boltzmann Method to Non-linear Solid Mechanics",
 * arXiv 2502.00920).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow FP64 CPU implementation of
 * what the paper defines, written to check the CUDA path against.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Every number is FP64.  Build with -ffp-contract=off so that x86 and Arm give
 * the same bits.
 *
 * Array layouts used at this interface (all row-major, node (x, y) at index
 * y*nx + x, x along the first lattice axis):
 *   u, v : [ny][nx][2]      displacement / velocity components (1, 2)
 *   P    : [ny][nx][4]      P11, P12, P21, P22 (first Piola-Kirchhoff stress)
 *   H    : [ny][nx][4]      H11, H12, H21, H22 with H_ab = d u_a / d X_b
 */
#ifndef LBS_ORACLE_H
#define LBS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_SVK = 0, ORA_NH = 1, ORA_LE = 2 };
enum { ORA_PERIODIC = 0, ORA_DIRICHLET = 1, ORA_NEUMANN = 2 };
/* time shapes of a prescribed boundary value; t is the iteration k or the
 * time k dt (ora_edge.time_unit) */
enum {
  ORA_CONST = 0,       /* amp                                                  */
  ORA_LINEAR_RAMP = 1, /* amp * clamp((k-t0)/(t1-t0), 0, 1)                    */
  ORA_SIN2_RAMP = 2,   /* amp * sin^2(pi/2 * clamp((k-t0)/(t1-t0), 0, 1))      */
  ORA_HALF_SINE = 3,   /* amp * sin(pi (k-t0)/(t1-t0)) on [t0, t1), else 0     */
  ORA_RICKER = 4,      /* amp * (1 - d^2/s) exp(-d^2/(2 s)), d = k-t0, k < t1  */
  ORA_DISP_RAMP = 5    /* Dirichlet only: amp is a displacement reached
                          linearly over [t0, t1); value = rho0 amp / duration */
};
/* Where the stress block sits in an iteration.  TEXT: after the displacement
 * update, so the collision at t uses S(u(t)) as the note on the source time
 * level in Sect. 3.1 requires.  LISTING: before it, as Algorithm 1 is
 * printed, so the collision at t uses S(u(t - dt)); kept only to show that
 * this order is unstable for nu > 1/4 even on a periodic lattice. */
enum { ORA_ORDER_TEXT = 0, ORA_ORDER_LISTING = 1 };
/* How the Neumann rule's r^bd, the node's own Pi entries and P + Pi(H) are
 * carried to the wall, which lies half a spacing beyond the boundary node
 * (Sect. 3.3, "extrapolated to the boundary").  OWN: the boundary node's
 * value (zeroth order; the default).  LINEAR: v + (v - v_in)/2 along the
 * normal of each wall the link crosses, v_in the value at the next node
 * inwards (both walls' terms at a corner). */
enum { ORA_EXTRAP_OWN = 0, ORA_EXTRAP_LINEAR = 1 };
enum { ORA_LEFT = 0, ORA_RIGHT = 1, ORA_BOTTOM = 2, ORA_TOP = 3 };

typedef struct {
  int type;       /* ORA_PERIODIC | ORA_DIRICHLET (momentum j*) | ORA_NEUMANN (traction T*) */
  int shape;      /* ORA_CONST ... ORA_DISP_RAMP */
  double amp[2];
  double t0, t1, s;
  int time_unit;  /* 0: t0, t1, s in iterations; 1: in time (t_k = k dt), s in time^2 */
} ora_edge;

typedef struct {
  int nx, ny;     /* lattice nodes along x and y (>= 3 each)               */
  double dx;      /* lattice spacing Delta X                               */
  double tau;     /* relaxation time in units of Delta t (> 0.5)           */
  int model;      /* ORA_SVK | ORA_NH | ORA_LE                             */
  double E, nu, rho0;
  double body[2]; /* body force density b                                  */
  ora_edge edge[4]; /* left (-x), right (+x), bottom (-y), top (+y)        */
  int order;      /* ORA_ORDER_TEXT (default) or ORA_ORDER_LISTING, below   */
  int extrap;     /* ORA_EXTRAP_OWN (default) or ORA_EXTRAP_LINEAR, below    */
} ora_config;

typedef struct ora_sim ora_sim;

/* Derived parameters: Lame constants (plane strain), shear wave speed c_s,
 * lattice speed c = sqrt(3) c_s, time step dt = dx / c. */
void ora_params(const ora_config *cfg, double out[5]); /* mu, lam, cs, c, dt */

/* Returns NULL on invalid input.  u0, v0 may be NULL (zero). */
ora_sim *ora_create(const ora_config *cfg, const double *u0, const double *v0);
void ora_step(ora_sim *s, long n);
long ora_iteration(const ora_sim *s);
/* u, v = j / rho0 with j = sum_q c_q f_q + dt/2 S (the momentum that the
 * collision at the current time uses) and P(H(u)); any pointer may be NULL. */
void ora_fields(const ora_sim *s, double *u, double *v, double *P);
void ora_destroy(ora_sim *s);
int ora_threads(void);

/* The state one iteration hands to the next, as a flat vector of
 * ora_state_size(s) doubles: the distributions f (before collision, [9][n]),
 * u ([2][n]), and P, Pi(H) ([4][n] each) and the source S ([2][n]) as they
 * stand (functions of u in the text order, of the previous u in the listing
 * order); node i = y*nx + x.  With the linear material and zero loads one
 * iteration is a linear map of this vector (used by the stability tests). */
long ora_state_size(const ora_sim *s);
void ora_get_state(const ora_sim *s, double *x);
void ora_set_state(ora_sim *s, const double *x);

/* Building blocks, exported for the pin tests. */
void ora_first_piola(int model, double lam, double mu, const double H[4], double P[4]);
void ora_pi_of_h(double mu, const double H[4], double Pi[4]);
void ora_equilibrium(double cs, double r, const double j[2], const double Pi[4], double feq[9]);
void ora_forcing(double cs, const double S[2], double psi[9]);
void ora_gradient(const ora_config *cfg, const double *u, double *H);
void ora_load(const ora_config *cfg, int edge, long k, double out[2]);
/* Grid error norms of Sect. 4 (Eq. griderror): E2 = (1/n) ||u - u_ref||_2 /
 * ||u_ref||_2 and Einf = ||u - u_ref||_inf / ||u_ref||_2 over n nodes, u and
 * u_ref [n][2]; ||a||_2 = sqrt(sum a . a), ||a||_inf = max of max(|a_1|, |a_2|)
 * (the reference's norm in the denominators). */
void ora_grid_error(long n, const double *u, const double *u_ref, double out[2]);
/* A node value a[y*nx + x] carried to the wall(s) (wx: ORA_LEFT/ORA_RIGHT or
 * -1, wy: ORA_BOTTOM/ORA_TOP or -1) a boundary link crosses, as the Neumann
 * rule of Sect. 3.3 takes r, the Pi entries and P + Pi(H) under cfg->extrap;
 * NAN if (x, y) is not on those walls. */
double ora_wall_value(const ora_config *cfg, const double *a, int x, int y, int wx, int wy);

#ifdef __cplusplus
}
#endif
#endif
