/*
 * lbs.h - C ABI of liblbs: the moment-chain lattice Boltzmann method for
 * geometrically and constitutively non-linear solids (Mueller, Faust,
 * Schlueter, Mueller, "Extending the Lattice Boltzmann Method to Non-linear
 * Solid Mechanics", arXiv 2502.00920), running on one NVIDIA GB300 (sm_103a).
 *
 * One time step is Algorithm 1 of the paper on a 2-D D2Q9 lattice (Tab. 1):
 * BGK collision with the constitutive forcing term (Sect. 3.2), streaming,
 * bounce-back (Dirichlet, Eq. bbcon) and anti-bounce-back (Neumann,
 * Eq. abbcon) boundary rules (Sect. 3.3), the trapezoidal displacement update,
 * the finite-difference displacement gradient and the St. Venant-Kirchhoff or
 * neo-Hooke first Piola-Kirchhoff stress (Sect. 4).  All of it runs in
 * hand-written CUDA kernels; the library never computes on the host.
 *
 * Conventions.
 *   - Node (x, y), 0 <= x < nx, 0 <= y < ny, sits at X = (x dx, y dx).
 *     Host and device field arrays are row-major with x fastest:
 *       u, v : double [ny][nx][2]          (components 1, 2)
 *       P    : double [ny][nx][4]          (P11, P12, P21, P22)
 *     with P_ab = P_ab(H), H_ab = d u_a / d X_b.
 *   - Edge order in lbs_bcs: left (-x), right (+x), bottom (-y), top (+y).
 *   - Times of boundary-value shapes are iteration counts k or times k dt.
 *   - Every function returns LBS_OK (0) or a negative LBS_E* code;
 *     lbs_last_error() gives a message for the calling thread.
 *   - The library owns all device memory of a handle (cudaMalloc, or the
 *     allocator installed with lbs_set_allocator).  The caller owns every
 *     buffer it passes in.  Handles are not thread-safe; separate handles may
 *     be used from separate threads and streams.
 *   - Work is issued on the handle's stream (its own non-blocking stream
 *     unless lbs_set_stream gave another) and is asynchronous unless stated.
 */
#ifndef LBS_H
#define LBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define LBS_OK 0
#define LBS_EINVAL (-1)    /* invalid argument or configuration             */
#define LBS_ENOMEM (-2)    /* device or host allocation failed              */
#define LBS_ECUDA (-3)     /* a CUDA runtime call failed                    */
#define LBS_EUNSTABLE (-4) /* a monitor found a non-finite value            */
#define LBS_ETIMEOUT (-5)  /* a bounded wait gave up                        */
#define LBS_EBUSY (-6)     /* resource busy (serving: queue full)           */
#define LBS_ENOTFOUND (-7) /* unknown ticket                                */
#define LBS_ECANCELED (-8) /* serving: the request was cancelled           */

/* ---- enumerations ----------------------------------------------------- */
/* storage precision of the distributions; u is kept at double precision or
 * as a compensated pair of floats (hi + lo), arithmetic as stated */
enum {
  LBS_FP64 = 0,  /* g, u: double; arithmetic double                          */
  LBS_FP32 = 1,  /* g: float; u: float pair; arithmetic float                */
  LBS_FP16S = 2  /* g: half, scaled by 2^gscale_log2; u: float pair; float   */
};
enum { LBS_SVK = 0, LBS_NH = 1, LBS_LE = 2 }; /* Sect. 4; LE: lam tr(H) I + mu (H + H^T) */
enum { LBS_PERIODIC = 0, LBS_DIRICHLET = 1, LBS_NEUMANN = 2 };
/* time shape s(t) of a boundary value amp * s(t); t is the iteration k or the
 * time k dt, per edge (lbs_edge.time_unit) */
enum { LBS_ITERATIONS = 0, LBS_TIME = 1 };
/* how a Neumann wall rule carries r, Pi and P + Pi(H) from the boundary node
 * to the wall a link crosses (Sect. 3.3 asks for values "extrapolated to the
 * boundary" without saying how) */
enum {
  LBS_EXTRAP_OWN = 0,   /* the boundary node's own values (zeroth order)      */
  LBS_EXTRAP_LINEAR = 1 /* two-point: v + (v - v_in) / 2 for each crossed wall,
                           v_in at the next node inwards along its normal     */
};
enum {
  LBS_CONST = 0,       /* 1                                                  */
  LBS_LINEAR_RAMP = 1, /* clamp((k - t0) / (t1 - t0), 0, 1)                  */
  LBS_SIN2_RAMP = 2,   /* sin^2(pi/2 clamp((k - t0) / (t1 - t0), 0, 1))      */
  LBS_HALF_SINE = 3,   /* sin(pi (k - t0) / (t1 - t0)) for t0 <= k < t1, else 0 */
  LBS_RICKER = 4,      /* (1 - d^2/s) exp(-d^2 / (2 s)), d = k - t0, for k < t1 */
  LBS_DISP_RAMP = 5    /* Dirichlet only: amp is a displacement reached linearly
                          over [t0, t1); the momentum is rho0 amp / duration
                          there and 0 elsewhere                               */
};

/* ---- configuration ---------------------------------------------------- */
typedef struct {
  int32_t nx, ny;      /* nodes per axis, each >= 3                          */
  double dx;           /* lattice spacing Delta X (> 0)                      */
  double tau;          /* BGK relaxation time in units of dt (> 0.5)         */
  int32_t precision;   /* LBS_FP64 | LBS_FP32 | LBS_FP16S                    */
  int32_t gscale_log2; /* LBS_FP16S: stored g = g * 2^gscale_log2; 0 = auto  */
  int32_t wall_extrap; /* LBS_EXTRAP_OWN (0) | LBS_EXTRAP_LINEAR; LINEAR keeps
                          a second layer of the boundary side array           */
} lbs_lattice;

typedef struct {
  int32_t model;  /* LBS_SVK | LBS_NH | LBS_LE                                */
  double E, nu;   /* Young's modulus, Poisson's ratio; plane-strain Lame      */
  double rho0;    /* reference density                                        */
  double body[2]; /* body force density b                                     */
} lbs_material;

typedef struct {
  int32_t type;      /* LBS_PERIODIC | LBS_DIRICHLET (momentum j*) | LBS_NEUMANN (traction T*) */
  int32_t shape;     /* LBS_CONST ... LBS_DISP_RAMP                          */
  double amp[2];     /* vector amplitude                                     */
  double t0, t1;     /* shape times                                          */
  double s;          /* LBS_RICKER width (time^2)                            */
  int32_t time_unit; /* LBS_ITERATIONS: k; LBS_TIME: t = k dt (the paper's)  */
} lbs_edge;

typedef struct {
  lbs_edge edge[4]; /* left, right, bottom, top; periodic edges must pair    */
} lbs_bcs;

typedef struct {
  int64_t iteration;  /* k at which the monitor was taken                    */
  int64_t nonfinite;  /* number of non-finite values in g and u              */
  double max_abs_u;   /* max over nodes and components of |u_a|              */
  double momentum[2]; /* sum over nodes of the first moment of g (momentum)  */
  double mass;        /* sum over nodes of the zeroth moment of g (r)        */
} lbs_monitors;

typedef struct lbs_handle lbs_handle;

/* ---- simulation handle ------------------------------------------------- */

/* Validate the configuration, derive mu, lam (plane strain, Sect. 3.2),
 * c_s = sqrt(mu/rho0), c = sqrt(3) c_s and dt = dx / c, allocate the state
 * on the current CUDA device and initialise it at rest (u = v = 0).
 * Errors: LBS_EINVAL (nx or ny < 3, tau <= 0.5, dx <= 0, rho0 <= 0, E <= 0,
 * nu outside (-1, 0.5), unpaired periodic edges, unknown enum, a ramp with
 * t1 <= t0, LBS_DISP_RAMP on a non-Dirichlet edge), LBS_ENOMEM, LBS_ECUDA.
 * A Poisson ratio above the paper's CFL bound (nu > 1/4 with first-order
 * boundary stencils, Sect. 3.2) is accepted; lbs_cfl_warning reports it. */
int lbs_create(const lbs_lattice *lat, const lbs_material *mat, const lbs_bcs *bcs, lbs_handle **out);

/* Destroy a handle and free its device memory.  NULL is accepted. */
int lbs_destroy(lbs_handle *h);

/* Issue further work of h on the given cudaStream_t (NULL: the handle's own
 * stream).  The stream must stay valid while h uses it. */
int lbs_set_stream(lbs_handle *h, void *cuda_stream);

/* Initial displacement u0 and velocity v0 ([ny][nx][2] doubles, host memory;
 * either may be NULL for zero).  Resets the iteration counter to 0 and builds
 * the initial distributions of Alg. 1 "Initialise": r0 = -rho0 tr H0,
 * Pi0 = Pi(H0) = -mu (H0 + H0^T + tr H0 I), f0 = feq(r0, rho0 v0 - dt/2 S0, Pi0).
 * The host arrays are copied into the handle's second state buffers (which
 * the first iteration overwrites) where they fit, else into a temporary
 * device buffer.  Synchronous. */
int lbs_set_initial(lbs_handle *h, const double *u0, const double *v0);

/* As lbs_set_initial with device pointers; asynchronous on the stream. */
int lbs_set_initial_device(lbs_handle *h, const double *u0, const double *v0);

/* Advance n >= 0 iterations (asynchronous).  Launches one fused kernel per
 * iteration, replayed from a CUDA graph in chunks (lbs_set_graph_chunk).
 * Returns LBS_EUNSTABLE if an earlier monitor already found a non-finite
 * value; the state then stays available for lbs_fields. */
int lbs_step(lbs_handle *h, int64_t n);

/* Wait for the handle's work; LBS_EUNSTABLE if a monitor found a
 * non-finite value (lbs_unstable_iteration tells where), LBS_ETIMEOUT if a
 * kernel gave up waiting for its tile copies (bounded wait; the state is then
 * not advanced for the affected tiles). */
int lbs_sync(lbs_handle *h);

/* Fields at the current iteration into caller-owned HOST buffers (any may be
 * NULL): u, the velocity v = j / rho0 with j = sum_q c_q f_q + dt/2 S (the
 * momentum of Alg. 1 at the current time) and P(H(u)).  The fields are staged
 * in the state buffers the next iteration overwrites (in more than one pass
 * when they do not fit at once; a field that fits nowhere, P under
 * LBS_FP16S, gets a temporary device buffer); the state itself is untouched.
 * Synchronous. */
int lbs_fields(lbs_handle *h, double *u, double *v, double *P);

/* As lbs_fields into caller-owned DEVICE buffers; asynchronous. */
int lbs_fields_device(lbs_handle *h, double *u, double *v, double *P);

/* As lbs_fields, but never allocating device memory.  (The paper has no
 * counterpart; this is a property of the library.)  lbs_fields stages the
 * output in the handle's idle state buffers and allocates a device
 * temporary the size of the lattice for a field that does not fit there
 * (P under LBS_FP16S).  Some callers cannot allow even that: a process
 * whose device memory is already taken (a server whose resident lattices
 * fill its HBM budget, or a framework's caching allocator holding most of
 * the free memory) would get LBS_ENOMEM for exactly the large lattices whose
 * results matter, and a caller with a latency budget cannot afford cudaFree,
 * which waits for the whole device.  This entry point instead copies the fields
 * out a block of rows at a time through one fixed staging array of 8 MiB
 * (2^20 doubles) in device memory, a file-scope static that every GPU which
 * loads the library holds until the process exits.  It calls no cudaMalloc
 * or cudaFree.
 *  - Limit: one row of the requested fields must fit the array, i.e.
 *    (2 [u] + 2 [v] + 4 [P]) * nx <= 2^20 doubles (nx <= 131072 with all
 *    three); larger rows are rejected with LBS_EINVAL.
 *  - The first call on a device (with that device current, as for every
 *    call on the handle) looks up the array's device address; make that
 *    first call before any stream capture.  After a device reset the next
 *    call looks it up again (the address belongs to the destroyed context).
 *  - On an error the call still waits for the copies it queued before
 *    returning, so no host buffer is written after it returns.
 *  - Every call on a device shares the one array, which keeps the last
 *    call's contents; each call overwrites every entry it copies out, so
 *    nothing needs clearing.  Calls that overlapped on the GPU would race on
 *    it: the library serialises calls with a process-wide lock and each call
 *    returns only after its copies finished, so they do not overlap.
 * Host buffers and layouts as lbs_fields (any may be NULL); synchronous. */
int lbs_fields_static(lbs_handle *h, double *u, double *v, double *P);

/* Displacements of n probe nodes idx[i] = y * nx + x into host out[2 n].
 * Synchronous. */
int lbs_probe(lbs_handle *h, int32_t n, const int32_t *idx, double *out);

/* Run the monitor reduction now (synchronous). */
int lbs_monitor(lbs_handle *h, lbs_monitors *out);

/* Grid error norms of the current displacement u against a reference field
 * u_ref (Sect. 4, Eq. griderror): with du = u - u_ref over the n = nx * ny
 * nodes, ||a||_2 = sqrt(sum_nodes a . a) and ||a||_inf = max over nodes of
 * max(|a_1|, |a_2|),
 *   out[0] = E2   = ||du||_2 / (n ||u_ref||_2),
 *   out[1] = Einf = ||du||_inf / ||u_ref||_2
 * (the norm in the denominators is the reference's).  u_ref: caller-owned,
 * [ny][nx][2] doubles like lbs_fields' u; lbs_grid_error takes it in host
 * memory (staged in the idle state buffers; a temporary only if they cannot
 * hold it), lbs_grid_error_device in device memory.  A deterministic
 * reduction on the handle's stream; synchronous.  LBS_EINVAL for null
 * arguments. */
int lbs_grid_error(lbs_handle *h, const double *u_ref, double out[2]);
int lbs_grid_error_device(lbs_handle *h, const double *u_ref, double out[2]);

/* Monitor every m iterations inside lbs_step (0 disables; default 1000).
 * A non-finite value makes later lbs_step / lbs_sync calls return
 * LBS_EUNSTABLE. */
int lbs_set_monitor_interval(lbs_handle *h, int64_t m);

/* Iterations per captured CUDA graph (even, >= 2; 0 launches directly).
 * Default 64. */
int lbs_set_graph_chunk(lbs_handle *h, int32_t k);

/* Kernel tile variant (an index from lbs_tile_variants).  Each precision has a
 * default (the fastest on a large lattice); lbs_autotune picks per lattice. */
int lbs_set_variant(lbs_handle *h, int32_t variant);

/* ---- checkpoint / resume (no counterpart in the paper) ------------------
 * A checkpoint is the state one iteration of Alg. 1 starts from: the
 * distributions g, the displacement u and the boundary side array (N of the
 * wall nodes), in the handle's storage precision, plus the iteration count and
 * the lattice's parameters.  Resuming from it reproduces, bitwise, the
 * iterations the saved handle would have run.
 *
 * lbs_checkpoint_bytes: size of the checkpoint of this handle (0 for NULL).
 * lbs_save: waits for the handle's stream, then copies the state into
 *   caller-owned host memory buf of at least that many bytes.  Errors:
 *   LBS_EINVAL (NULL, buffer too small), LBS_EUNSTABLE / LBS_ETIMEOUT (as
 *   lbs_sync), LBS_ECUDA.
 * lbs_load: replaces the handle's state (and iteration count) with a
 *   checkpoint taken from a handle created with the same lattice, material,
 *   boundary set-up and precision (LBS_EINVAL otherwise, or for a truncated
 *   buffer); clears the unstable flag; LBS_ECUDA on copy failure. */
size_t lbs_checkpoint_bytes(const lbs_handle *h);
int lbs_save(lbs_handle *h, void *buf, size_t bytes);
int lbs_load(lbs_handle *h, const void *buf, size_t bytes);

/* Self-test of the bounded waits (no counterpart in the paper).  The TMA step
 * kernels wait on an mbarrier for their tile copies with a bounded number of
 * polls and report LBS_ETIMEOUT (through lbs_sync) instead of hanging.  This
 * launches one block that arms an mbarrier for tx_bytes of transfer that is
 * never issued (tx_bytes = 0: none expected, so the barrier completes at
 * once) and polls it at most `polls` times with the same helper; *timed_out
 * receives 1 if the wait ran out, 0 if the barrier completed, and *seconds
 * (if not NULL) the wall time of the call.  The GPU context stays usable.
 * Synchronous; allocates a 4-byte flag.  Errors: LBS_EINVAL (tx_bytes >=
 * 2^20, polls == 0, timed_out NULL), LBS_ECUDA. */
int lbs_selftest_bounded_wait(uint32_t tx_bytes, uint32_t polls, int32_t *timed_out, double *seconds);

/* The handle's current tile variant (LBS_EINVAL for a null handle). */
int32_t lbs_variant(const lbs_handle *h);

int64_t lbs_iteration(const lbs_handle *h);
/* first iteration at which a monitor saw a non-finite value, or -1 */
int64_t lbs_unstable_iteration(const lbs_handle *h);
/* 1 if nu exceeds the first-order-boundary CFL bound c_d <= c (nu > 1/4) */
int lbs_cfl_warning(const lbs_handle *h);
/* device bytes of the handle's state */
size_t lbs_device_bytes(const lbs_handle *h);
/* kernels launched for this handle so far, counting every kernel node of a
 * replayed CUDA graph */
int64_t lbs_launch_count(const lbs_handle *h);

/* ---- host utilities (no GPU needed) ------------------------------------ */

/* mu, lam, c_s, c, dt of a configuration (out[5]).  LBS_EINVAL on bad input. */
int lbs_params(const lbs_lattice *lat, const lbs_material *mat, double out[5]);

/* Device bytes lbs_create would allocate for this lattice. */
size_t lbs_footprint(const lbs_lattice *lat);

/* First Piola-Kirchhoff stress P(H) and the constitutive source tensor
 * N(H) = P(H) + Pi(H), Pi(H) = -mu (H + H^T + tr H I) (Eq. source), evaluated
 * on the host with the same formulas the kernels use (double precision).
 * H, P, N: row-major 2x2. */
int lbs_constitutive(int32_t model, double lam, double mu, const double H[4], double P[4], double N[4]);

/* Number of tile variants compiled for a precision, and their shapes
 * (cells along x and y per thread block).  tx and ty (caller-owned) receive
 * *count entries each; pass NULL for both to learn the count first.
 * Errors: LBS_EINVAL for an unknown precision. */
int lbs_tile_variants(int32_t precision, int32_t *count, int32_t *tx, int32_t *ty);

/* 1 if a tile variant stages its interior tiles in shared memory with TMA
 * (cp.async.bulk.tensor), 0 if it reads global memory directly; negative
 * LBS_EINVAL for an unknown precision or variant. */
int lbs_tile_variant_kind(int32_t precision, int32_t variant);

/* Name of the kernel that updates a variant's interior tiles (a static
 * string: "step_interior_kernel", "step_tma_kernel", "step_tma2_kernel" or
 * "step_march_kernel"; frame tiles always go to "step_edge_kernel"), or NULL
 * for an unknown precision or variant. */
const char *lbs_tile_variant_name(int32_t precision, int32_t variant);

/* ---- autotuner ---------------------------------------------------------- */

/* Time every tile variant (lbs_tile_variants) for this configuration on a
 * scratch lattice with the same material, edges and precision and at most
 * 4096 x 4096 nodes (direct launches, CUDA events, `steps` iterations after
 * two untimed ones) and return the fastest in *best.  ms, if not NULL,
 * receives the time per iteration of each variant (caller-owned, as many
 * entries as lbs_tile_variants reports for the precision).  Results are cached per
 * (nx, ny, precision, model, periodic axes) for the life of the process;
 * a cached configuration is not timed again.  Allocates a scratch lattice. */
int lbs_autotune(const lbs_lattice *lat, const lbs_material *mat, const lbs_bcs *bcs, int32_t steps, int32_t *best,
                 float *ms);

/* Tune (or look up) the handle's configuration and select the winner. */
int lbs_autotune_handle(lbs_handle *h, int32_t steps);

/* Save / load the tuning cache as JSON lines
 * {"nx": .., "ny": .., "precision": .., "model": .., "per_x": .., "per_y": .., "variant": .., "ms": [..]}.
 * Loading merges into the cache (unknown variants are ignored). */
int lbs_autotune_save(const char *path);
int lbs_autotune_load(const char *path);

/* Install the device allocator used for handle state (NULL, NULL restores
 * cudaMalloc/cudaFree).  alloc(bytes, stream, ctx) returns a device pointer
 * aligned to 256 bytes, or NULL; release(ptr, stream, ctx) frees it.  A block
 * that is not so aligned is released again and lbs_create fails with
 * LBS_ENOMEM.  Affects handles created afterwards. */
typedef void *(*lbs_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*lbs_free_fn)(void *ptr, void *stream, void *ctx);
int lbs_set_allocator(lbs_alloc_fn alloc, lbs_free_fn release, void *ctx);

/* Static description of an LBS_* code ("unknown error" for others). */
const char *lbs_strerror(int code);
/* Message of the last failure in the calling thread (thread-local; valid
 * until that thread's next failing call), "" if none. */
const char *lbs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBS_H */
