/*
 * lbs_serve.h - continuous-batching server of liblbs (see lbs.h).
 *
 * Many independent simulations (lattices of different sizes, materials and
 * boundary loads; each one Algorithm 1 of the paper from rest for a given
 * number of iterations) share one GPU.  A worker thread admits queued
 * requests while their device footprint (lbs_footprint) fits the HBM budget,
 * keeps the admitted lattices' state resident, and advances all of them
 * together: every iteration launches batched kernels that walk tile tables
 * spanning all resident lattices (interior tiles, frame tiles); once per
 * chunk one launch evaluates the edges' prescribed values of every lattice for
 * the chunk's iterations and one advances their iteration counters.  The
 * worker runs `chunk`
 * iterations between scheduling points; a lattice that reaches
 * its iteration count stops (its tiles return at once), is checked for
 * non-finite values, has u, v and P copied to host memory owned by the server
 * and its device memory released, after which queued requests are admitted.
 * Host work overlaps the GPU's: the worker launches a chunk and, while it
 * runs, creates the handles of newly admitted requests and finishes the
 * lattices that left the batch after the previous chunk; it waits for the
 * chunk only then.
 * Every 1000 iterations (at the next scheduling point) each resident lattice
 * is also checked for non-finite values; one that has some is retired at once
 * as LBS_EUNSTABLE, like a handle whose monitor saw them.
 *
 * Preemption (preempt_after_s > 0; no counterpart in the paper).  When the
 * request at the head of the queue has waited preempt_after_s seconds and its
 * footprint does not fit, resident lattices are swapped out to make room: those
 * resident for at least preempt_after_s, the most remaining iterations first,
 * and only lattices with more remaining iterations than the waiting request.
 * A swapped-out lattice's state goes to host memory owned by the server
 * (lbs_save), its device memory is released and it rejoins the queue at the
 * back; on re-admission it resumes from that state (lbs_load), so its result
 * is bitwise the one it would have had without the interruption.  Nothing is
 * swapped out unless the waiting request then fits.
 * Each lattice computes exactly what lbs_step computes for it alone, with
 * either wall reading (lbs_lattice.wall_extrap) and any mix of the two.
 *
 * Batch tile shapes (no counterpart in the paper).  The batched kernels come
 * in the four global-memory tile shapes of lbs_tile_variants (0..3), which
 * compute every node with the same operations.  Unless batch_shape fixes
 * one, the worker times them: a trial runs one chunk on each candidate
 * shape (real work, not a rehearsal) and keeps the one with the most node
 * updates per second of device time.  The first trial takes all four; a new
 * trial starts when the resident node count has halved or doubled since the
 * last, and takes the two fastest of the previous one.  Results do not
 * depend on the shape.
 *
 * The server owns its device memory and its results until lbs_result hands
 * them over.  All functions are thread-safe.
 */
#ifndef LBS_SERVE_H
#define LBS_SERVE_H

#include "lbs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbs_server lbs_server;

typedef struct {
  size_t hbm_budget;     /* device bytes for resident lattices (0: 80 % of free memory) */
  int32_t precision;     /* storage precision of every request (LBS_FP32 ...)          */
  int32_t chunk;         /* iterations between scheduling points (0: 64)               */
  int32_t max_resident;  /* cap on resident lattices (0: none)                          */
  int32_t queue_limit;   /* lbs_submit returns LBS_EBUSY beyond this many queued (0: none) */
  double preempt_after_s; /* > 0: preemption, below (0: never; < 0: LBS_EINVAL)           */
  int32_t batch_shape;   /* 0: batch tile shape picked by timing, below; k >= 1: always
                            shape k - 1 (lbs_tile_variants' global-memory tiles 0..3)    */
} lbs_server_config;

enum { LBS_TICKET_QUEUED = 0, LBS_TICKET_RUNNING = 1, LBS_TICKET_DONE = 2, LBS_TICKET_FAILED = 3 };

typedef struct {
  int32_t state;       /* LBS_TICKET_*                                           */
  int32_t error;       /* LBS_OK, or why it failed (LBS_EUNSTABLE, LBS_ENOMEM ...) */
  int64_t iterations;  /* iterations completed                                    */
  int64_t nsteps;      /* iterations requested                                    */
  int32_t nx, ny;
  double t_submit;     /* seconds on the server clock (0 = server creation)       */
  double t_admit;      /* admission to the GPU (-1 while queued)                  */
  double t_done;       /* completion (-1 until done or failed)                    */
  size_t device_bytes; /* footprint while resident                                */
  int64_t swaps;       /* times it was swapped out by preemption                  */
} lbs_ticket_info;

typedef struct {
  int64_t submitted, completed, failed, queued, resident;
  int64_t node_updates;   /* nodes x iterations of finished lattices          */
  double busy_seconds;    /* wall time with at least one resident lattice      */
  size_t bytes_in_use;    /* device bytes of resident lattices                 */
  size_t hbm_budget;
  int64_t launches;       /* kernels launched by the worker                    */
  int64_t preemptions;    /* lattices swapped out to host memory               */
  int32_t batch_shape;    /* current batch tile shape (0..3)                   */
  int32_t batch_tx, batch_ty; /* its nodes along x and y                       */
  int64_t batch_tunings;  /* completed timing trials of the shapes             */
} lbs_server_stats;

/* Start a server on the current CUDA device.  Errors: LBS_EINVAL (bad
 * precision or negative sizes), LBS_ECUDA. */
int lbs_server_create(const lbs_server_config *cfg, lbs_server **out);

/* Queue a simulation from rest for nsteps iterations.  The precision of the
 * lattice is replaced by the server's.  *ticket identifies it.  Errors:
 * LBS_EINVAL (as lbs_create), LBS_ENOMEM (larger than the whole budget),
 * LBS_EBUSY (queue limit). */
int lbs_submit(lbs_server *s, const lbs_lattice *lat, const lbs_material *mat, const lbs_bcs *bcs, int64_t nsteps,
               uint64_t *ticket);

/* Status of a ticket.  LBS_ENOTFOUND for unknown or already collected tickets. */
int lbs_poll(lbs_server *s, uint64_t ticket, lbs_ticket_info *info);

/* Block until the ticket is done or failed, at most timeout_s seconds
 * (< 0: no limit).  LBS_ETIMEOUT if the time ran out. */
int lbs_wait(lbs_server *s, uint64_t ticket, double timeout_s);

/* Copy the final fields of a finished ticket into caller-owned host buffers
 * (layouts as lbs_fields; any may be NULL) and forget the ticket.  Returns
 * the ticket's error code for a failed ticket (its fields as they stood when
 * it stopped are still copied), LBS_EBUSY if it is not finished. */
int lbs_result(lbs_server *s, uint64_t ticket, double *u, double *v, double *P);

/* Cancel a ticket (no counterpart in the paper).  A queued request (also one
 * swapped out by preemption) leaves the queue at once; a running one stops at
 * the worker's next scheduling point, its fields as they stood then kept for
 * lbs_result, and its device memory is released.  Either way the ticket ends
 * failed with LBS_ECANCELED.  Cancelling a ticket that has already ended
 * changes nothing.  Errors: LBS_ENOTFOUND. */
int lbs_cancel(lbs_server *s, uint64_t ticket);

/* Block until every submitted ticket is done or failed (timeout as lbs_wait). */
int lbs_server_drain(lbs_server *s, double timeout_s);

int lbs_server_get_stats(lbs_server *s, lbs_server_stats *out);

/* Stop the worker (after the iteration chunk in flight), free everything. */
int lbs_server_destroy(lbs_server *s);

#ifdef __cplusplus
}
#endif
#endif /* LBS_SERVE_H */
