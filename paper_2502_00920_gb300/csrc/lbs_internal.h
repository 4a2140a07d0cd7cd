// Host-side declarations shared by the liblbs translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/lbs.h"
#include "lbs_tiles.h"

namespace lbs {

// Per-lattice parameters handed to every kernel by value.  Everything the
// kernels need to know about one lattice: geometry, material, boundary
// edges and the derived coefficients of the scheme.
struct Params {
  int nx, ny, pitch;  // nodes per axis; row pitch in elements (g planes, u rows)
  int per_x, per_y;   // periodic axes
  int blen;           // entries per edge of the boundary side array
  int model;
  int gshift;         // FP16S: stored g = g * 2^gshift
  int extrap;         // Neumann wall values: 0 the boundary node's own, 1 two-point linear
  int etype[4], eshape[4], eunit[4];
  double eamp[4][2], et0[4], et1[4], es[4];
  double mu, lam, rho0, cs, c, dt, dx, tau;
  double body[2];
  // derived coefficients of the scheme (see lbs_api.cu, derive())
  double omega;    // 1 / tau
  double sigma;    // c dt / cs^2
  double kappa;    // c dt / (2 rho0)
  double inv_dx;   // 1 / dx
  double inv_cs2;  // 1 / cs^2
};

// A second stream and two events with which one iteration runs its
// frame-tile launches beside the interior-tile launch (fork, join).
struct StreamFork {
  cudaStream_t side;
  cudaEvent_t fork, join;
};

// Device pointers of one lattice for one step: in/out buffers of the
// distributions g (9 planes of ny*pitch), the displacement u (one record per
// node) and the boundary side array (4 edges x blen x 4 entries of N = P + Pi(H)
// at the wall nodes; under two-point extrapolation a second such layer holds N
// at the nodes one step inwards from each wall).
struct StepPtrs {
  const void *g_in;
  void *g_out;
  const void *u_in;
  void *u_out;
  const void *b_in;
  void *b_out;
  const int64_t *kptr;  // iteration counter base (device)
  int64_t koff;         // iteration = *kptr + koff
  const void *tm_g;     // host pointers to the TMA descriptors of g_in and
  const void *tm_u;     //   u_in (TMA tile variants only)
  int *err;             // device flag set when a bounded wait gives up
  const StreamFork *fork;  // host: run the frame tiles beside the interior tiles (or null)
  const double *sev;    // the four edges' prescribed values at this iteration ([4][2],
                        //   device), or null: the frame tiles evaluate them
};

struct TileShape {
  int tx, ty;
};

// One resident lattice of a batch (device memory): its parameters, both
// buffers of each state array, and its iteration counter and end.
struct BatchLattice {
  Params P;
  void *g[2], *u[2], *b[2];
  int64_t k;     // iteration at the start of the current chunk (launch `it` of the
                 // chunk steps iteration k + it, buffers [(k + it) & 1]); advanced
                 // on the device once per chunk (launch_batch_advance)
  int64_t kend;  // the lattice stops here (its tiles return at once)
  double *sev;   // the edges' prescribed values for the iterations of the chunk,
                 // [it][4][2] (filled once per chunk, launch_batch_edges)
};

// advance every lattice's chunk-start iteration by a chunk of n launches
// (to its end at most); one launch
cudaError_t launch_batch_advance(BatchLattice *lats, int nlats, int n, cudaStream_t st);
cudaError_t launch_batch_edges(BatchLattice *lats, int nlats, int n, cudaStream_t st);

// One tile of a batch: lattice index and tile coordinates (in tiles).
struct BatchTile {
  int lat, a, b;
};



// Launchers, one set per precision (kernels_fp*.cu).  `variant` picks a tile
// shape (0 = default).  Return a cudaError_t of the launch.
struct Launchers {
  int nvariants;
  int tma_mask;   // bit v set: variant v stages its interior tiles by TMA
  int default_variant;
  TileShape (*shape)(int variant);
  const char *(*name)(int variant);  // the interior kernel of a variant, e.g. "step_tma_kernel"
  // one call of a variant: iterations_per_call iterations (2 for the fused
  // two-iteration variant on lattices it applies to, else 1), buffers s.*_in ->
  // s.*_out; kernels_per_step counts the kernels of one call
  cudaError_t (*step)(const Params &p, const StepPtrs &s, int variant, cudaStream_t st);
  int (*kernels_per_step)(const Params &p, int variant);
  int (*iterations_per_call)(const Params &p, int variant);
  // exactly one iteration whatever the variant (global-memory tiles; the
  // last iteration of an odd count under a fused variant); one or two kernels
  cudaError_t (*step1)(const Params &p, const StepPtrs &s, cudaStream_t st);
  int (*kernels_per_step1)(const Params &p);
  // TMA descriptors of one (g, u) buffer pair for a tile variant; returns
  // false if the variant does not use TMA.  out_g/out_u: CUtensorMap storage.
  bool (*tma_maps)(const Params &p, int variant, const void *g, const void *u, void *out_g, void *out_u);
  cudaError_t (*init)(const Params &p, void *g, void *u, void *b, const double *u0, const double *v0,
                      cudaStream_t st);
  cudaError_t (*fields)(const Params &p, const void *g, const void *u, double *uo, double *vo, double *Po,
                        cudaStream_t st);
  cudaError_t (*monitor)(const Params &p, const void *g, const void *u, double *partials, int nblocks,
                         double *out7, int64_t k, cudaStream_t st);
  cudaError_t (*probe)(const Params &p, const void *u, const int32_t *idx, int n, double *out, cudaStream_t st);
  // grid error norms against a device reference field (out3: E2, Einf, ||u_ref||_2)
  cudaError_t (*grid_error)(const Params &p, const void *u, const double *uref, double *partials, int nblocks,
                            double *out3, cudaStream_t st);
  // launch `it` of a chunk: one iteration of every unfinished lattice of a
  // batch, each at its iteration k + it (k: its iteration at the start of the
  // chunk): interior tiles, frame tiles, frame tiles of the lattices with
  // two-point wall extrapolation (their own kernel), on tiles of batch shape
  // `shape` (0 .. nbatch_shapes - 1, global-memory tiles; every shape computes
  // each node with the same operations, so a server may switch between them)
  // (`fork`, if given, runs the frame tiles on its side stream, concurrently
  // with the interior tiles; both have finished when the next launch starts)
  cudaError_t (*batch_step)(int shape, BatchLattice *lats, int nlats, const BatchTile *interior, int ni,
                            const BatchTile *edge, int ne, const BatchTile *edge_lin, int nl, int it, int *err,
                            cudaStream_t st, const StreamFork *fork);
  int nbatch_shapes;
  TileShape (*batch_shape)(int shape);
  size_t g_elem, u_elem, b_elem;  // bytes per stored g value, per u record, per boundary entry
};

const Launchers &launchers_fp64();
const Launchers &launchers_fp32();
const Launchers &launchers_fp16();

// number of blocks the monitor reduction uses for a lattice
int monitor_blocks(const Params &p);

void set_error(const std::string &msg);

// device allocator of a handle (lbs_set_allocator or cudaMalloc)
struct Allocator {
  lbs_alloc_fn alloc;
  lbs_free_fn release;
  void *ctx;
};

}  // namespace lbs

// State of one lattice (the C ABI's opaque lbs_handle).
struct lbs_handle {
  lbs::Params P;
  int precision;
  const lbs::Launchers *L;
  int variant;
  lbs::Allocator alloc;
  cudaStream_t own_stream;
  cudaStream_t stream;
  void *g[2], *u[2], *b[2];
  void *mon_block;          // partials, out[8], counters
  double *mon_partials;
  double *mon_out;          // device: bad, max|u|, mx, my, mass, flag
  int64_t *kdev;            // device iteration base used by graph replays
  int64_t *zero_dev;        // device constant 0 (direct launches)
  double *mon_host;         // pinned copy of mon_out
  cudaEvent_t mon_event;
  bool mon_pending;
  int64_t mon_k;            // iteration of the pending monitor
  int64_t mon_interval, next_mon;
  int parity;               // the current state sits in buffers [parity]
  int64_t k;                // iteration counter
  int64_t kdev_value;       // value held by *kdev (host mirror)
  int64_t unstable_at;
  int graph_chunk;
  cudaGraphExec_t graph[2];
  int graph_variant[2];
  size_t bytes;
  int cfl_warn;
  int64_t launches;         // kernels launched for this handle
  int *errdev;              // device flag: a bounded wait in a kernel gave up
  CUtensorMap tm_g[2];      // TMA descriptors of g[0], g[1] and u[0], u[1]
  CUtensorMap tm_u[2];      //   for the current variant (TMA variants only)
  bool tma;                 // the current variant stages tiles with TMA
  lbs::StreamFork fork;     // side stream and events: frame tiles beside interior tiles
  lbs_lattice lat;          // the configuration the handle was created with
  lbs_material mat;
  lbs_bcs bcs;
};
