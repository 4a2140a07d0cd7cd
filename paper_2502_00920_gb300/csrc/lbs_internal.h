// Host-side declarations shared by the liblbs translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/lbs.h"

namespace lbs {

enum { kLeft = 0, kRight = 1, kBottom = 2, kTop = 3 };

// Per-lattice parameters handed to every kernel by value.  Everything the
// kernels need to know about one lattice: geometry, material, boundary
// edges and the derived coefficients of the scheme.
struct Params {
  int nx, ny, pitch;  // nodes per axis; row pitch in elements (g planes, u rows)
  int per_x, per_y;   // periodic axes
  int blen;           // entries per edge of the boundary side array
  int model;
  int gshift;         // FP16S: stored g = g * 2^gshift
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

// Device pointers of one lattice for one step: in/out buffers of the
// distributions g (9 planes of ny*pitch), the displacement u (one record per
// node) and the boundary side array (4 edges x blen x 4 entries of N = P + Pi(H)).
struct StepPtrs {
  const void *g_in;
  void *g_out;
  const void *u_in;
  void *u_out;
  const void *b_in;
  void *b_out;
  const int64_t *kptr;  // iteration counter base (device)
  int64_t koff;         // iteration = *kptr + koff
};

struct TileShape {
  int tx, ty;
};

// Launchers, one set per precision (kernels_fp*.cu).  `variant` picks a tile
// shape (0 = default).  Return a cudaError_t of the launch.
struct Launchers {
  int nvariants;
  TileShape (*shape)(int variant);
  cudaError_t (*step)(const Params &p, const StepPtrs &s, int variant, cudaStream_t st);
  int (*kernels_per_step)(const Params &p, int variant);
  cudaError_t (*init)(const Params &p, void *g, void *u, void *b, const double *u0, const double *v0,
                      cudaStream_t st);
  cudaError_t (*fields)(const Params &p, const void *g, const void *u, double *uo, double *vo, double *Po,
                        cudaStream_t st);
  cudaError_t (*monitor)(const Params &p, const void *g, const void *u, double *partials, int nblocks,
                         double *out6, cudaStream_t st);
  cudaError_t (*probe)(const Params &p, const void *u, const int32_t *idx, int n, double *out, cudaStream_t st);
  size_t g_elem, u_elem, b_elem;  // bytes per stored g value, per u record, per boundary entry
};

const Launchers &launchers_fp64();
const Launchers &launchers_fp32();
const Launchers &launchers_fp16();

// number of blocks the monitor reduction uses for a lattice
int monitor_blocks(const Params &p);

void set_error(const std::string &msg);

}  // namespace lbs
