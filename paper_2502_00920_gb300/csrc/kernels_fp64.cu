// FP64 storage and arithmetic: kernel instantiations and launchers of liblbs.
#include "lbs_device.cuh"
#include "lbs_batch.cuh"

namespace lbs {
namespace {
using P = F64;
// tile variants (nodes along x, nodes along y, thread rows)
using V0 = Cfg<P, 32, 16, 8>;
using V1 = Cfg<P, 32, 8, 8>;
using V2 = Cfg<P, 64, 8, 4>;
using V3 = Cfg<P, 32, 24, 8>;  // 32x32 would need 57 KB of static shared memory in FP64
using V4 = Cfg<P, 32, 8, 8>;  // interior tiles staged by TMA
constexpr int kVariants = 5;

TileShape shape(int v) {
  switch (v) {
    case 1: return {V1::TX, V1::TY};
    case 2: return {V2::TX, V2::TY};
    case 3: return {V3::TX, V3::TY};
    case 4: return {V4::TX, V4::TY};
    default: return {V0::TX, V0::TY};
  }
}

const char *name(int v) {
  switch (v) {
    case 4: return "step_tma_kernel";
    default: return "step_interior_kernel";
  }
}

cudaError_t step(const Params &p, const StepPtrs &s, int v, cudaStream_t st) {
  switch (v) {
    case 1: return launch_step<V1>(p, s, st);
    case 2: return launch_step<V2>(p, s, st);
    case 3: return launch_step<V3>(p, s, st);
    case 4: return launch_step_tma<V4>(p, s, st);
    default: return launch_step<V0>(p, s, st);
  }
}

int kernels_per_step(const Params &p, int v) {
  switch (v) {
    case 1: return step_kernel_count<V1>(p);
    case 2: return step_kernel_count<V2>(p);
    case 3: return step_kernel_count<V3>(p);
    case 4: return step_kernel_count<V4>(p);
    default: return step_kernel_count<V0>(p);
  }
}

int iterations_per_call(const Params &, int) { return 1; }

bool tma_maps(const Params &p, int v, const void *g, const void *u, void *og, void *ou) {
  if (v != 4) return false;
  return make_tma_maps<V4>(p, g, u, og, ou);
}

// the server's batch tile shapes: the global-memory tiles V0-V3
constexpr int kBatchShapes = 4;
TileShape batch_shape(int b) { return shape(b); }
cudaError_t batch_step(int b, BatchLattice *lats, int nlats, const BatchTile *interior, int ni, const BatchTile *edge,
                       int ne, const BatchTile *edge_lin, int nl, int it, int *err, cudaStream_t st,
                       const StreamFork *fork) {
  switch (b) {
    case 1: return launch_batch_step<V1>(lats, nlats, interior, ni, edge, ne, edge_lin, nl, it, err, st, fork);
    case 2: return launch_batch_step<V2>(lats, nlats, interior, ni, edge, ne, edge_lin, nl, it, err, st, fork);
    case 3: return launch_batch_step<V3>(lats, nlats, interior, ni, edge, ne, edge_lin, nl, it, err, st, fork);
    default: return launch_batch_step<V0>(lats, nlats, interior, ni, edge, ne, edge_lin, nl, it, err, st, fork);
  }
}

const Launchers kL = {kVariants,
                      1 << 4,
                      3,  // default: the fastest on the 16384^2 roofline lattice
                      shape,
                      name,
                      step,
                      kernels_per_step,
                      iterations_per_call,
                      launch_step<V0>,
                      step_kernel_count<V0>,
                      tma_maps,
                      launch_init<V0>,
                      launch_fields<V0>,
                      launch_monitor<V0>,
                      launch_probe<V0>,
                      launch_grid_error<V0>,
                      batch_step,
                      kBatchShapes,
                      batch_shape,
                      sizeof(typename P::gs),
                      sizeof(typename P::us),
                      sizeof(typename P::real)};
}  // namespace

const Launchers &launchers_fp64() { return kL; }

}  // namespace lbs
