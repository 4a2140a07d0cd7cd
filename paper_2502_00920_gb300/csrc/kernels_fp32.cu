// FP32 storage and arithmetic, u as a float pair: kernel instantiations and launchers of liblbs.
#include "lbs_device.cuh"
#include "lbs_batch.cuh"

namespace lbs {
namespace {
using P = F32;
// tile variants (nodes along x, nodes along y, thread rows)
using V0 = Cfg<P, 32, 16, 8>;
using V1 = Cfg<P, 32, 8, 8>;
using V2 = Cfg<P, 64, 8, 4>;
using V3 = Cfg<P, 32, 24, 8>;
using V4 = Cfg<P, 32, 16, 8>;
using M6 = MarchCfg<V4, 8, 128, 2>;
using V8 = Cfg<P, 32, 32, 8>;
using V9 = Cfg<P, 32, 16, 16>;  // one node per thread, 512 threads
// 0-3: V0-V3 tiles read from global memory; 4: V4 tiles staged by TMA;
// 5: V4 tiles, persistent blocks with a two-stage TMA ring; 6: row-marching
// strips over the V4 tile columns; 7: V3 tiles staged by TMA; 8: V8 tiles
// (four nodes per thread) read from global memory; 9: two fused iterations per
// launch on V9 tiles (periodic lattices; one V0 iteration per call otherwise).
constexpr int kVariants = 10;

TileShape shape(int v) {
  switch (v) {
    case 1: return {V1::TX, V1::TY};
    case 2: return {V2::TX, V2::TY};
    case 3:
    case 7: return {V3::TX, V3::TY};
    case 4:
    case 5:
    case 6: return {V4::TX, V4::TY};
    case 8: return {V8::TX, V8::TY};
    case 9: return {V9::TX, V9::TY};
    default: return {V0::TX, V0::TY};
  }
}

const char *name(int v) {
  switch (v) {
    case 4: return "step_tma_kernel";
    case 5: return "step_tma2_kernel";
    case 6: return "step_march_kernel";
    case 7: return "step_tma_kernel";
    case 9: return "step_fused2_tma_kernel";
    default: return "step_interior_kernel";
  }
}

cudaError_t step(const Params &p, const StepPtrs &s, int v, cudaStream_t st) {
  switch (v) {
    case 1: return launch_step<V1>(p, s, st);
    case 2: return launch_step<V2>(p, s, st);
    case 3: return launch_step<V3>(p, s, st);
    case 4: return launch_step_tma<V4>(p, s, st);
    case 5: return launch_step_tma2<V4>(p, s, st);
    case 6: return launch_step_march<V4, M6>(p, s, st);
    case 7: return launch_step_tma<V3>(p, s, st);
    case 8: return launch_step<V8>(p, s, st);
    case 9: return fused2_applies(p) ? launch_step_fused2<V9>(p, s, st) : launch_step<V0>(p, s, st);
    default: return launch_step<V0>(p, s, st);
  }
}

int kernels_per_step(const Params &p, int v) {
  switch (v) {
    case 1: return step_kernel_count<V1>(p);
    case 2: return step_kernel_count<V2>(p);
    case 3:
    case 7: return step_kernel_count<V3>(p);
    case 4:
    case 5:
    case 6: return step_kernel_count<V4>(p);
    case 8: return step_kernel_count<V8>(p);
    case 9: {
      if (!fused2_applies(p)) return step_kernel_count<V0>(p);
      const int ntx = (p.nx + V9::TX - 1) / V9::TX, nty = (p.ny + V9::TY - 1) / V9::TY;
      int a_lo, a_hi, b_lo, b_hi;
      interior_range_m(p.nx, p.ny, V9::TX, V9::TY, 6, a_lo, a_hi, b_lo, b_hi);
      const int ni = (a_hi - a_lo) * (b_hi - b_lo);
      return (ni > 0 ? 1 : 0) + (ntx * nty > ni ? 1 : 0);
    }
    default: return step_kernel_count<V0>(p);
  }
}

int iterations_per_call(const Params &p, int v) { return v == 9 && fused2_applies(p) ? 2 : 1; }

bool tma_maps(const Params &p, int v, const void *g, const void *u, void *og, void *ou) {
  if (v == 9) return make_fused2_maps<V9>(p, g, u, og, ou);
  if (v == 6) return make_march_maps<V4, M6>(p, g, u, og, ou);
  if (v == 7) return make_tma_maps<V3>(p, g, u, og, ou);
  if (v != 4 && v != 5) return false;
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
                      (1 << 4) | (1 << 5) | (1 << 6) | (1 << 7) | (1 << 9),
                      4,  // default: the fastest on the 16384^2 roofline lattice
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

const Launchers &launchers_fp32() { return kL; }

}  // namespace lbs
