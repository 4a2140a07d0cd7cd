// Batched step kernels of liblbs's server: persistent walks over a tile table
// spanning many resident lattices (each tile runs step_tile of
// lbs_device.cuh on its own lattice's buffers), and their launcher.  Included
// by kernels_fp64.cu / kernels_fp32.cu / kernels_fp16.cu after lbs_device.cuh.
#pragma once
#include "lbs_device.cuh"

namespace lbs {

// ------------------------------------------------------------------ batches
// A persistent-style walk over a tile table spanning many lattices of
// different sizes: block i takes tiles i, i + grid, ...  Each tile runs the
// same step_tile code as the single-lattice kernels, on its lattice's buffers
// chosen by the parity of that lattice's iteration k + it (k: its iteration at
// the start of the chunk, it: this launch's place in the chunk).
// SPLIT (frame tiles only): each table tile is run as CPT tiles of one node
// per thread.
template <class C, bool EDGE, bool LIN, bool SPLIT>
__device__ __forceinline__ void batch_walk(const BatchLattice *lats, const BatchTile *tiles, int ntiles, int it,
                                           int *err) {
  using H = typename FrameCfg<C, SPLIT>::type;
  constexpr int parts = C::TY / H::TY;
  __shared__ Params sP;
  __shared__ StepPtrs sS;
  __shared__ BatchTile sT;
  __shared__ int skip;
  static_assert(sizeof(Params) % 8 == 0, "the tile header is copied in 8-byte words");
  for (int t = blockIdx.x; t < ntiles * parts; t += gridDim.x) {
    // the tile's lattice header, read by the first warp: every lane reads the
    // entry and the counters (one broadcast each) and copies a share of the
    // parameters, so the copy costs one round trip instead of one per word
    if (threadIdx.x < 32) {
      const BatchTile T = tiles[t / parts];
      const BatchLattice &L = lats[T.lat];
      const bool sk = L.k + it >= L.kend;
      if (!sk)
        for (int w = threadIdx.x; w < (int)(sizeof(Params) / 8); w += 32)
          ((long long *)&sP)[w] = ((const long long *)&L.P)[w];
      if (threadIdx.x == 0) {
        skip = sk;
        sT = T;
      }
      if (threadIdx.x == 0 && !sk) {
        const int p = (int)((L.k + it) & 1);
        sS.g_in = L.g[p];
        sS.g_out = L.g[p ^ 1];
        sS.u_in = L.u[p];
        sS.u_out = L.u[p ^ 1];
        sS.b_in = L.b[p];
        sS.b_out = L.b[p ^ 1];
        sS.kptr = &lats[T.lat].k;
        sS.koff = it;
        sS.tm_g = sS.tm_u = nullptr;
        sS.err = err;
        sS.fork = nullptr;
        sS.sev = L.sev ? L.sev + (size_t)it * 8 : nullptr;
      }
    }
    __syncthreads();
    if (!skip) step_tile<H, EDGE, LIN>(sP, sS, sT.a * C::TX, sT.b * C::TY + (t % parts) * H::TY);
    __syncthreads();  // the next tile reuses the shared memory
  }
}

template <class C, bool EDGE, bool LIN = false, bool SPLIT = false>
__global__ void __launch_bounds__(FrameCfg<C, SPLIT>::type::NT) batch_step_kernel(const BatchLattice *lats,
                                                                                  const BatchTile *tiles, int ntiles,
                                                                                  int it, int *err) {
  batch_walk<C, EDGE, LIN, SPLIT>(lats, tiles, ntiles, it, err);
}

// The same walks held to more blocks per SM (single precision): a batch tile
// waits on the latency of its global loads, and another block per SM hides
// more of it than the registers it gives up cost.  Interior tiles: four
// blocks (64 registers, no spills); frame tiles with own wall values: three
// (80 registers).  The FP16-storage and FP64 code would spill.
template <class C>
__global__ void __launch_bounds__(C::NT, 4) batch_interior4_kernel(const BatchLattice *lats, const BatchTile *tiles,
                                                                   int ntiles, int it, int *err) {
  batch_walk<C, false, false, false>(lats, tiles, ntiles, it, err);
}
template <class C>
__global__ void __launch_bounds__(C::NT, 3) batch_frame3_kernel(const BatchLattice *lats, const BatchTile *tiles,
                                                                int ntiles, int it, int *err) {
  batch_walk<C, true, false, false>(lats, tiles, ntiles, it, err);
}

// resident blocks of a batch kernel on this device
template <class C>
int batch_resident(void (*kernel)(const BatchLattice *, const BatchTile *, int, int, int *)) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, C::NT, 0);
  return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
}

// launch `it` of a chunk: the interior tiles and the frame tiles of every
// unfinished lattice at its iteration k + it
template <class C>
cudaError_t launch_batch_step(BatchLattice *lats, int nlats, const BatchTile *interior, int ni, const BatchTile *edge,
                              int ne, const BatchTile *edge_lin, int nl, int it, int *err, cudaStream_t st,
                              const StreamFork *fork) {
  using KFn = void (*)(const BatchLattice *, const BatchTile *, int, int, int *);
  // single precision: the interior and own-value frame walks held to four
  // and three blocks per SM (the other precisions would spill)
  KFn ki, kf;
  if constexpr (sizeof(typename C::gs) == 4 && sizeof(typename C::real) == 4) {
    ki = batch_interior4_kernel<C>;
    kf = batch_frame3_kernel<C>;
  } else {
    ki = batch_step_kernel<C, false>;
    kf = batch_step_kernel<C, true>;
  }
  const KFn kl = batch_step_kernel<C, true, true>;
  // resident blocks of each persistent walk (computed once; the
  // initialisation of a function-local static is thread-safe)
  static const int bi = batch_resident<C>(ki), bf = batch_resident<C>(kf), bl = batch_resident<C>(kl);
  // the frame tiles (few, long, latency-bound) run beside the interior tiles
  // when a side stream is given and the interior walk is short (beside a
  // long persistent walk they would hold back blocks whose tiles are fixed):
  // both read iteration k and write k + 1 of disjoint nodes; the counters
  // advance once both have finished
  const bool split = fork && ni > 0 && ni <= kForkWalk * bi && (ne > 0 || nl > 0);
  // no more frame tiles than SMs: run each as CPT blocks of one node per
  // thread (the frame launch is then the iteration's critical path)
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  auto frame = [&](cudaStream_t fs) {
    if constexpr (C::CPT >= 2) {
      if (ne + nl <= sms) {
        using H = typename FrameCfg<C, true>::type;
        if (ne > 0) batch_step_kernel<C, true, false, true><<<C::CPT * ne, H::NT, 0, fs>>>(lats, edge, ne, it, err);
        if (nl > 0)
          batch_step_kernel<C, true, true, true><<<C::CPT * nl, H::NT, 0, fs>>>(lats, edge_lin, nl, it, err);
        return;
      }
    }
    if (ne > 0) kf<<<ne < bf ? ne : bf, C::NT, 0, fs>>>(lats, edge, ne, it, err);
    if (nl > 0) kl<<<nl < bl ? nl : bl, C::NT, 0, fs>>>(lats, edge_lin, nl, it, err);
  };
  if (split) {
    cudaEventRecord(fork->fork, st);
    cudaStreamWaitEvent(fork->side, fork->fork, 0);
    frame(fork->side);
  }
  if (ni > 0) ki<<<ni < bi ? ni : bi, C::NT, 0, st>>>(lats, interior, ni, it, err);
  if (!split) frame(st);
  if (split) {
    cudaEventRecord(fork->join, fork->side);
    cudaStreamWaitEvent(st, fork->join, 0);
  }
  return cudaGetLastError();
}

}  // namespace lbs
