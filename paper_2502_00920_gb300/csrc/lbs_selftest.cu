// Self-test of the bounded waits: a wait on an mbarrier that never completes
// must end by its own bound and report, leaving the GPU context usable.
#include <chrono>

#include "lbs_device.cuh"
#include "lbs_internal.h"

namespace {

// One block: thread 0 arms the barrier for tx_bytes of transfer that no copy
// will deliver (tx_bytes = 0: none, so its arrival completes the phase); every
// thread polls it at most `polls` times with the helper the step kernels use,
// and the block agrees on the outcome as they do.
__global__ void bounded_wait_kernel(uint32_t tx_bytes, uint32_t polls, int *timed_out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    lbs::mbar_init(&bar, 1);
    lbs::mbar_expect_tx(&bar, tx_bytes);
  }
  __syncthreads();
  int ok = 0;
  for (uint32_t i = 0; i < polls; ++i)
    if (lbs::mbar_try_wait(&bar, 0)) {
      ok = 1;
      break;
    }
  if (!__syncthreads_and(ok) && threadIdx.x == 0) *timed_out = 1;
}

}  // namespace

extern "C" int lbs_selftest_bounded_wait(uint32_t tx_bytes, uint32_t polls, int32_t *timed_out, double *seconds) {
  if (!timed_out || polls == 0 || tx_bytes >= (1u << 20)) {
    lbs::set_error("lbs_selftest_bounded_wait: tx_bytes must be < 2^20, polls > 0, timed_out not NULL");
    return LBS_EINVAL;
  }
  int *flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    lbs::set_error("lbs_selftest_bounded_wait: no device memory for the flag");
    return LBS_ECUDA;
  }
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaMemset(flag, 0, sizeof(int));
  if (e == cudaSuccess) {
    bounded_wait_kernel<<<1, 128>>>(tx_bytes, polls, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  cudaFree(flag);
  if (e != cudaSuccess) {
    lbs::set_error(std::string("lbs_selftest_bounded_wait: ") + cudaGetErrorString(e));
    return LBS_ECUDA;
  }
  *timed_out = h;
  return LBS_OK;
}
