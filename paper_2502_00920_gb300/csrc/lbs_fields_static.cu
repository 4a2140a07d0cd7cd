// lbs_fields_static: field output without device allocation.
//
// lbs_fields stages u, v and P in the handle's idle state buffers, whole
// fields at a time, and allocates a device temporary for a field that fits
// nowhere there (P under FP16 storage: 8.6 GB for a 16384^2 lattice).  This
// variant stages them through one fixed 8 MiB array in device memory, a row
// block at a time, so a call never allocates.  The kernel is a variant of the
// field-output kernel that writes only the rows of one block.
#include <mutex>

#include "lbs_device.cuh"
#include "lbs_internal.h"

namespace lbs {
namespace {

// staging for the row blocks; every GPU that loads the library holds it
constexpr size_t kStageDoubles = (size_t)1 << 20;  // 8 MiB
static __device__ __align__(256) double g_fields_stage[kStageDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_stage_mu;
// the array's device address per device, with the identifier of the context
// it was looked up in: a device reset destroys that context (and the address
// with it), and the next call looks the address up again in the new one
double *g_stage_ptr[kMaxDevices] = {};
unsigned long long g_stage_ctx[kMaxDevices] = {};

// unique identifier of the calling thread's current context (0 if unknown);
// identifiers are never reused within a process
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static const GetCurrent get_current = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return (GetCurrent)fn;
  }();
  static const GetId get_id = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return (GetId)fn;
  }();
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// u, v, P of rows [y_lo, y_hi) into dense row-block arrays (x fastest)
template <class C>
__global__ void __launch_bounds__(C::NT) fields_rows_kernel(const Params P, const typename C::gs *g,
                                                            const typename C::us *u, int y_lo, int y_hi, double *uo,
                                                            double *vo, double *Po) {
  using R = typename C::real;
  __shared__ typename C::Smem sm;
  const int x0 = blockIdx.x * C::TX, y0 = (y_lo / C::TY + blockIdx.y) * C::TY;
  load_r2_from_state<C>(sm, P, u, x0, y0);
  __syncthreads();
  if (vo || Po) {
    phase_n<C, true>(sm, P, x0, y0, (R *)nullptr);
    __syncthreads();
  }
  const size_t plane = (size_t)P.ny * P.pitch;
  const double cr = P.c / P.rho0, hr = (0.5 * P.dt) / P.rho0;
  const int tx = threadIdx.x % C::TX, ty = threadIdx.x / C::TX;
  for (int i = 0; i < C::CPT; ++i) {
    const int lx = tx, ly = ty + i * C::NTY, x = x0 + lx, y = y0 + ly;
    if (x >= P.nx || y < y_lo || y >= y_hi) continue;
    node_fields<C>(sm, P, g, plane, (size_t)y * P.pitch + x, lx, ly, x, y, (size_t)(y - y_lo) * P.nx + x, cr, hr,
                   uo, vo, Po);
  }
}

template <class Pr>
cudaError_t launch_rows(const Params &P, const void *g, const void *u, int y_lo, int y_hi, double *uo, double *vo,
                        double *Po, cudaStream_t st) {
  using C = Cfg<Pr, 32, 16, 8>;
  const int b_first = y_lo / C::TY, b_last = (y_hi - 1) / C::TY;
  dim3 grid((P.nx + C::TX - 1) / C::TX, b_last - b_first + 1);
  fields_rows_kernel<C><<<grid, C::NT, 0, st>>>(P, (const typename C::gs *)g, (const typename C::us *)u, y_lo, y_hi,
                                                uo, vo, Po);
  return cudaGetLastError();
}

}  // namespace
}  // namespace lbs

extern "C" int lbs_fields_static(lbs_handle *h, double *u, double *v, double *P) {
  using namespace lbs;
  if (!h) {
    set_error("null handle");
    return LBS_EINVAL;
  }
  const int nx = h->P.nx, ny = h->P.ny;
  const int wu = u ? 2 : 0, wv = v ? 2 : 0, wp = P ? 4 : 0;
  const size_t per_row = (size_t)(wu + wv + wp) * nx;
  if (per_row == 0) return LBS_OK;
  if (per_row > kStageDoubles) {
    set_error("lbs_fields_static: one row of " + std::to_string(nx) + " nodes needs " + std::to_string(per_row) +
              " doubles of staging, more than the static 8 MiB array holds (" + std::to_string(kStageDoubles) +
              "); use lbs_fields");
    return LBS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_stage_mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error("lbs_fields_static: no usable current device");
    return LBS_ECUDA;
  }
  // (cudaGetDevice does not create the context; the address lookup below
  // does, so the identifier is taken after it on the first call)
  const unsigned long long ctx = current_context_id();
  if (!g_stage_ptr[dev] || ctx == 0 || ctx != g_stage_ctx[dev]) {
    // the array's name is a host-side stand-in; its device address is looked
    // up once per device (and context), with that device current
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fields_stage);
    if (e != cudaSuccess || !p) {
      set_error(std::string("lbs_fields_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return LBS_ECUDA;
    }
    g_stage_ptr[dev] = (double *)p;
    g_stage_ctx[dev] = current_context_id();
  }
  double *stage = g_stage_ptr[dev];
  // an error after the first launch leaves earlier blocks' copies queued:
  // wait for them while the lock is still held, so that the next call cannot
  // overwrite the array under them and no host buffer is written after the
  // return
  auto fail_queued = [&](const std::string &msg) {
    cudaStreamSynchronize(h->stream);
    set_error(msg);
    return LBS_ECUDA;
  };
  const int rows = (int)(kStageDoubles / per_row);
  for (int y_lo = 0; y_lo < ny; y_lo += rows) {
    const int y_hi = y_lo + rows < ny ? y_lo + rows : ny;
    const size_t n = (size_t)(y_hi - y_lo) * nx;
    double *su = stage, *sv = su + wu * n, *sp = sv + wv * n;
    cudaError_t le;
    if (h->precision == LBS_FP64)
      le = launch_rows<F64>(h->P, h->g[h->parity], h->u[h->parity], y_lo, y_hi, u ? su : nullptr, v ? sv : nullptr,
                            P ? sp : nullptr, h->stream);
    else if (h->precision == LBS_FP32)
      le = launch_rows<F32>(h->P, h->g[h->parity], h->u[h->parity], y_lo, y_hi, u ? su : nullptr, v ? sv : nullptr,
                            P ? sp : nullptr, h->stream);
    else
      le = launch_rows<F16>(h->P, h->g[h->parity], h->u[h->parity], y_lo, y_hi, u ? su : nullptr, v ? sv : nullptr,
                            P ? sp : nullptr, h->stream);
    if (le != cudaSuccess) return fail_queued(std::string("lbs_fields_static: launch: ") + cudaGetErrorString(le));
    h->launches += 1;
    // the next block's kernel follows these copies on the same stream
    if ((u && cudaMemcpyAsync(u + (size_t)2 * y_lo * nx, su, 2 * n * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream) != cudaSuccess) ||
        (v && cudaMemcpyAsync(v + (size_t)2 * y_lo * nx, sv, 2 * n * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream) != cudaSuccess) ||
        (P && cudaMemcpyAsync(P + (size_t)4 * y_lo * nx, sp, 4 * n * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream) != cudaSuccess))
      return fail_queued("lbs_fields_static: copy to host failed");
  }
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
    set_error(std::string("lbs_fields_static: ") + cudaGetErrorString(e));
    return LBS_ECUDA;
  }
  return LBS_OK;
}
