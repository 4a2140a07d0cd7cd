// C ABI of liblbs (include/lbs.h): handle life cycle, the CUDA-graph step
// loop, monitors and field output.  All arithmetic of the method runs in the
// kernels of lbs_device.cuh; this file only validates, allocates and launches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>

#include "lbs_device.cuh"
#include "lbs_internal.h"
#include "lbs_trace.h"

namespace lbs {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

// ---- device allocator hook ----------------------------------------------
static std::mutex g_alloc_mu;
static lbs_alloc_fn g_alloc = nullptr;
static lbs_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;



static Allocator current_allocator() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return {g_alloc, g_free, g_alloc_ctx};
}

static void *dev_alloc(const Allocator &a, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  if (a.alloc) {
    void *p = a.alloc(bytes, (void *)st, a.ctx);
    // the kernels make 16-byte vector and tensor-copy accesses from the
    // buffer's base: refuse a block that is not 256-byte aligned
    if (p && ((uintptr_t)p & 255u) != 0) {
      if (a.release) a.release(p, (void *)st, a.ctx);
      lbs::set_error("the installed allocator returned a block that is not 256-byte aligned");
      return nullptr;
    }
    return p;
  }
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void dev_free(const Allocator &a, void *p, cudaStream_t st) {
  if (!p) return;
  if (a.release) a.release(p, (void *)st, a.ctx);
  else cudaFree(p);
}

#define LBS_CK(call)                                                                            \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      lbs::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                       \
      return LBS_ECUDA;                                                                         \
    }                                                                                           \
  } while (0)

static int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

// ---- parameters -----------------------------------------------------------

static bool valid_edge(const lbs_edge &e) {
  if (e.type < LBS_PERIODIC || e.type > LBS_NEUMANN) return false;
  if (e.shape < LBS_CONST || e.shape > LBS_DISP_RAMP) return false;
  if ((e.shape == LBS_LINEAR_RAMP || e.shape == LBS_SIN2_RAMP || e.shape == LBS_HALF_SINE ||
       e.shape == LBS_DISP_RAMP) && !(e.t1 > e.t0))
    return false;
  if (e.shape == LBS_RICKER && !(e.s > 0.0)) return false;
  if (e.shape == LBS_DISP_RAMP && e.type != LBS_DIRICHLET) return false;
  if (e.time_unit != LBS_ITERATIONS && e.time_unit != LBS_TIME) return false;
  return isfinite(e.amp[0]) && isfinite(e.amp[1]);
}

static int validate(const lbs_lattice *lat, const lbs_material *mat, const lbs_bcs *bcs) {
  if (!lat || !mat) return fail(LBS_EINVAL, "null lattice or material");
  if (lat->nx < 3 || lat->ny < 3) return fail(LBS_EINVAL, "nx and ny must be >= 3");
  if ((int64_t)lat->nx * lat->ny > (int64_t)1 << 34) return fail(LBS_EINVAL, "lattice too large");
  if (!(lat->tau > 0.5)) return fail(LBS_EINVAL, "tau must exceed 0.5");
  if (!(lat->dx > 0.0)) return fail(LBS_EINVAL, "dx must be positive");
  if (lat->precision < LBS_FP64 || lat->precision > LBS_FP16S) return fail(LBS_EINVAL, "unknown precision");
  if (lat->gscale_log2 < -30 || lat->gscale_log2 > 30) return fail(LBS_EINVAL, "gscale_log2 out of range");
  if (lat->wall_extrap != LBS_EXTRAP_OWN && lat->wall_extrap != LBS_EXTRAP_LINEAR)
    return fail(LBS_EINVAL, "unknown wall extrapolation");
  if (mat->model < LBS_SVK || mat->model > LBS_LE) return fail(LBS_EINVAL, "unknown material model");
  if (!(mat->E > 0.0) || !(mat->rho0 > 0.0)) return fail(LBS_EINVAL, "E and rho0 must be positive");
  if (!(mat->nu > -1.0 && mat->nu < 0.5)) return fail(LBS_EINVAL, "nu must lie in (-1, 0.5)");
  if (!isfinite(mat->body[0]) || !isfinite(mat->body[1])) return fail(LBS_EINVAL, "body force not finite");
  if (bcs) {
    for (int e = 0; e < 4; ++e)
      if (!valid_edge(bcs->edge[e])) return fail(LBS_EINVAL, "invalid boundary edge " + std::to_string(e));
    if ((bcs->edge[kLeft].type == LBS_PERIODIC) != (bcs->edge[kRight].type == LBS_PERIODIC))
      return fail(LBS_EINVAL, "periodic x edges must pair");
    if ((bcs->edge[kBottom].type == LBS_PERIODIC) != (bcs->edge[kTop].type == LBS_PERIODIC))
      return fail(LBS_EINVAL, "periodic y edges must pair");
  }
  return LBS_OK;
}

// derived parameters (Sect. 3.1, 3.2): plane-strain Lame constants,
// c_s = sqrt(mu/rho0), c = sqrt(3) c_s, dt = dx / c
static void derive(const lbs_lattice *lat, const lbs_material *mat, double out[5]) {
  const double mu = mat->E / (2.0 * (1.0 + mat->nu));
  const double lam = mat->E * mat->nu / ((1.0 + mat->nu) * (1.0 - 2.0 * mat->nu));
  const double cs = sqrt(mu / mat->rho0);
  const double c = sqrt(3.0) * cs;
  out[0] = mu;
  out[1] = lam;
  out[2] = cs;
  out[3] = c;
  out[4] = lat->dx / c;
}

static int pitch_of(int nx) { return (nx + 31) / 32 * 32; }

static const Launchers &launchers_for(int precision) {
  if (precision == LBS_FP64) return launchers_fp64();
  if (precision == LBS_FP32) return launchers_fp32();
  return launchers_fp16();
}

static int auto_gshift(const lbs_lattice *lat, const lbs_material *mat) {
  if (lat->precision != LBS_FP16S) return 0;
  if (lat->gscale_log2 != 0) return lat->gscale_log2;
  // distributions are O(rho0) at strains and speeds of order one; keep the
  // largest well below the half-precision maximum 65504
  return 12 - (int)lround(log2(mat->rho0));
}

static Params make_params(const lbs_lattice *lat, const lbs_material *mat, const lbs_bcs *bcs) {
  Params p;
  memset(&p, 0, sizeof(p));
  p.nx = lat->nx;
  p.ny = lat->ny;
  p.pitch = pitch_of(lat->nx);
  p.blen = lat->nx > lat->ny ? lat->nx : lat->ny;
  p.model = mat->model;
  p.gshift = auto_gshift(lat, mat);
  p.extrap = lat->wall_extrap == LBS_EXTRAP_LINEAR;
  lbs_bcs zero;
  memset(&zero, 0, sizeof(zero));
  for (int e = 0; e < 4; ++e) zero.edge[e].type = LBS_NEUMANN;
  const lbs_bcs *b = bcs ? bcs : &zero;
  for (int e = 0; e < 4; ++e) {
    p.etype[e] = b->edge[e].type;
    p.eshape[e] = b->edge[e].shape;
    p.eunit[e] = b->edge[e].time_unit;
    p.eamp[e][0] = b->edge[e].amp[0];
    p.eamp[e][1] = b->edge[e].amp[1];
    p.et0[e] = b->edge[e].t0;
    p.et1[e] = b->edge[e].t1;
    p.es[e] = b->edge[e].s;
  }
  p.per_x = p.etype[kLeft] == LBS_PERIODIC;
  p.per_y = p.etype[kBottom] == LBS_PERIODIC;
  double d[5];
  derive(lat, mat, d);
  p.mu = d[0];
  p.lam = d[1];
  p.cs = d[2];
  p.c = d[3];
  p.dt = d[4];
  p.dx = lat->dx;
  p.tau = lat->tau;
  p.rho0 = mat->rho0;
  p.body[0] = mat->body[0];
  p.body[1] = mat->body[1];
  p.omega = 1.0 / lat->tau;
  p.inv_cs2 = 1.0 / (p.cs * p.cs);
  p.sigma = p.c * p.dt * p.inv_cs2;
  p.kappa = p.c * p.dt / (2.0 * p.rho0);
  p.inv_dx = 1.0 / lat->dx;
  return p;
}

int monitor_blocks(const Params &p) {
  const int64_t n = (int64_t)p.nx * p.ny;
  int64_t b = (n + kMonThreads - 1) / kMonThreads;
  return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}

// sizes of the per-handle device buffers
struct Sizes {
  size_t g, u, b, mon;
};
static Sizes sizes_of(const Params &p, const Launchers &L) {
  Sizes s;
  s.g = (size_t)9 * p.ny * p.pitch * L.g_elem;
  s.u = (size_t)p.ny * p.pitch * L.u_elem;
  s.b = (size_t)(p.extrap ? 2 : 1) * 4 * p.blen * 4 * L.b_elem;
  s.mon = (size_t)monitor_blocks(p) * 5 * sizeof(double) + 8 * sizeof(double) + 3 * sizeof(int64_t);
  return s;
}

// Device room for host transfers without allocating: the g and u buffers of
// the parity the state is not in.  The next iteration overwrites them without
// reading them, so set_initial stages u0, v0 there and fields stages its
// outputs there.  Blocks are handed out 256-byte aligned.
struct Scratch {
  char *base[2];
  size_t cap[2], used[2];
};
static Scratch scratch_of(const lbs_handle *h, int parity) {
  const Sizes sz = sizes_of(h->P, *h->L);
  return Scratch{{(char *)h->g[parity], (char *)h->u[parity]}, {sz.g, sz.u}, {0, 0}};
}
static double *scratch_take(Scratch &s, size_t bytes) {
  for (int i = 0; i < 2; ++i)
    if (s.used[i] <= s.cap[i] && s.cap[i] - s.used[i] >= bytes) {
      char *p = s.base[i] + s.used[i];
      s.used[i] += (bytes + 255) / 256 * 256;
      return (double *)p;
    }
  return nullptr;
}

__global__ void set_counter_kernel(int64_t *k, int64_t v) { *k = v; }
__global__ void add_counter_kernel(int64_t *k, int64_t d) { *k += d; }

}  // namespace lbs

using namespace lbs;



namespace {

StepPtrs ptrs(const lbs_handle *h, int parity, const int64_t *kptr, int64_t koff) {
  StepPtrs s;
  s.g_in = h->g[parity];
  s.g_out = h->g[parity ^ 1];
  s.u_in = h->u[parity];
  s.u_out = h->u[parity ^ 1];
  s.b_in = h->b[parity];
  s.b_out = h->b[parity ^ 1];
  s.kptr = kptr;
  s.koff = koff;
  s.tm_g = h->tma ? (const void *)&h->tm_g[parity] : nullptr;
  s.tm_u = h->tma ? (const void *)&h->tm_u[parity] : nullptr;
  s.err = h->errdev;
  s.fork = h->fork.side ? &h->fork : nullptr;
  s.sev = nullptr;
  return s;
}

void drop_graphs(lbs_handle *h) {
  for (int i = 0; i < 2; ++i) {
    if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
    h->graph[i] = nullptr;
  }
}

int capture_graph(lbs_handle *h, int parity) {
  cudaGraph_t graph = nullptr;
  LBS_CK(cudaStreamBeginCapture(h->own_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  // graph_chunk iterations: calls of iterations_per_call iterations each
  const int its = h->L->iterations_per_call(h->P, h->variant);
  for (int i = 0; i < h->graph_chunk / its && err == cudaSuccess; ++i)
    err = h->L->step(h->P, ptrs(h, parity ^ (i & 1), h->kdev, (int64_t)i * its), h->variant, h->own_stream);
  if (err == cudaSuccess) {
    add_counter_kernel<<<1, 1, 0, h->own_stream>>>(h->kdev, h->graph_chunk);
    err = cudaGetLastError();
  }
  cudaError_t e2 = cudaStreamEndCapture(h->own_stream, &graph);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    set_error(std::string("graph capture: ") + cudaGetErrorString(err != cudaSuccess ? err : e2));
    return LBS_ECUDA;
  }
  cudaGraphExec_t exec = nullptr;
  err = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  LBS_CK(err);
  h->graph[parity] = exec;
  h->graph_variant[parity] = h->variant;
  return LBS_OK;
}

// read back a finished monitor; returns LBS_EUNSTABLE once a non-finite value was seen
int check_monitor(lbs_handle *h, bool wait) {
  if (h->unstable_at >= 0) return LBS_EUNSTABLE;
  if (!h->mon_pending) return LBS_OK;
  cudaError_t q = wait ? cudaEventSynchronize(h->mon_event) : cudaEventQuery(h->mon_event);
  if (q == cudaErrorNotReady) return LBS_OK;
  LBS_CK(q);
  h->mon_pending = false;
  if (h->mon_host[5] != 0.0) {
    h->unstable_at = (int64_t)h->mon_host[6];
    return fail(LBS_EUNSTABLE, "non-finite value at iteration " + std::to_string(h->unstable_at));
  }
  return LBS_OK;
}

int launch_monitor_async(lbs_handle *h) {
  LBS_CK(h->L->monitor(h->P, h->g[h->parity], h->u[h->parity], h->mon_partials, monitor_blocks(h->P), h->mon_out,
                       h->k, h->stream));
  LBS_CK(cudaMemcpyAsync(h->mon_host, h->mon_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LBS_CK(cudaEventRecord(h->mon_event, h->stream));
  h->launches += 2;
  h->mon_pending = true;
  h->mon_k = h->k;
  return LBS_OK;
}

// select a tile variant; TMA variants get their descriptors built here
int select_variant(lbs_handle *h, int variant) {
  bool tma = h->L->tma_maps(h->P, variant, h->g[0], h->u[0], &h->tm_g[0], &h->tm_u[0]);
  if (tma) tma = h->L->tma_maps(h->P, variant, h->g[1], h->u[1], &h->tm_g[1], &h->tm_u[1]);
  if (!tma && ((h->L->tma_mask >> variant) & 1))
    return fail(LBS_ECUDA, "TMA descriptors could not be built for tile variant " + std::to_string(variant));
  h->tma = tma;
  h->variant = variant;
  return LBS_OK;
}

int reset_state_counters(lbs_handle *h) {
  h->k = 0;
  h->parity = 0;
  h->unstable_at = -1;
  h->mon_pending = false;
  h->next_mon = h->mon_interval;
  set_counter_kernel<<<1, 1, 0, h->stream>>>(h->kdev, 0);
  LBS_CK(cudaGetLastError());
  h->launches += 1;
  h->kdev_value = 0;
  LBS_CK(cudaMemsetAsync(h->mon_out, 0, 7 * sizeof(double), h->stream));
  return LBS_OK;
}

}  // namespace

extern "C" {

const char *lbs_strerror(int code) {
  switch (code) {
    case LBS_OK: return "ok";
    case LBS_EINVAL: return "invalid argument";
    case LBS_ENOMEM: return "out of memory";
    case LBS_ECUDA: return "CUDA error";
    case LBS_EUNSTABLE: return "non-finite value detected";
    case LBS_ETIMEOUT: return "timed out";
    case LBS_EBUSY: return "busy";
    case LBS_ENOTFOUND: return "not found";
    case LBS_ECANCELED: return "cancelled";
    default: return "unknown error";
  }
}

const char *lbs_last_error(void) { return g_last_error.c_str(); }

int lbs_set_allocator(lbs_alloc_fn alloc, lbs_free_fn release, void *ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return fail(LBS_EINVAL, "allocator needs both functions");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = release;
  g_alloc_ctx = ctx;
  return LBS_OK;
}

int lbs_params(const lbs_lattice *lat, const lbs_material *mat, double out[5]) {
  int rc = validate(lat, mat, nullptr);
  if (rc) return rc;
  if (!out) return fail(LBS_EINVAL, "null output");
  derive(lat, mat, out);
  return LBS_OK;
}

size_t lbs_footprint(const lbs_lattice *lat) {
  if (!lat || lat->nx < 3 || lat->ny < 3 || lat->precision < LBS_FP64 || lat->precision > LBS_FP16S ||
      (lat->wall_extrap != LBS_EXTRAP_OWN && lat->wall_extrap != LBS_EXTRAP_LINEAR))
    return 0;
  lbs_material m = {LBS_NH, 1.0, 0.3, 1.0, {0.0, 0.0}};
  Params p = make_params(lat, &m, nullptr);
  Sizes s = sizes_of(p, launchers_for(lat->precision));
  return 2 * (s.g + s.u + s.b) + s.mon;
}

int lbs_constitutive(int32_t model, double lam, double mu, const double H[4], double P[4], double N[4]) {
  if (model < LBS_SVK || model > LBS_LE || !H) return fail(LBS_EINVAL, "bad constitutive arguments");
  double n[4];
  constitutive_n<double>(model, lam, mu, H, n);
  const double trH = H[0] + H[3];
  if (N)
    for (int m = 0; m < 4; ++m) N[m] = n[m];
  if (P) {
    P[0] = n[0] + mu * (2 * H[0] + trH);
    P[1] = n[1] + mu * (H[1] + H[2]);
    P[2] = n[2] + mu * (H[1] + H[2]);
    P[3] = n[3] + mu * (2 * H[3] + trH);
  }
  return LBS_OK;
}

int lbs_tile_variant_kind(int32_t precision, int32_t variant) {
  if (precision < LBS_FP64 || precision > LBS_FP16S) return fail(LBS_EINVAL, "unknown precision");
  const Launchers &L = launchers_for(precision);
  if (variant < 0 || variant >= L.nvariants) return fail(LBS_EINVAL, "unknown tile variant");
  return (L.tma_mask >> variant) & 1;
}

const char *lbs_tile_variant_name(int32_t precision, int32_t variant) {
  if (precision < LBS_FP64 || precision > LBS_FP16S) return nullptr;
  const Launchers &L = launchers_for(precision);
  if (variant < 0 || variant >= L.nvariants) return nullptr;
  return L.name(variant);
}

int32_t lbs_variant(const lbs_handle *h) { return h ? h->variant : LBS_EINVAL; }

int lbs_tile_variants(int32_t precision, int32_t *count, int32_t *tx, int32_t *ty) {
  if (precision < LBS_FP64 || precision > LBS_FP16S) return fail(LBS_EINVAL, "unknown precision");
  const Launchers &L = launchers_for(precision);
  if (count) *count = L.nvariants;
  for (int v = 0; v < L.nvariants; ++v) {
    TileShape s = L.shape(v);
    if (tx) tx[v] = s.tx;
    if (ty) ty[v] = s.ty;
  }
  return LBS_OK;
}

int lbs_create(const lbs_lattice *lat, const lbs_material *mat, const lbs_bcs *bcs, lbs_handle **out) {
  if (!out) return fail(LBS_EINVAL, "null output handle");
  *out = nullptr;
  int rc = validate(lat, mat, bcs);
  if (rc) return rc;
  lbs_handle *h = new (std::nothrow) lbs_handle();
  if (!h) return fail(LBS_ENOMEM, "host allocation");
  h->P = make_params(lat, mat, bcs);
  h->lat = *lat;
  h->mat = *mat;
  if (bcs) {
    h->bcs = *bcs;
  } else {
    memset(&h->bcs, 0, sizeof(h->bcs));
    for (int e = 0; e < 4; ++e) h->bcs.edge[e].type = LBS_NEUMANN;
  }
  h->precision = lat->precision;
  h->L = &launchers_for(lat->precision);
  h->variant = -1;
  h->alloc = current_allocator();
  h->mon_interval = 1000;
  h->graph_chunk = 64;
  h->unstable_at = -1;
  h->cfl_warn = mat->nu > 0.25;
  if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(LBS_ECUDA, "stream creation failed (no CUDA device?)");
  }
  h->stream = h->own_stream;
  Sizes s = sizes_of(h->P, *h->L);
  bool ok = true;
  for (int i = 0; i < 2 && ok; ++i) {
    h->g[i] = dev_alloc(h->alloc, s.g, h->stream);
    h->u[i] = dev_alloc(h->alloc, s.u, h->stream);
    h->b[i] = dev_alloc(h->alloc, s.b, h->stream);
    ok = h->g[i] && h->u[i] && h->b[i];
  }
  if (ok) {
    h->mon_block = dev_alloc(h->alloc, s.mon, h->stream);
    ok = h->mon_block != nullptr;
  }
  if (ok && cudaMallocHost(&h->mon_host, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    h->mon_host = nullptr;
    ok = false;
  }
  if (ok && cudaEventCreateWithFlags(&h->mon_event, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ok = false;
  }
  if (ok && (cudaStreamCreateWithFlags(&h->fork.side, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&h->fork.fork, cudaEventDisableTiming) != cudaSuccess ||
             cudaEventCreateWithFlags(&h->fork.join, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    ok = false;
  }
  if (!ok) {
    lbs_destroy(h);
    return fail(LBS_ENOMEM, "device allocation of " + std::to_string(2 * (s.g + s.u + s.b)) + " bytes failed");
  }
  char *mb = (char *)h->mon_block;
  h->mon_partials = (double *)mb;
  h->mon_out = (double *)(mb + (size_t)monitor_blocks(h->P) * 5 * sizeof(double));
  h->kdev = (int64_t *)(h->mon_out + 8);
  h->zero_dev = h->kdev + 1;
  h->errdev = (int *)(h->kdev + 2);
  h->bytes = 2 * (s.g + s.u + s.b) + s.mon;
  rc = select_variant(h, h->L->default_variant);
  if (!rc && cudaMemsetAsync(h->zero_dev, 0, 2 * sizeof(int64_t), h->stream) != cudaSuccess) rc = LBS_ECUDA;
  if (!rc) rc = lbs_set_initial_device(h, nullptr, nullptr);
  if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = fail(LBS_ECUDA, "initialisation failed");
  if (rc) {
    lbs_destroy(h);
    return rc;
  }
  *out = h;
  return LBS_OK;
}

int lbs_destroy(lbs_handle *h) {
  if (!h) return LBS_OK;
  if (h->own_stream) cudaStreamSynchronize(h->own_stream);
  if (h->stream && h->stream != h->own_stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  for (int i = 0; i < 2; ++i) {
    dev_free(h->alloc, h->g[i], h->own_stream);
    dev_free(h->alloc, h->u[i], h->own_stream);
    dev_free(h->alloc, h->b[i], h->own_stream);
  }
  dev_free(h->alloc, h->mon_block, h->own_stream);
  if (h->mon_host) cudaFreeHost(h->mon_host);
  if (h->mon_event) cudaEventDestroy(h->mon_event);
  if (h->fork.side) cudaStreamSynchronize(h->fork.side);
  if (h->fork.side) cudaStreamDestroy(h->fork.side);
  if (h->fork.fork) cudaEventDestroy(h->fork.fork);
  if (h->fork.join) cudaEventDestroy(h->fork.join);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
  return LBS_OK;
}

int lbs_set_stream(lbs_handle *h, void *cuda_stream) {
  if (!h) return fail(LBS_EINVAL, "null handle");
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
  if (s != h->stream) {
    // order the new stream after the work already issued
    cudaEvent_t ev;
    LBS_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    LBS_CK(cudaEventRecord(ev, h->stream));
    LBS_CK(cudaStreamWaitEvent(s, ev, 0));
    cudaEventDestroy(ev);
    h->stream = s;
  }
  return LBS_OK;
}

int lbs_set_initial_device(lbs_handle *h, const double *u0, const double *v0) {
  if (!h) return fail(LBS_EINVAL, "null handle");
  int rc = reset_state_counters(h);
  if (rc) return rc;
  LBS_CK(h->L->init(h->P, h->g[0], h->u[0], h->b[0], u0, v0, h->stream));
  h->launches += 1;
  return LBS_OK;
}

int lbs_set_initial(lbs_handle *h, const double *u0, const double *v0) {
  if (!h) return fail(LBS_EINVAL, "null handle");
  const size_t bytes = (size_t)h->P.nx * h->P.ny * 2 * sizeof(double);
  // the initialisation writes the buffers of parity 0: stage u0, v0 in those
  // of parity 1 (allocate only what does not fit there)
  Scratch sc = scratch_of(h, 1);
  const double *hosts[2] = {u0, v0};
  double *dev[2] = {nullptr, nullptr};
  bool owned[2] = {false, false};
  int rc = LBS_OK;
  for (int i = 0; i < 2 && !rc; ++i) {
    if (!hosts[i]) continue;
    dev[i] = scratch_take(sc, bytes);
    if (!dev[i]) {
      dev[i] = (double *)dev_alloc(h->alloc, bytes, h->stream);
      owned[i] = dev[i] != nullptr;
      if (!dev[i]) rc = fail(LBS_ENOMEM, "initial field buffer");
    }
    if (!rc && cudaMemcpyAsync(dev[i], hosts[i], bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      rc = fail(LBS_ECUDA, "initial field copy");
  }
  if (!rc) rc = lbs_set_initial_device(h, dev[0], dev[1]);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess && !rc) rc = fail(LBS_ECUDA, "initialisation failed");
  for (int i = 0; i < 2; ++i)
    if (owned[i]) dev_free(h->alloc, dev[i], h->stream);
  return rc;
}

int lbs_step(lbs_handle *h, int64_t n) {
  const lbs::TraceRange trace("lbs_step");
  if (!h || n < 0) return fail(LBS_EINVAL, "bad step arguments");
  int rc = check_monitor(h, false);
  if (rc) return rc;
  while (n > 0) {
    if (h->graph_chunk > 0 && n >= h->graph_chunk) {
      if (!h->graph[h->parity] || h->graph_variant[h->parity] != h->variant) {
        if (h->graph[h->parity]) {
          cudaGraphExecDestroy(h->graph[h->parity]);
          h->graph[h->parity] = nullptr;
        }
        rc = capture_graph(h, h->parity);
        if (rc) return rc;
      }
      if (h->kdev_value != h->k) {
        set_counter_kernel<<<1, 1, 0, h->stream>>>(h->kdev, h->k);
        LBS_CK(cudaGetLastError());
        h->launches += 1;
      }
      LBS_CK(cudaGraphLaunch(h->graph[h->parity], h->stream));
      const int its = h->L->iterations_per_call(h->P, h->variant), calls = h->graph_chunk / its;
      h->launches += (int64_t)calls * h->L->kernels_per_step(h->P, h->variant) + 1;
      h->parity ^= calls & 1;  // the buffers swap once per call
      h->k += h->graph_chunk;
      h->kdev_value = h->k;
      n -= h->graph_chunk;
    } else {
      const int its = h->L->iterations_per_call(h->P, h->variant);
      if (its > 1 && n >= its) {
        LBS_CK(h->L->step(h->P, ptrs(h, h->parity, h->zero_dev, h->k), h->variant, h->stream));
        h->launches += h->L->kernels_per_step(h->P, h->variant);
      } else if (its > 1) {
        // the last iteration of an odd count under a fused variant
        LBS_CK(h->L->step1(h->P, ptrs(h, h->parity, h->zero_dev, h->k), h->stream));
        h->launches += h->L->kernels_per_step1(h->P);
      } else {
        LBS_CK(h->L->step(h->P, ptrs(h, h->parity, h->zero_dev, h->k), h->variant, h->stream));
        h->launches += h->L->kernels_per_step(h->P, h->variant);
      }
      const int done = (its > 1 && n >= its) ? its : 1;
      h->parity ^= 1;
      h->k += done;
      n -= done;
    }
    // monitors run at the first chunk boundary at or after each multiple of the interval
    if (h->mon_interval > 0 && h->k >= h->next_mon) {
      rc = launch_monitor_async(h);
      if (rc) return rc;
      while (h->next_mon <= h->k) h->next_mon += h->mon_interval;
    }
  }
  return LBS_OK;
}

int lbs_sync(lbs_handle *h) {
  if (!h) return fail(LBS_EINVAL, "null handle");
  LBS_CK(cudaStreamSynchronize(h->stream));
  int err = 0;
  LBS_CK(cudaMemcpy(&err, h->errdev, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) return fail(LBS_ETIMEOUT, "a kernel gave up waiting for its tile copies");
  return check_monitor(h, true);
}

int lbs_fields_device(lbs_handle *h, double *u, double *v, double *P) {
  if (!h) return fail(LBS_EINVAL, "null handle");
  if (!u && !v && !P) return LBS_OK;
  LBS_CK(h->L->fields(h->P, h->g[h->parity], h->u[h->parity], u, v, P, h->stream));
  h->launches += 1;
  return LBS_OK;
}

int lbs_fields(lbs_handle *h, double *u, double *v, double *P) {
  if (!h) return fail(LBS_EINVAL, "null handle");
  const size_t n = (size_t)h->P.nx * h->P.ny;
  double *hosts[3] = {u, v, P};
  const size_t bytes[3] = {n * 2 * sizeof(double), n * 2 * sizeof(double), n * 4 * sizeof(double)};
  bool done[3] = {!u, !v, !P};
  double *owned[3] = {nullptr, nullptr, nullptr};
  int rc = LBS_OK;
  // passes over the fields: each stages what fits in the buffers of the
  // other parity (allocating one field that fits nowhere), then copies it
  // out; stream order keeps a pass from overwriting the last one's copies
  while (!rc && !(done[0] && done[1] && done[2])) {
    Scratch sc = scratch_of(h, h->parity ^ 1);
    double *dev[3] = {nullptr, nullptr, nullptr};
    bool any = false;
    for (int i = 0; i < 3; ++i)
      if (!done[i] && (dev[i] = scratch_take(sc, bytes[i]))) any = true;
    if (!any) {
      const int i = !done[0] ? 0 : (!done[1] ? 1 : 2);
      if (!(owned[i] = dev[i] = (double *)dev_alloc(h->alloc, bytes[i], h->stream))) {
        rc = fail(LBS_ENOMEM, "field buffer");
        break;
      }
    }
    rc = lbs_fields_device(h, dev[0], dev[1], dev[2]);
    for (int i = 0; i < 3 && !rc; ++i) {
      if (!dev[i]) continue;
      if (cudaMemcpyAsync(hosts[i], dev[i], bytes[i], cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        rc = fail(LBS_ECUDA, "field copy");
      done[i] = true;
    }
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess && !rc) rc = fail(LBS_ECUDA, "field output failed");
  for (int i = 0; i < 3; ++i) dev_free(h->alloc, owned[i], h->stream);
  return rc;
}

int lbs_probe(lbs_handle *h, int32_t n, const int32_t *idx, double *out) {
  if (!h || n < 0 || (n > 0 && (!idx || !out))) return fail(LBS_EINVAL, "bad probe arguments");
  if (n == 0) return LBS_OK;
  const int64_t nn = (int64_t)h->P.nx * h->P.ny;
  for (int i = 0; i < n; ++i)
    if (idx[i] < 0 || idx[i] >= nn) return fail(LBS_EINVAL, "probe index out of range");
  char *buf = (char *)dev_alloc(h->alloc, (size_t)n * (sizeof(int32_t) + 2 * sizeof(double)) + 16, h->stream);
  if (!buf) return fail(LBS_ENOMEM, "probe buffer");
  double *dout = (double *)buf;
  int32_t *didx = (int32_t *)(buf + (size_t)n * 2 * sizeof(double));
  int rc = LBS_OK;
  if (cudaMemcpyAsync(didx, idx, n * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      h->L->probe(h->P, h->u[h->parity], didx, n, dout, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(out, dout, (size_t)n * 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    rc = fail(LBS_ECUDA, "probe failed");
  h->launches += 1;
  dev_free(h->alloc, buf, h->stream);
  return rc;
}

int lbs_grid_error_device(lbs_handle *h, const double *u_ref, double out[2]) {
  if (!h || !u_ref || !out) return fail(LBS_EINVAL, "null argument");
  // the monitors' partials (5 per block) hold the 3 per block needed here
  LBS_CK(h->L->grid_error(h->P, h->u[h->parity], u_ref, h->mon_partials, monitor_blocks(h->P), h->mon_out,
                          h->stream));
  h->launches += 2;
  double o[3];
  LBS_CK(cudaMemcpyAsync(o, h->mon_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LBS_CK(cudaStreamSynchronize(h->stream));
  out[0] = o[0];
  out[1] = o[1];
  return LBS_OK;
}

int lbs_grid_error(lbs_handle *h, const double *u_ref, double out[2]) {
  if (!h || !u_ref || !out) return fail(LBS_EINVAL, "null argument");
  const size_t bytes = (size_t)h->P.nx * h->P.ny * 2 * sizeof(double);
  // stage the reference field in the buffers of the other parity (the next
  // iteration overwrites them unread), else in a temporary
  Scratch sc = scratch_of(h, h->parity ^ 1);
  double *dev = scratch_take(sc, bytes);
  const bool owned = dev == nullptr;
  if (owned && !(dev = (double *)dev_alloc(h->alloc, bytes, h->stream))) return fail(LBS_ENOMEM, "reference buffer");
  int rc = LBS_OK;
  if (cudaMemcpyAsync(dev, u_ref, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    rc = fail(LBS_ECUDA, "reference copy");
  if (!rc) rc = lbs_grid_error_device(h, dev, out);
  if (owned) {
    cudaStreamSynchronize(h->stream);
    dev_free(h->alloc, dev, h->stream);
  }
  return rc;
}

int lbs_monitor(lbs_handle *h, lbs_monitors *out) {
  if (!h || !out) return fail(LBS_EINVAL, "null argument");
  int rc = launch_monitor_async(h);
  if (rc) return rc;
  LBS_CK(cudaEventSynchronize(h->mon_event));
  h->mon_pending = false;
  out->iteration = h->k;
  out->nonfinite = (int64_t)h->mon_host[0];
  out->max_abs_u = h->mon_host[1];
  out->momentum[0] = h->mon_host[2];
  out->momentum[1] = h->mon_host[3];
  out->mass = h->mon_host[4];
  if (h->mon_host[5] != 0.0 && h->unstable_at < 0) h->unstable_at = (int64_t)h->mon_host[6];
  return LBS_OK;
}

int lbs_set_monitor_interval(lbs_handle *h, int64_t m) {
  if (!h || m < 0) return fail(LBS_EINVAL, "bad monitor interval");
  h->mon_interval = m;
  h->next_mon = m > 0 ? (h->k / m + 1) * m : 0;
  return LBS_OK;
}

int lbs_set_graph_chunk(lbs_handle *h, int32_t k) {
  if (!h || k < 0 || k == 1 || (k % 2)) return fail(LBS_EINVAL, "graph chunk must be 0 or an even number >= 2");
  if (k != h->graph_chunk) {
    LBS_CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    h->graph_chunk = k;
  }
  return LBS_OK;
}

int lbs_set_variant(lbs_handle *h, int32_t variant) {
  if (!h || variant < 0 || variant >= h->L->nvariants) return fail(LBS_EINVAL, "unknown tile variant");
  if (variant != h->variant) LBS_CK(cudaStreamSynchronize(h->stream));
  return select_variant(h, variant);
}

int lbs_autotune_handle(lbs_handle *h, int32_t steps) {
  if (!h) return fail(LBS_EINVAL, "null handle");
  int32_t best = 0;
  int rc = lbs_autotune(&h->lat, &h->mat, &h->bcs, steps, &best, nullptr);
  if (rc) return rc;
  return lbs_set_variant(h, best);
}

// ---- checkpoint / resume
// Layout: CkptHeader, then g (nine planes of ny x pitch), u (ny x pitch
// records), the boundary side array, each in the handle's storage format.
namespace {
struct CkptHeader {
  char magic[8];        // "LBSCKPT1"
  int32_t precision;
  int32_t reserved;
  int64_t k;            // iteration of the saved state
  uint64_t g, u, b;     // bytes of each array
  Params P;             // the lattice's parameters (must match on load)
};
const char kCkptMagic[8] = {'L', 'B', 'S', 'C', 'K', 'P', 'T', '1'};
}  // namespace

size_t lbs_checkpoint_bytes(const lbs_handle *h) {
  if (!h) return 0;
  const Sizes sz = sizes_of(h->P, *h->L);
  return sizeof(CkptHeader) + sz.g + sz.u + sz.b;
}

int lbs_save(lbs_handle *h, void *buf, size_t bytes) {
  if (!h || !buf) return fail(LBS_EINVAL, "null argument");
  if (bytes < lbs_checkpoint_bytes(h)) return fail(LBS_EINVAL, "checkpoint buffer too small");
  int rc = lbs_sync(h);
  if (rc) return rc;
  const Sizes sz = sizes_of(h->P, *h->L);
  CkptHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kCkptMagic, 8);
  hd.precision = h->precision;
  hd.k = h->k;
  hd.g = sz.g;
  hd.u = sz.u;
  hd.b = sz.b;
  hd.P = h->P;
  char *out = (char *)buf;
  memcpy(out, &hd, sizeof(hd));
  out += sizeof(hd);
  LBS_CK(cudaMemcpy(out, h->g[h->parity], sz.g, cudaMemcpyDeviceToHost));
  LBS_CK(cudaMemcpy(out + sz.g, h->u[h->parity], sz.u, cudaMemcpyDeviceToHost));
  LBS_CK(cudaMemcpy(out + sz.g + sz.u, h->b[h->parity], sz.b, cudaMemcpyDeviceToHost));
  return LBS_OK;
}

int lbs_load(lbs_handle *h, const void *buf, size_t bytes) {
  if (!h || !buf) return fail(LBS_EINVAL, "null argument");
  if (bytes < sizeof(CkptHeader)) return fail(LBS_EINVAL, "checkpoint too short");
  CkptHeader hd;
  memcpy(&hd, buf, sizeof(hd));
  const Sizes sz = sizes_of(h->P, *h->L);
  if (memcmp(hd.magic, kCkptMagic, 8) != 0) return fail(LBS_EINVAL, "not a liblbs checkpoint");
  if (hd.precision != h->precision || hd.g != sz.g || hd.u != sz.u || hd.b != sz.b ||
      memcmp(&hd.P, &h->P, sizeof(Params)) != 0)
    return fail(LBS_EINVAL, "checkpoint of a different lattice, material, boundary set-up or precision");
  if (bytes < sizeof(CkptHeader) + sz.g + sz.u + sz.b || hd.k < 0) return fail(LBS_EINVAL, "checkpoint truncated");
  LBS_CK(cudaStreamSynchronize(h->stream));
  const char *in = (const char *)buf + sizeof(CkptHeader);
  LBS_CK(cudaMemcpy(h->g[h->parity], in, sz.g, cudaMemcpyHostToDevice));
  LBS_CK(cudaMemcpy(h->u[h->parity], in + sz.g, sz.u, cudaMemcpyHostToDevice));
  LBS_CK(cudaMemcpy(h->b[h->parity], in + sz.g + sz.u, sz.b, cudaMemcpyHostToDevice));
  h->k = hd.k;
  h->kdev_value = -1;  // graph replays re-read the iteration base
  h->unstable_at = -1;
  h->mon_pending = false;
  h->next_mon = h->mon_interval > 0 ? (h->k / h->mon_interval + 1) * h->mon_interval : 0;
  LBS_CK(cudaMemsetAsync(h->mon_out, 0, 7 * sizeof(double), h->stream));
  LBS_CK(cudaStreamSynchronize(h->stream));
  return LBS_OK;
}

int64_t lbs_iteration(const lbs_handle *h) { return h ? h->k : -1; }
int64_t lbs_unstable_iteration(const lbs_handle *h) { return h ? h->unstable_at : -1; }
int lbs_cfl_warning(const lbs_handle *h) { return h ? h->cfl_warn : 0; }
size_t lbs_device_bytes(const lbs_handle *h) { return h ? h->bytes : 0; }
int64_t lbs_launch_count(const lbs_handle *h) { return h ? h->launches : 0; }

}  // extern "C"
