// Continuous-batching server of liblbs (include/lbs_serve.h): admission by
// device footprint, resident state, one batched step kernel per iteration over
// a tile table spanning all resident lattices, retirement at chunk boundaries.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lbs_serve.h"
#include "lbs_device.cuh"
#include "lbs_internal.h"
#include "lbs_trace.h"

using lbs::BatchLattice;
using lbs::BatchTile;

namespace lbs {

// every lattice's chunk-start iteration advances by the chunk's n launches,
// to its end at most
static __global__ void batch_advance_kernel(BatchLattice *lats, int nlats, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlats) return;
  const int64_t k = lats[i].k, kend = lats[i].kend;
  if (k < kend) lats[i].k = k + n < kend ? k + n : kend;
}

cudaError_t launch_batch_advance(BatchLattice *lats, int nlats, int n, cudaStream_t st) {
  if (nlats > 0 && n > 0) batch_advance_kernel<<<(nlats + 127) / 128, 128, 0, st>>>(lats, nlats, n);
  return cudaGetLastError();
}

// the edges' prescribed values of every lattice for the n iterations of the
// chunk (iteration k + it, k its chunk start), with the frame tiles' own
// function: one thread per lattice, iteration and edge
static __global__ void batch_edges_kernel(BatchLattice *lats, int nlats, int n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nlats * n * 4) return;
  const int e = (int)(i % 4), it = (int)((i / 4) % n), l = (int)(i / (4 * (int64_t)n));
  const BatchLattice &L = lats[l];
  if (L.sev) edge_value(L.P, e, L.k + it, L.sev + ((size_t)it * 4 + e) * 2);
}

cudaError_t launch_batch_edges(BatchLattice *lats, int nlats, int n, cudaStream_t st) {
  const int64_t m = (int64_t)nlats * n * 4;
  if (m > 0) batch_edges_kernel<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(lats, nlats, n);
  return cudaGetLastError();
}

}  // namespace lbs

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t id = 0;
  lbs_lattice lat;
  lbs_material mat;
  lbs_bcs bcs;
  int64_t nsteps = 0;
  int state = LBS_TICKET_QUEUED;
  int error = LBS_OK;
  int64_t k = 0;
  double t_submit = 0, t_admit = -1, t_done = -1;
  double t_queued = 0;    // when it (last) entered the queue
  double t_resident = 0;  // when it (last) became resident
  int64_t swaps = 0;      // times it was swapped out to make room
  size_t bytes = 0;
  lbs_handle *h = nullptr;
  std::vector<unsigned char> ckpt;  // state while swapped out (lbs_save)
  bool cancel = false;              // lbs_cancel on a running request (under the server's lock)
  std::vector<double> u, v, P;
};

}  // namespace

struct lbs_server {
  lbs_server_config cfg;
  int device = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Req *> queue;
  std::map<uint64_t, Req *> tickets;
  uint64_t next_id = 1;
  size_t used = 0;
  Clock::time_point t0;
  lbs_server_stats st;
  // owned by the worker thread
  cudaStream_t stream = nullptr;
  lbs::StreamFork fork = {nullptr, nullptr, nullptr};  // frame tiles beside interior tiles
  BatchLattice *d_lats = nullptr;
  int lat_cap = 0;
  BatchTile *d_tiles = nullptr;
  int tile_cap = 0;
  double *d_sev = nullptr;  // the chunk's edge values, [lattice][it][4][2]
  int sev_cap = 0;
  int *d_err = nullptr;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void finish(lbs_server *s, Req *r, int error) {
  // the batch advanced the state outside the handle: bring it up to date
  lbs_handle *h = r->h;
  if (h) {
    h->k = r->k;
    h->parity = (int)(r->k & 1);
    h->kdev_value = -1;
    if (!error) {
      lbs_monitors m;
      if (lbs_monitor(h, &m) == LBS_OK && m.nonfinite > 0) error = LBS_EUNSTABLE;
    }
    const size_t n = (size_t)r->lat.nx * r->lat.ny;
    r->u.resize(2 * n);
    r->v.resize(2 * n);
    r->P.resize(4 * n);
    if (lbs_fields(h, r->u.data(), r->v.data(), r->P.data()) != LBS_OK && !error) error = LBS_ECUDA;
    lbs_destroy(h);
    r->h = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->used -= r->bytes;
  r->error = error;
  r->state = error ? LBS_TICKET_FAILED : LBS_TICKET_DONE;
  r->t_done = s->now();
  s->st.resident -= 1;
  if (error) s->st.failed += 1;
  else s->st.completed += 1;
  s->st.node_updates += (int64_t)r->lat.nx * r->lat.ny * r->k;
  s->cv_done.notify_all();
}

template <class T>
bool ensure(T *&ptr, int &cap, int need) {
  if (need <= cap) return true;
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  int c = std::max(need, 2 * cap);
  if (cudaMalloc(&ptr, sizeof(T) * (size_t)c) != cudaSuccess) {
    cudaGetLastError();
    cap = 0;
    return false;
  }
  cap = c;
  return true;
}

// iterations between the worker's checks for non-finite values (the same
// interval as a handle's default monitor)
constexpr int64_t kCheckEvery = 1000;

// requests admitted at one scheduling point at most: a long queue joins the
// batch over several chunks, its handles created while the GPU runs the
// chunks of the lattices already admitted
constexpr int kAdmitPerChunk = 16;

// bring the handle up to date with the batch's advance of the lattice
void sync_handle(Req *r) {
  lbs_handle *h = r->h;
  h->k = r->k;
  h->parity = (int)(r->k & 1);
  h->kdev_value = -1;
}

// true if the lattice's state holds a non-finite value (brings the handle's
// iteration and buffer parity up to date with the batch first)
bool unstable(Req *r) {
  sync_handle(r);
  lbs_monitors m;
  return lbs_monitor(r->h, &m) == LBS_OK && m.nonfinite > 0;
}

// Swap-out victims for a queued request that does not fit: resident lattices
// resident for at least `protect` seconds, the most remaining iterations
// first, each with more remaining iterations than the request, until the
// request fits the budget; empty if it cannot be made to fit.  Called with the
// server's lock held.
std::vector<Req *> pick_victims(lbs_server *s, const std::vector<Req *> &res, const Req *head, double now,
                                double protect) {
  std::vector<Req *> cand;
  for (Req *r : res)
    if (now - r->t_resident >= protect) cand.push_back(r);
  std::sort(cand.begin(), cand.end(), [](const Req *a, const Req *b) { return a->nsteps - a->k > b->nsteps - b->k; });
  std::vector<Req *> out;
  size_t used = s->used;
  for (Req *r : cand) {
    if (used + head->bytes <= s->cfg.hbm_budget) break;
    if (r->nsteps - r->k <= head->nsteps - head->k) break;
    out.push_back(r);
    used -= r->bytes;
  }
  if (used + head->bytes > s->cfg.hbm_budget) out.clear();
  return out;
}

// one chunk of `n` iterations of every resident lattice: replays of a CUDA
// graph captured for the current tile tables (after one direct chunk on
// them), else direct launches
struct ChunkGraph {
  cudaGraphExec_t exec = nullptr;
  int64_t n = 0;
  bool warm = false;  // one direct chunk ran on the current tables
  void drop() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    n = 0;
    warm = false;
  }
};

cudaError_t run_chunk(lbs_server *s, const lbs::Launchers &L, int shape, int nres, int ni, int ne, int nl, int64_t n,
                      ChunkGraph &G) {
  const lbs::TraceRange trace("lbs_server chunk");
  auto direct = [&]() -> cudaError_t {
    const cudaError_t e0 = lbs::launch_batch_edges(s->d_lats, nres, (int)n, s->stream);
    if (e0 != cudaSuccess) return e0;
    for (int64_t it = 0; it < n; ++it) {
      const BatchTile *t = s->d_tiles;
      const cudaError_t e = L.batch_step(shape, s->d_lats, nres, t, ni, t + ni, ne, t + ni + ne, nl, (int)it,
                                         s->d_err, s->stream, &s->fork);
      if (e != cudaSuccess) return e;
    }
    return lbs::launch_batch_advance(s->d_lats, nres, (int)n, s->stream);
  };
  if (n != s->cfg.chunk || n < 2) return direct();
  if (!G.warm) {
    G.warm = true;
    return direct();
  }
  if (!G.exec || G.n != n) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const cudaError_t e = direct();
      const cudaError_t ec = cudaStreamEndCapture(s->stream, &g);
      if (e == cudaSuccess && ec == cudaSuccess && g && cudaGraphInstantiate(&G.exec, g, 0) != cudaSuccess)
        G.exec = nullptr;
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    G.n = G.exec ? n : 0;
  }
  if (!G.exec) return direct();
  return cudaGraphLaunch(G.exec, s->stream);
}

void run(lbs_server *s) {
  cudaSetDevice(s->device);
  int64_t since_check = 0;
  ChunkGraph graph;
  std::vector<Req *> res;                     // lattices in the batch tables
  std::vector<std::pair<Req *, int>> retire;  // left the batch; finished while the next chunk runs
  std::vector<BatchLattice> hl;
  std::vector<BatchTile> ht;
  int ni = 0, ne = 0, nl = 0;  // interior tiles, frame tiles, frame tiles of two-point-extrapolation lattices
  bool dirty = true;
  // Batch tile shape: fixed by the configuration, or picked by timing.  A
  // trial runs one chunk on each candidate shape (every shape computes each
  // node with the same operations, so the results do not depend on it) and
  // keeps the one with the most node updates per second of device time.  The
  // first trial takes every shape; a new one starts when the resident node
  // count has halved or doubled since the last, and takes the two fastest of
  // the previous trial (a trial's chunks on slow shapes cost throughput).
  const bool tune = s->cfg.batch_shape == 0;
  int shape = tune ? 0 : s->cfg.batch_shape - 1;
  int trial = -1;            // place in `cand` of the shape under trial, -1 outside a trial
  int64_t tuned_nodes = -1;  // resident nodes when the last trial ended
  std::vector<int> cand;     // shapes of the current trial
  std::vector<double> rate;  // node updates per ms of each shape, last measured
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  const lbs::Launchers &L = s->cfg.precision == LBS_FP64   ? lbs::launchers_fp64()
                            : s->cfg.precision == LBS_FP32 ? lbs::launchers_fp32()
                                                           : lbs::launchers_fp16();
  // The chunk in flight.  The worker launches a chunk and, while the GPU runs
  // it, creates the handles of newly admitted requests and finishes the
  // lattices that left the batch after the previous chunk (their fields
  // copied out, their memory released); only then does it wait for the chunk.
  struct Flight {
    bool on = false;
    cudaError_t err = cudaSuccess;
    int64_t chunk = 0, work = 0, launched = 0, nodes = 0;
    int shape = 0;
    bool timed = false;
    double t0 = 0;
  } fl;
  // wait for the chunk in flight, account for it, and move the lattices that
  // reached their end (and, every kCheckEvery iterations, those that went
  // non-finite) from the batch to `retire`
  auto complete = [&]() {
    if (!fl.on) return;
    fl.on = false;
    std::vector<Req *> cancelled;
    cudaError_t e = fl.err;
    const cudaError_t es = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = es;
    if (fl.timed && e == cudaSuccess) {
      float ms = 0;
      cudaEventElapsedTime(&ms, ev0, ev1);
      rate[fl.shape] = ms > 0 ? (double)fl.work / ms : 0.0;
      if (++trial < (int)cand.size()) {
        shape = cand[trial];
      } else {
        shape = cand[0];
        for (int b : cand)
          if (rate[b] > rate[shape]) shape = b;
        trial = -1;
        tuned_nodes = fl.nodes;
        std::lock_guard<std::mutex> lk(s->mu);
        s->st.batch_tunings += 1;
      }
      dirty = true;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.busy_seconds += s->now() - fl.t0;
      s->st.launches += fl.launched;
      s->st.batch_shape = fl.shape;
      s->st.batch_tx = L.batch_shape(fl.shape).tx;
      s->st.batch_ty = L.batch_shape(fl.shape).ty;
      for (Req *r : res) r->k = std::min(r->k + fl.chunk, r->nsteps);
      for (Req *r : res)
        if (r->cancel) cancelled.push_back(r);
    }
    since_check += fl.chunk;
    const bool check = since_check >= kCheckEvery;
    if (check) since_check = 0;
    std::vector<Req *> keep;
    for (Req *r : res) {
      if (e != cudaSuccess) retire.emplace_back(r, LBS_ECUDA);
      else if (std::find(cancelled.begin(), cancelled.end(), r) != cancelled.end())
        retire.emplace_back(r, LBS_ECANCELED);
      else if (r->k >= r->nsteps) retire.emplace_back(r, LBS_OK);
      else if (check && unstable(r)) retire.emplace_back(r, LBS_EUNSTABLE);
      else keep.push_back(r);
    }
    if (keep.size() != res.size()) dirty = true;
    res.swap(keep);
  };
  auto finish_retired = [&]() {
    for (auto &x : retire) finish(s, x.first, x.second);
    retire.clear();
  };
  for (;;) {
    // admission: FIFO while the footprint fits
    std::vector<Req *> admit, victims;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (res.empty() && s->queue.empty() && !fl.on && retire.empty()) {
        if (s->stop) break;
        s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
        if (s->stop && s->queue.empty()) break;
      }
      if (s->stop) break;
      while (!s->queue.empty()) {
        Req *r = s->queue.front();
        if (s->cfg.max_resident > 0 && (int)(res.size() + admit.size()) >= s->cfg.max_resident) break;
        if (s->used + r->bytes > s->cfg.hbm_budget || (int)admit.size() >= kAdmitPerChunk) break;
        s->queue.pop_front();
        s->used += r->bytes;
        s->st.queued -= 1;
        s->st.resident += 1;
        admit.push_back(r);
      }
      // preemption: the queue's head has waited long enough and does not fit
      const double now = s->now();
      if (s->cfg.preempt_after_s > 0 && admit.empty() && !s->queue.empty() &&
          now - s->queue.front()->t_queued >= s->cfg.preempt_after_s)
        victims = pick_victims(s, res, s->queue.front(), now, s->cfg.preempt_after_s);
    }
    // swap the victims out: state to host memory, device memory released; they
    // rejoin the queue at the back and resume from their saved state (the
    // chunk in flight is waited for first: it advances their state)
    if (!victims.empty()) {
      complete();
      finish_retired();
    }
    for (Req *r : victims) {
      if (std::find(res.begin(), res.end(), r) == res.end()) continue;  // it finished meanwhile
      sync_handle(r);
      r->ckpt.resize(lbs_checkpoint_bytes(r->h));
      const int rc = lbs_save(r->h, r->ckpt.data(), r->ckpt.size());
      if (rc) {  // the copy failed: the request ends here
        r->ckpt.clear();
        finish(s, r, rc);
      } else {
        lbs_destroy(r->h);
        r->h = nullptr;
        std::lock_guard<std::mutex> lk(s->mu);
        s->used -= r->bytes;
        s->st.resident -= 1;
        s->st.queued += 1;
        s->st.preemptions += 1;
        r->state = LBS_TICKET_QUEUED;
        r->swaps += 1;
        r->t_queued = s->now();
        s->queue.push_back(r);
      }
      res.erase(std::find(res.begin(), res.end(), r));
      dirty = true;
    }
    if (!victims.empty()) continue;  // admit into the room just made
    // new handles (their initialisation runs on their own streams, beside the
    // chunk in flight)
    std::vector<Req *> created;
    for (Req *r : admit) {
      int rc = lbs_create(&r->lat, &r->mat, &r->bcs, &r->h);
      if (!rc && !r->ckpt.empty()) rc = lbs_load(r->h, r->ckpt.data(), r->ckpt.size());
      if (rc) {
        if (r->h) lbs_destroy(r->h);
        r->h = nullptr;
        finish(s, r, rc);
        continue;
      }
      r->ckpt.clear();
      r->ckpt.shrink_to_fit();
      lbs_set_monitor_interval(r->h, 0);
      std::lock_guard<std::mutex> lk(s->mu);
      r->state = LBS_TICKET_RUNNING;
      if (r->t_admit < 0) r->t_admit = s->now();
      r->t_resident = s->now();
      created.push_back(r);
    }
    complete();
    for (Req *r : created) res.push_back(r);
    if (!created.empty()) dirty = true;
    if (res.empty()) {
      finish_retired();
      continue;
    }
    int64_t nodes = 0;
    for (Req *r : res) nodes += (int64_t)r->lat.nx * r->lat.ny;
    if (tune && trial < 0 && (tuned_nodes < 0 || nodes >= 2 * tuned_nodes || 2 * nodes <= tuned_nodes)) {
      cand.clear();
      if (tuned_nodes < 0) {
        rate.assign(L.nbatch_shapes, 0.0);
        for (int b = 0; b < L.nbatch_shapes; ++b) cand.push_back(b);
      } else {
        std::vector<int> order(L.nbatch_shapes);
        for (int b = 0; b < L.nbatch_shapes; ++b) order[b] = b;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return rate[a] > rate[b]; });
        cand.assign(order.begin(), order.begin() + std::min(2, L.nbatch_shapes));
      }
      trial = 0;
      if (shape != cand[0]) dirty = true;
      shape = cand[0];
    }
    // batch tables
    if (dirty) {
      graph.drop();
      hl.resize(res.size());
      ht.clear();
      std::vector<BatchTile> edge, edge_lin;
      const lbs::TileShape bs = L.batch_shape(shape);
      const int TX = bs.tx, TY = bs.ty;
      for (size_t i = 0; i < res.size(); ++i) {
        lbs_handle *h = res[i]->h;
        BatchLattice &B = hl[i];
        B.P = h->P;
        for (int p = 0; p < 2; ++p) {
          B.g[p] = h->g[p];
          B.u[p] = h->u[p];
          B.b[p] = h->b[p];
        }
        B.k = res[i]->k;
        B.kend = res[i]->nsteps;
        B.sev = nullptr;  // set once the table is allocated
        const int ntx = (h->P.nx + TX - 1) / TX, nty = (h->P.ny + TY - 1) / TY;
        int a_lo, a_hi, b_lo, b_hi;
        lbs::interior_range(h->P.nx, h->P.ny, TX, TY, a_lo, a_hi, b_lo, b_hi);
        for (int b = 0; b < nty; ++b)
          for (int a = 0; a < ntx; ++a) {
            const bool in = a >= a_lo && a < a_hi && b >= b_lo && b < b_hi;
            (in ? ht : (h->P.extrap ? edge_lin : edge)).push_back(BatchTile{(int)i, a, b});
          }
      }
      ni = (int)ht.size();
      ne = (int)edge.size();
      nl = (int)edge_lin.size();
      ht.insert(ht.end(), edge.begin(), edge.end());
      ht.insert(ht.end(), edge_lin.begin(), edge_lin.end());
      const int sev_need = (int)hl.size() * (int)s->cfg.chunk * 8;
      const bool sev_ok = ensure(s->d_sev, s->sev_cap, sev_need);
      for (size_t i = 0; i < hl.size(); ++i) hl[i].sev = sev_ok ? s->d_sev + i * (size_t)s->cfg.chunk * 8 : nullptr;
      if (!ensure(s->d_lats, s->lat_cap, (int)hl.size()) || !ensure(s->d_tiles, s->tile_cap, (int)ht.size())) {
        for (Req *r : res) retire.emplace_back(r, LBS_ENOMEM);
        res.clear();
        finish_retired();
        continue;
      }
      cudaMemcpyAsync(s->d_lats, hl.data(), sizeof(BatchLattice) * hl.size(), cudaMemcpyHostToDevice, s->stream);
      cudaMemcpyAsync(s->d_tiles, ht.data(), sizeof(BatchTile) * ht.size(), cudaMemcpyHostToDevice, s->stream);
      dirty = false;
    }
    // one chunk of iterations for every resident lattice, launched; the
    // lattices that left the batch are finished while it runs
    int64_t chunk = s->cfg.chunk;
    int64_t longest = 0;
    for (Req *r : res) longest = std::max(longest, r->nsteps - r->k);
    chunk = std::min(chunk, longest);
    fl.t0 = s->now();
    fl.chunk = chunk;
    fl.launched = chunk > 0 ? chunk * ((ni > 0) + (ne > 0) + (nl > 0)) + 1 : 0;
    fl.work = 0;  // node updates this chunk executes
    for (Req *r : res) fl.work += (int64_t)r->lat.nx * r->lat.ny * std::min(chunk, r->nsteps - r->k);
    fl.nodes = nodes;
    fl.shape = shape;
    fl.timed = trial >= 0;
    if (fl.timed) cudaEventRecord(ev0, s->stream);
    fl.err = run_chunk(s, L, shape, (int)res.size(), ni, ne, nl, chunk, graph);
    if (fl.timed) cudaEventRecord(ev1, s->stream);
    fl.on = true;
    finish_retired();
  }
  // shutdown: wait for the chunk in flight, release what is still resident
  complete();
  finish_retired();
  graph.drop();
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  for (Req *r : res) {
    if (r->h) lbs_destroy(r->h);
    r->h = nullptr;
  }
}

}  // namespace

extern "C" {

int lbs_server_create(const lbs_server_config *cfg, lbs_server **out) {
  if (!cfg || !out || cfg->precision < LBS_FP64 || cfg->precision > LBS_FP16S || cfg->chunk < 0 ||
      cfg->max_resident < 0 || cfg->queue_limit < 0 || !(cfg->preempt_after_s >= 0) || cfg->batch_shape < 0 ||
      cfg->batch_shape > (cfg->precision == LBS_FP64   ? lbs::launchers_fp64()
                          : cfg->precision == LBS_FP32 ? lbs::launchers_fp32()
                                                       : lbs::launchers_fp16())
                             .nbatch_shapes) {
    lbs::set_error("bad server configuration");
    return LBS_EINVAL;
  }
  lbs_server *s = new lbs_server();
  s->cfg = *cfg;
  if (s->cfg.chunk == 0) s->cfg.chunk = 64;
  memset(&s->st, 0, sizeof(s->st));
  s->t0 = Clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->fork.side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->fork.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->fork.join, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(&s->d_err, sizeof(int)) != cudaSuccess || cudaMemset(s->d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->fork.side) cudaStreamDestroy(s->fork.side);
    if (s->fork.fork) cudaEventDestroy(s->fork.fork);
    if (s->fork.join) cudaEventDestroy(s->fork.join);
    delete s;
    lbs::set_error("server: CUDA set-up failed");
    return LBS_ECUDA;
  }
  if (s->cfg.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    s->cfg.hbm_budget = fr / 10 * 8;
  }
  s->st.hbm_budget = s->cfg.hbm_budget;
  s->worker = std::thread(run, s);
  *out = s;
  return LBS_OK;
}

int lbs_submit(lbs_server *s, const lbs_lattice *lat, const lbs_material *mat, const lbs_bcs *bcs, int64_t nsteps,
               uint64_t *ticket) {
  if (!s || !lat || !mat || !ticket || nsteps < 0) return LBS_EINVAL;
  Req *r = new Req();
  r->lat = *lat;
  r->lat.precision = s->cfg.precision;
  r->mat = *mat;
  if (bcs) {
    r->bcs = *bcs;
  } else {
    memset(&r->bcs, 0, sizeof(r->bcs));
    for (int e = 0; e < 4; ++e) r->bcs.edge[e].type = LBS_NEUMANN;
  }
  double p[5];
  int rc = lbs_params(&r->lat, &r->mat, p);
  if (rc) {
    delete r;
    return rc;
  }
  r->nsteps = nsteps;
  r->bytes = lbs_footprint(&r->lat);
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->bytes > s->cfg.hbm_budget) {
    delete r;
    lbs::set_error("request larger than the server's HBM budget");
    return LBS_ENOMEM;
  }
  if (s->cfg.queue_limit > 0 && (int64_t)s->queue.size() >= s->cfg.queue_limit) {
    delete r;
    lbs::set_error("queue full");
    return LBS_EBUSY;
  }
  r->id = s->next_id++;
  r->t_submit = s->now();
  r->t_queued = r->t_submit;
  s->tickets[r->id] = r;
  s->queue.push_back(r);
  s->st.submitted += 1;
  s->st.queued += 1;
  *ticket = r->id;
  s->cv_work.notify_one();
  return LBS_OK;
}

int lbs_poll(lbs_server *s, uint64_t ticket, lbs_ticket_info *info) {
  if (!s || !info) return LBS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return LBS_ENOTFOUND;
  const Req *r = it->second;
  info->state = r->state;
  info->error = r->error;
  info->iterations = r->k;
  info->nsteps = r->nsteps;
  info->nx = r->lat.nx;
  info->ny = r->lat.ny;
  info->t_submit = r->t_submit;
  info->t_admit = r->t_admit;
  info->t_done = r->t_done;
  info->device_bytes = r->bytes;
  info->swaps = r->swaps;
  return LBS_OK;
}

int lbs_wait(lbs_server *s, uint64_t ticket, double timeout_s) {
  if (!s) return LBS_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto done = [&] {
    auto it = s->tickets.find(ticket);
    return it == s->tickets.end() || it->second->state >= LBS_TICKET_DONE;
  };
  if (s->tickets.find(ticket) == s->tickets.end()) return LBS_ENOTFOUND;
  if (timeout_s < 0) s->cv_done.wait(lk, done);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) return LBS_ETIMEOUT;
  return LBS_OK;
}

int lbs_result(lbs_server *s, uint64_t ticket, double *u, double *v, double *P) {
  if (!s) return LBS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return LBS_ENOTFOUND;
  Req *r = it->second;
  if (r->state < LBS_TICKET_DONE) return LBS_EBUSY;
  if (u && !r->u.empty()) memcpy(u, r->u.data(), r->u.size() * sizeof(double));
  if (v && !r->v.empty()) memcpy(v, r->v.data(), r->v.size() * sizeof(double));
  if (P && !r->P.empty()) memcpy(P, r->P.data(), r->P.size() * sizeof(double));
  const int err = r->error;
  s->tickets.erase(it);
  delete r;
  return err;
}

int lbs_cancel(lbs_server *s, uint64_t ticket) {
  if (!s) return LBS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return LBS_ENOTFOUND;
  Req *r = it->second;
  if (r->state >= LBS_TICKET_DONE) return LBS_OK;
  auto q = std::find(s->queue.begin(), s->queue.end(), r);
  if (q != s->queue.end()) {  // not resident: it ends here
    s->queue.erase(q);
    r->ckpt.clear();
    r->error = LBS_ECANCELED;
    r->state = LBS_TICKET_FAILED;
    r->t_done = s->now();
    s->st.queued -= 1;
    s->st.failed += 1;
    s->cv_done.notify_all();
    return LBS_OK;
  }
  r->cancel = true;  // resident (or being admitted): the worker stops it at its next scheduling point
  return LBS_OK;
}

int lbs_server_drain(lbs_server *s, double timeout_s) {
  if (!s) return LBS_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] {
    for (auto &kv : s->tickets)
      if (kv.second->state < LBS_TICKET_DONE) return false;
    return true;
  };
  if (timeout_s < 0) s->cv_done.wait(lk, idle);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), idle)) return LBS_ETIMEOUT;
  return LBS_OK;
}

int lbs_server_get_stats(lbs_server *s, lbs_server_stats *out) {
  if (!s || !out) return LBS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->bytes_in_use = s->used;
  return LBS_OK;
}

int lbs_server_destroy(lbs_server *s) {
  if (!s) return LBS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto &kv : s->tickets) {
    if (kv.second->h) lbs_destroy(kv.second->h);
    delete kv.second;
  }
  if (s->d_lats) cudaFree(s->d_lats);
  if (s->d_tiles) cudaFree(s->d_tiles);
  if (s->d_sev) cudaFree(s->d_sev);
  if (s->d_err) cudaFree(s->d_err);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->fork.side) cudaStreamDestroy(s->fork.side);
  if (s->fork.fork) cudaEventDestroy(s->fork.fork);
  if (s->fork.join) cudaEventDestroy(s->fork.join);
  delete s;
  return LBS_OK;
}

}  // extern "C"
