// Autotuner of liblbs: picks the tile variant of the fused step kernel per
// lattice configuration by timing every variant on a scratch lattice, with a
// process-wide cache that can be saved to and loaded from JSON lines.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "lbs_internal.h"

namespace {

using Key = std::tuple<int, int, int, int, int, int>;  // nx, ny, precision, model, per_x, per_y

struct Entry {
  int variant;
  std::vector<float> ms;
};

std::mutex g_mu;
std::map<Key, Entry> g_cache;

Key key_of(const lbs_lattice *lat, const lbs_material *mat, const lbs_bcs *bcs) {
  const int px = bcs && bcs->edge[0].type == LBS_PERIODIC;
  const int py = bcs && bcs->edge[2].type == LBS_PERIODIC;
  return Key(lat->nx, lat->ny, lat->precision, mat->model, px, py);
}

int time_variants(const lbs_lattice *lat, const lbs_material *mat, const lbs_bcs *bcs, int steps,
                  std::vector<float> &ms) {
  lbs_lattice scratch = *lat;
  if (scratch.nx > 4096) scratch.nx = 4096;
  if (scratch.ny > 4096) scratch.ny = 4096;
  lbs_handle *h = nullptr;
  int rc = lbs_create(&scratch, mat, bcs, &h);
  if (rc) return rc;
  int32_t nvar = 0;
  lbs_tile_variants(lat->precision, &nvar, nullptr, nullptr);
  rc = lbs_set_graph_chunk(h, 0);
  if (!rc) rc = lbs_set_monitor_interval(h, 0);
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc && (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
              cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = LBS_ECUDA;
  if (!rc) rc = lbs_set_stream(h, (void *)st);
  ms.assign(nvar, 0.0f);
  for (int v = 0; v < nvar && !rc; ++v) {
    rc = lbs_set_variant(h, v);
    if (!rc) rc = lbs_step(h, 2);
    if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = LBS_ECUDA;
    if (!rc) rc = lbs_step(h, steps);
    if (!rc && cudaEventRecord(e1, st) != cudaSuccess) rc = LBS_ECUDA;
    if (!rc) rc = lbs_sync(h);
    float t = 0.0f;
    if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = LBS_ECUDA;
    ms[v] = t / (float)steps;
  }
  lbs_set_stream(h, nullptr);
  lbs_destroy(h);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  return rc;
}

}  // namespace

extern "C" {

int lbs_autotune(const lbs_lattice *lat, const lbs_material *mat, const lbs_bcs *bcs, int32_t steps, int32_t *best,
                 float *ms) {
  if (!lat || !mat || !best || steps < 1) {
    lbs::set_error("bad autotune arguments");
    return LBS_EINVAL;
  }
  const Key key = key_of(lat, mat, bcs);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *best = it->second.variant;
      // ms has one entry per tile variant of this build; a loaded entry may
      // carry fewer (unknown entries read 0) or more (ignored)
      int32_t nvar = 0;
      lbs_tile_variants(lat->precision, &nvar, nullptr, nullptr);
      if (ms)
        for (int32_t v = 0; v < nvar; ++v) ms[v] = (size_t)v < it->second.ms.size() ? it->second.ms[v] : 0.0f;
      return LBS_OK;
    }
  }
  std::vector<float> t;
  int rc = time_variants(lat, mat, bcs, steps, t);
  if (rc) return rc;
  int b = 0;
  for (size_t v = 1; v < t.size(); ++v)
    if (t[v] < t[b]) b = (int)v;
  *best = b;
  if (ms)
    for (size_t v = 0; v < t.size(); ++v) ms[v] = t[v];
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = Entry{b, t};
  return LBS_OK;
}

int lbs_autotune_save(const char *path) {
  if (!path) return LBS_EINVAL;
  FILE *f = fopen(path, "w");
  if (!f) {
    lbs::set_error(std::string("cannot write ") + path);
    return LBS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  for (const auto &kv : g_cache) {
    const Key &k = kv.first;
    fprintf(f, "{\"nx\": %d, \"ny\": %d, \"precision\": %d, \"model\": %d, \"per_x\": %d, \"per_y\": %d, \"variant\": %d, \"ms\": [",
            std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k),
            kv.second.variant);
    for (size_t v = 0; v < kv.second.ms.size(); ++v) fprintf(f, "%s%.6g", v ? ", " : "", kv.second.ms[v]);
    fprintf(f, "]}\n");
  }
  fclose(f);
  return LBS_OK;
}

int lbs_autotune_load(const char *path) {
  if (!path) return LBS_EINVAL;
  FILE *f = fopen(path, "r");
  if (!f) {
    lbs::set_error(std::string("cannot read ") + path);
    return LBS_EINVAL;
  }
  char line[1024];
  std::lock_guard<std::mutex> lk(g_mu);
  while (fgets(line, sizeof(line), f)) {
    int nx, ny, prec, model, px, py, var;
    if (sscanf(line, " {\"nx\": %d, \"ny\": %d, \"precision\": %d, \"model\": %d, \"per_x\": %d, \"per_y\": %d, \"variant\": %d",
               &nx, &ny, &prec, &model, &px, &py, &var) != 7)
      continue;
    int32_t nvar = 0;
    if (prec < LBS_FP64 || prec > LBS_FP16S || lbs_tile_variants(prec, &nvar, nullptr, nullptr) || var < 0 ||
        var >= nvar)
      continue;
    Entry e{var, {}};
    const char *p = strchr(line, '[');
    while (p && *p && *p != ']') {
      ++p;
      char *end = nullptr;
      float x = strtof(p, &end);
      if (end == p) break;
      if ((int32_t)e.ms.size() < nvar) e.ms.push_back(x);
      p = end;
      while (*p == ' ') ++p;
    }
    g_cache[Key(nx, ny, prec, model, px, py)] = e;
  }
  fclose(f);
  return LBS_OK;
}

}  // extern "C"
