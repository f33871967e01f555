// Autotuner: picks the lanes per work item (the "warps per vertex" of the
// explore, refine, edge-table and join kernels: 4, 8, 16 or 32 lanes; then,
// for the join alone, 4 or 8 lanes per partial row when that is faster) and
// the number of refinement rounds (none, 1, 2 or 4: Section 3.6 finds one
// round the fastest refined variant, and exploration already prunes every
// candidate against all its query edges) for a graph and a kind of query load, by
// timing the captured pipeline on the caller's queries.  Results do not
// depend on either knob (refinement only prunes; the join checks every
// edge), so the choice is purely about speed.
//
// The choice is cached in a text file, one line per entry:
//   <graph hash> <gpu name with '_' for spaces> <load signature> <group> <rounds> <ms> <join group>
// and reused by later gs_tune calls with the same key.  Batches created on
// the graph afterwards use the tuned values.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "gs_host.h"

using namespace gs;

namespace {

std::string gpu_name(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  for (char &c : s)
    if (c == ' ') c = '_';
  return s;
}

// Signature of a query load: size classes that change the best schedule.
uint64_t load_signature(const gs_query *qs, uint32_t n, const gs_match_opts *o) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t x) { h = (h ^ x) * 1099511628211ull; };
  uint64_t kk = 0, mm = 0, bound = 0;
  for (uint32_t i = 0; i < n; ++i) {
    kk += qs[i].k;
    mm += qs[i].m;
    for (uint32_t u = 0; u < qs[i].k; ++u) bound += qs[i].vbind[u] != GS_UNBOUND;
  }
  uint32_t lg = 0;
  while ((1u << lg) < n) ++lg;
  mix(lg);                                    // batch size class
  mix(n ? (10 * kk) / n : 0);                 // mean k (tenths)
  mix(n ? (10 * mm) / n : 0);                 // mean m (tenths)
  mix(kk ? (20 * bound) / kk : 0);            // bound fraction (1/20)
  mix(o ? o->mode : 0);
  return h;
}

bool cache_lookup(const char *path, const std::string &key, uint32_t *group, uint32_t *rounds, double *ms,
                  uint32_t *jgroup) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string h, gpu, sig;
    uint32_t g, r;
    double t;
    if (!(is >> h >> gpu >> sig >> g >> r >> t)) continue;
    uint32_t jg = 0;
    if (!(is >> jg)) jg = 0;  // a line without a join group: the join follows the group
    if (h + " " + gpu + " " + sig == key) {
      *group = g;
      *rounds = r;
      *ms = t;
      *jgroup = jg;
      found = true;  // the last line for a key wins
    }
  }
  return found;
}

void cache_store(const char *path, const std::string &key, uint32_t group, uint32_t rounds, double ms,
                 uint32_t jgroup) {
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << group << " " << rounds << " " << ms << " " << jgroup << "\n";
}

}  // namespace

extern "C" gs_status gs_tune(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                             const char *cache_path, gs_tuning *out) {
  if (!g || !out || (n && !qs)) return fail(GS_ERR_INVALID, "gs_tune: null argument");
  if (n == 0) return fail(GS_ERR_INVALID, "gs_tune: no queries");
  GS_CUDA(cudaSetDevice(g->device));
  char hk[64], sk[64];
  snprintf(hk, sizeof hk, "%016llx", (unsigned long long)g->hash);
  snprintf(sk, sizeof sk, "%016llx", (unsigned long long)load_signature(qs, n, opts));
  const std::string key = std::string(hk) + " " + gpu_name(g->device) + " " + sk;
  memset(out, 0, sizeof(*out));
  uint32_t group = 0, rounds = 0, jgroup = 0;
  double best = 0;
  if (cache_lookup(cache_path, key, &group, &rounds, &best, &jgroup)) {
    out->group = group;
    out->refine_rounds = rounds;
    out->ms = best;
    out->from_cache = 1;
    out->join_group = jgroup ? jgroup : group;
    g->tuned_group = group;
    g->tuned_rounds = rounds;
    g->tuned_jgroup = jgroup;
    return GS_OK;
  }
  gs_batch *b = nullptr;
  gs_status st = batch_create(g, qs, n, opts, 0, &b);
  if (st != GS_OK) return st;
  cudaEvent_t e0, e1;
  GS_CUDA(cudaEventCreate(&e0));
  GS_CUDA(cudaEventCreate(&e1));
  const uint32_t groups[] = {4, 8, 16, 32};
  const uint32_t round_opts[] = {GS_ROUNDS_NONE, 1, 2, 4};
  best = 1e30;
  uint32_t tried = 0;
  // the fastest of a few timed runs (the first run captures the graphs)
  auto time_runs = [&](double &tmin) {
    tmin = 1e30;
    for (int rep = 0; rep < 4 && st == GS_OK; ++rep) {
      cudaEventRecord(e0, b->stream);
      st = run_waves(b);
      cudaEventRecord(e1, b->stream);
      if (st != GS_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(GS_ERR_CUDA, "tuning run failed"); break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tmin = std::min(tmin, (double)ms);
    }
    if (st == GS_OK) tried++;
  };
  for (uint32_t gi : groups) {
    for (uint32_t r : round_opts) {
      st = gs_batch_set(b, 1, (int)gi, r);
      if (st != GS_OK) break;
      double tmin;
      time_runs(tmin);
      if (st != GS_OK) break;
      if (tmin < best) {
        best = tmin;
        group = gi;
        rounds = r;
      }
    }
    if (st != GS_OK) break;
  }
  // then the join's own lanes (it often wants fewer than exploration and
  // the edge tables), with the best refinement rounds
  for (uint32_t gi : groups) {
    for (uint32_t jg : {4u, 8u}) {
      if (st != GS_OK || jg == gi) continue;
      st = gs_batch_set(b, 1, (int)gi, rounds);
      if (st != GS_OK) break;
      b->jgroup = (int)jg;
      double tmin;
      time_runs(tmin);
      if (st == GS_OK && tmin < best) {
        best = tmin;
        group = gi;
        jgroup = jg;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  batch_destroy(b);
  if (st != GS_OK) return st;
  out->group = group;
  out->refine_rounds = rounds;
  out->ms = best;
  out->configs_tried = tried;
  out->join_group = jgroup ? jgroup : group;
  g->tuned_group = group;
  g->tuned_rounds = rounds;
  g->tuned_jgroup = jgroup;
  cache_store(cache_path, key, group, rounds, best, jgroup);
  return GS_OK;
}

extern "C" gs_status gs_tune_set(gs_graph *g, uint32_t group, uint32_t refine_rounds) {
  if (!g) return fail(GS_ERR_INVALID, "gs_tune_set: null graph");
  if (group && group != 4 && group != 8 && group != 16 && group != 32)
    return fail(GS_ERR_INVALID, "group must be 4, 8, 16 or 32 (0 = default)");
  if (refine_rounds > kMaxRounds && refine_rounds != GS_ROUNDS_NONE)
    return fail(GS_ERR_INVALID, "too many refinement rounds");
  g->tuned_group = group;
  g->tuned_rounds = refine_rounds;
  g->tuned_jgroup = 0;
  return GS_OK;
}
