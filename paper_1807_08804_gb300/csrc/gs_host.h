// Host-side functions shared by the engine's translation units.
#pragma once

#include <map>
#include <vector>

#include "gs_engine.cuh"

using gs::DQuery;
using gs::KK_N;
using gs::Wave;
using gs::WaveDesc;

// A prepared batch: packed queries, waves, device pools and captured graphs.
struct gs_batch {
  gs_graph *g = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 0;
  int group = 32;
  uint32_t refine_rounds = 8;
  bool fixpoint = true;            // loop rounds on the host until nothing changes (non-graph runs)
  bool use_graph = true;
  uint32_t n = 0;
  std::vector<DQuery> hq;
  std::vector<uint32_t> hstatus;   // gs_status per query from the host checks
  std::vector<WaveDesc> waves;
  std::vector<int> wave_k;
  uint32_t nq_s = 0, nqv_s = 0, nqe_s = 0;
  std::vector<void *> allocs;
  Wave W{};
  DQuery *all_dq = nullptr;
  WaveDesc *dwaves = nullptr;
  uint64_t *scan_tmp = nullptr;
  uint32_t *type_count = nullptr;
  std::map<int, cudaGraphExec_t> execs;
  // stats
  bool stats_on = false;
  struct Ev { int kind; cudaEvent_t a, b; };
  std::vector<Ev> evs;
  std::map<int, std::vector<Ev>> graph_evs;
  double ms[KK_N] = {0};
  uint64_t launches[KK_N] = {0};
  uint64_t bytes_base[KK_N] = {0};
  bool ran = false, finished = false;
  // host results
  std::vector<uint64_t> count, fp, nrows, word_off;
  std::vector<uint32_t> status;
  std::vector<uint32_t> rows;        // store contents
  std::vector<std::vector<uint32_t>> fb_rows;  // rows of queries finished on the fallback path
  std::vector<uint8_t> fb_done;
};

namespace gs {

gs_status pack_query(const DevGraph &G, const gs_query *q, const gs_match_opts *o, DQuery *d);
gs_status batch_create(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts, uint32_t wave_queries,
                       gs_batch **out);
void batch_destroy(gs_batch *b);
gs_status run_waves(gs_batch *b);
gs_status batch_finish(gs_batch *b);
gs_status batch_fetch(gs_batch *b, gs_result *outs);
// Finish query i of a finished run on the host-driven path (chunked join).
gs_status fallback_query(gs_batch *b, uint32_t i);
void enqueue_wave(gs_batch *b, int K, bool capture, std::vector<gs_batch::Ev> *evs);
void enqueue_wave_tail(gs_batch *b, int K, bool capture, std::vector<gs_batch::Ev> *evs, int stop);
gs_status refine_to_fixpoint(gs_batch *b);

}  // namespace gs
