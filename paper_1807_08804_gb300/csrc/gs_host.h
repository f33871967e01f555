// Host-side functions shared by the engine's translation units.
#pragma once

#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "gs_engine.cuh"

// Host array in page-locked memory (direct DMA for uploads and result
// downloads); grows geometrically, never shrinks.
template <typename T>
struct PinnedVec {
  T *p = nullptr;
  size_t n = 0, cap = 0;
  PinnedVec() = default;
  PinnedVec(const PinnedVec &) = delete;
  PinnedVec &operator=(const PinnedVec &) = delete;
  ~PinnedVec() {
    if (p) cudaFreeHost(p);
  }
  void resize(size_t m) {
    if (m > cap) {
      size_t c = cap ? cap : 16;
      while (c < m) c *= 2;
      T *q = nullptr;
      if (cudaMallocHost((void **)&q, sizeof(T) * c) != cudaSuccess) throw std::bad_alloc();
      if (p) {
        memcpy(q, p, sizeof(T) * n);
        cudaFreeHost(p);
      }
      p = q;
      cap = c;
    }
    n = m;
  }
  void assign(size_t m, const T &v) {
    resize(m);
    for (size_t i = 0; i < m; ++i) p[i] = v;
  }
  T *data() { return p; }
  const T *data() const { return p; }
  size_t size() const { return n; }
  T &operator[](size_t i) { return p[i]; }
  const T &operator[](size_t i) const { return p[i]; }
};

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
  int jgroup = 0;  // lanes per partial row in the join (0: the same as group)
  uint32_t refine_rounds = 8;
  bool fixpoint = true;            // loop rounds on the host until nothing changes (non-graph runs)
  bool use_graph = true;
  uint32_t n = 0;
  PinnedVec<DQuery> hq;
  std::vector<uint32_t> hstatus;   // gs_status per query from the host checks
  std::vector<WaveDesc> waves;
  std::vector<int> wave_k;
  uint32_t nq_s = 0, nqv_s = 0, nqe_s = 0;
  std::vector<void *> allocs;
  Wave W{};
  DQuery *all_dq = nullptr;
  WaveDesc *dwaves = nullptr;
  uint64_t *scan_tmp = nullptr;  // scan scratch: zeroed when allocated, used by scans only
  uint64_t scan_tmp_words = 0;
  uint32_t *type_count = nullptr;
  std::map<int, cudaGraphExec_t> execs;
  // stats
  bool stats_on = false;
  struct Ev { int kind; cudaEvent_t a, b; };
  std::vector<Ev> evs;
  std::map<int, std::vector<Ev>> graph_evs;
  double ms[KK_N] = {0};
  // each timed launch as an interval from the run's anchor event (recorded
  // before the run's first launch; shared by batches run together), so that
  // the time some launch of a kind was running can be taken over batches
  // whose launches overlap
  struct Span { uint64_t run; int kind; float t0, t1; };
  std::vector<Span> spans;
  cudaEvent_t anchor = nullptr, own_anchor = nullptr;
  bool shared_anchor = false;  // the anchor belongs to a concurrent run
  bool defer_harvest = false;  // events are read once every batch of the run is queued
  uint64_t run_id = 0;
  uint64_t launches[KK_N] = {0};
  uint64_t bytes_base[KK_N] = {0};
  bool ran = false, finished = false;
  // host results
  PinnedVec<uint64_t> count, fp, nrows, word_off;
  PinnedVec<uint32_t> status;
  PinnedVec<uint32_t> rows;          // store contents
  std::vector<std::vector<uint32_t>> fb_rows;  // rows of queries finished on the fallback path
  std::vector<uint8_t> fb_done;
  std::vector<uint8_t> fb_more;      // fallback, projected: more distinct tuples than cap
  bool has_proj = false;             // some query returns projected rows
  bool has_rev = false;              // some query refines in reversed order
  uint32_t max_k = 1;                // largest query
  // capacity and options (for reuse by later calls with the same options)
  uint32_t n_cap = 0;
  gs_chunk_cb on_chunk = nullptr;  // GS_CHUNKED: where every embedding goes
  void *chunk_user = nullptr;
  uint64_t key_cap = 0, key_chunk = 0;
  uint32_t key_mode = 0, key_rounds = 0;
  void *key_stream = nullptr;
  // accounting
  std::map<int, uint64_t> kernels_per_exec;
  uint64_t kernel_launches = 0;
  uint64_t h2d_bytes = 0, d2h_bytes = 0;
  uint64_t last_upload_bytes = 0;
  bool big = false;                // fallback context sizing
  uint64_t pool_hint = 0;          // fixed candidate-pool entries (serving slots)
  // the epilogue as a separate graph; the large-output sort launched directly
  std::vector<Ev> sort_evs_direct;
  cudaGraphExec_t epi_exec = nullptr;
  std::vector<Ev> epi_evs;
  uint64_t epi_kernels = 0;
  uint64_t *flag = nullptr;        // pinned words read between graphs
  bool sorting = false;            // this run wants rows (reads the large-output flags)
  uint64_t large_sorts = 0;
  uint64_t fallbacks = 0;          // queries finished on the chunked path by the last finish
  uint64_t regrows = 0;            // times pools were enlarged after a run
};

namespace gs {

gs_status pack_query(const DevGraph &G, const gs_query *q, const gs_match_opts *o, DQuery *d);
gs_status batch_create(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts, uint32_t wave_queries,
                       gs_batch **out, bool big = false);
void batch_destroy(gs_batch *b);
bool batch_rearm(gs_batch *b, const gs_query *qs, uint32_t n, const gs_match_opts *opts);
gs_status batch_create_capacity(gs_graph *g, const gs_match_opts *opts, uint32_t n_cap, uint32_t nqv_s, uint32_t nqe_s,
                                gs_batch **out);
gs_status run_waves(gs_batch *b);
// The two halves of a one-wave run, for callers that must not block: after
// run_begin, wait (poll an event recorded on the batch's stream) before
// run_end.
gs_status run_begin(gs_batch *b);
gs_status run_end(gs_batch *b);
// Several single-stream batches at once on their own streams (see gs_batch_run_all).
gs_status run_batches(gs_batch *const *bs, uint32_t nb, cudaStream_t parent);
gs_status batch_finish(gs_batch *b);
gs_status batch_fetch(gs_batch *b, gs_result *outs);
gs_status batch_fetch_views(gs_batch *b, gs_result *outs, uint32_t *store);
// Finish query i of a finished run on the host-driven path (chunked join).
gs_status fallback_query(gs_batch *b, uint32_t i);
void enqueue_wave(gs_batch *b, int K, bool capture, std::vector<gs_batch::Ev> *evs);
void enqueue_wave_tail(gs_batch *b, int K, bool capture, std::vector<gs_batch::Ev> *evs, int stop);
gs_status refine_to_fixpoint(gs_batch *b);
// Matching through a compressed graph: query i's candidates must lie in
// nodes set in the weighted-graph bitmaps at device address wmask[i] (one
// bitmap per query vertex, wstride words apart; 0 = no restriction), the node
// of data vertex v being wgroup[v].  Uploads the batch's queries again.
gs_status batch_set_wmasks(gs_batch *b, const uint64_t *wmask, uint32_t wstride, const uint32_t *wgroup);

}  // namespace gs
