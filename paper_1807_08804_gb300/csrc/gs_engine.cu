// Host orchestration: query checks and packing, batches of waves, the
// captured pipeline graph, result transfer, and the C ABI entry points for
// matching (Algorithm "FilteringAndJoining", thesis Ch. 3).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gs_engine.cuh"
#include "gs_host.h"

using namespace gs;

namespace gs {

// ------------------------------------------------------------ query packing
gs_status pack_query(const DevGraph &G, const gs_query *q, const gs_match_opts *o, DQuery *d) {
  memset(d, 0, sizeof(*d));
  if (!q) return fail(GS_ERR_INVALID, "null query");
  if (q->k == 0 || q->k > kMaxK) return fail(GS_ERR_INVALID, "query k must be in [1, 16]");
  if (q->m > 4 * kMaxM) return fail(GS_ERR_INVALID, "query has too many edges");
  if (!q->vtype || !q->vbind || (q->m && (!q->esrc || !q->edst || !q->erel)))
    return fail(GS_ERR_INVALID, "query has a null array");
  const uint32_t k = q->k;
  for (uint32_t u = 0; u < k; ++u) {
    if (q->vtype[u] != kAny && q->vtype[u] >= G.T) return fail(GS_ERR_INVALID, "query type out of range");
    if (q->vbind[u] != kUnbound && q->vbind[u] >= G.V) return fail(GS_ERR_INVALID, "query binding out of range");
  }
  uint32_t m = 0;
  for (uint32_t j = 0; j < q->m; ++j) {
    uint32_t a = q->esrc[j], b = q->edst[j], r = q->erel[j];
    if (a >= k || b >= k) return fail(GS_ERR_INVALID, "query edge endpoint out of range");
    if (a == b) return fail(GS_ERR_INVALID, "query self-loop");
    if (r >= G.R) return fail(GS_ERR_INVALID, "query relation out of range");
    bool dup = false;
    for (uint32_t i = 0; i < m; ++i)
      if (d->esrc[i] == a && d->edst[i] == b && d->erel[i] == r) dup = true;
    if (dup) continue;
    if (m >= kMaxM) return fail(GS_ERR_INVALID, "query has more than 120 distinct edges");
    d->esrc[m] = (uint8_t)a; d->edst[m] = (uint8_t)b; d->erel[m] = (uint8_t)r;
    m++;
  }
  // connectivity over the undirected view
  uint32_t seen = 1, grow = 1;
  while (grow) {
    grow = 0;
    for (uint32_t i = 0; i < m; ++i) {
      uint32_t a = 1u << d->esrc[i], b = 1u << d->edst[i];
      if ((seen & a) && !(seen & b)) { seen |= b; grow = 1; }
      if ((seen & b) && !(seen & a)) { seen |= a; grow = 1; }
    }
  }
  if (seen != ((k == 32) ? 0xFFFFFFFFu : ((1u << k) - 1)))
    return fail(GS_ERR_UNSUPPORTED, "disconnected query graphs are not supported");
  d->k = k; d->m = m;
  for (uint32_t u = 0; u < k; ++u) { d->vtype[u] = q->vtype[u]; d->vbind[u] = q->vbind[u]; }
  uint32_t ni = 0, nn = 0;
  for (uint32_t u = 0; u < k; ++u) {
    d->inc_begin[u] = (uint8_t)ni;
    d->need_begin[u] = (uint8_t)nn;
    for (uint32_t i = 0; i < m; ++i)
      if (d->esrc[i] == u || d->edst[i] == u) d->inc_edge[ni++] = (uint8_t)i;
    // degree needs per (direction, relation)
    for (uint32_t i = 0; i < m; ++i) {
      int dir = d->esrc[i] == u ? 0 : (d->edst[i] == u ? 1 : -1);
      if (dir < 0) continue;
      uint16_t plane = (uint16_t)(dir * G.R + d->erel[i]);
      bool found = false;
      for (uint32_t t = d->need_begin[u]; t < nn; ++t)
        if (d->need_plane[t] == plane) { d->need_cnt[t]++; found = true; }
      if (!found) { d->need_plane[nn] = plane; d->need_cnt[nn] = 1; nn++; }
    }
  }
  d->inc_begin[k] = (uint8_t)ni;
  d->need_begin[k] = (uint8_t)nn;
  d->mode = o ? o->mode : GS_ENUMERATE;
  d->cap = o ? o->cap : 0;
  d->force_root = 0xFF;
  d->force_from_src = 0xFF;
  d->status = QS_OK;
  return GS_OK;
}

}  // namespace gs


namespace gs {

template <typename T>
static gs_status dalloc(gs_batch *b, T **p, uint64_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (batch pools)");
  b->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return GS_OK;
}

static int bits_for(uint64_t maxval) {
  int b = 1;
  while (b < 32 && (maxval >> b)) ++b;
  return b;
}

// Pool capacities for one wave slot.
struct Sizing {
  uint64_t tlist, alist, flist, ec_items, ec_vals, lvl_words, out_rows, out_words, store_words;
};

static Sizing size_pools(const gs_batch *b, const gs_match_opts *o) {
  const uint64_t V = b->g->d.V;
  Sizing s;
  const uint64_t L = 1ull << 27;  // 128M entries per candidate-list pool at most
  s.tlist = std::min<uint64_t>((uint64_t)b->nq_s * V, L);
  s.alist = std::min<uint64_t>((uint64_t)b->nqv_s * V, L);
  s.flist = s.alist;
  s.ec_items = std::min<uint64_t>((uint64_t)b->nqe_s * V, 1ull << 27);
  s.ec_vals = std::min<uint64_t>((uint64_t)b->nqe_s * std::max<uint64_t>(b->g->d.E, 1), 1ull << 28);
  uint64_t chunk = (o && o->chunk_bytes) ? o->chunk_bytes : (1ull << 30);
  s.lvl_words = std::max<uint64_t>(chunk / 4 / 2, 1ull << 16);
  uint64_t want_rows = 0, want_words = 0;
  for (uint32_t i = 0; i < b->n; ++i) {
    if (b->hstatus[i] != GS_OK || b->hq[i].mode == GS_COUNT_ONLY) continue;
    want_rows += b->hq[i].cap;
    want_words += b->hq[i].cap * b->hq[i].k;
  }
  uint64_t per_wave_rows = 0, per_wave_words = 0;
  for (const auto &w : b->waves) {
    uint64_t r = 0, wd = 0;
    for (uint32_t i = w.q0; i < w.q0 + w.nq; ++i) {
      if (b->hstatus[i] != GS_OK || b->hq[i].mode == GS_COUNT_ONLY) continue;
      r += b->hq[i].cap;
      wd += b->hq[i].cap * b->hq[i].k;
    }
    per_wave_rows = std::max(per_wave_rows, r);
    per_wave_words = std::max(per_wave_words, wd);
  }
  s.out_rows = std::min<uint64_t>(per_wave_rows, 1ull << 25);
  s.out_words = std::min<uint64_t>(per_wave_words, 1ull << 27);
  s.store_words = std::min<uint64_t>(want_words, 1ull << 28);
  return s;
}

static gs_status batch_alloc(gs_batch *b, const gs_match_opts *o) {
  const DevGraph &G = b->g->d;
  Wave &W = b->W;
  W.G = G;
  W.nq = b->nq_s;
  W.nqv = b->nqv_s;
  W.nqe = b->nqe_s;
  const uint64_t ipg = G.ipg;
  W.slot_words = ((uint64_t)G.W0 + G.W1 + 31) / 32 * 32;
  Sizing s = size_pools(b, o);
  gs_status st;
#define A(ptr, n) \
  if ((st = dalloc(b, &(ptr), (n))) != GS_OK) return st
  A(W.dq, W.nq + 1);
  A(W.qs, W.nq);
  A(W.ctrl, 1);
  A(W.qv_q, W.nqv);
  A(W.qe_q, W.nqe);
  A(b->all_dq, b->n);
  A(b->dwaves, b->waves.size());
  W.all_dq = b->all_dq;
  W.waves = b->dwaves;
  A(W.bo.count, b->n);
  A(W.bo.fp, b->n);
  A(W.bo.nrows, b->n);
  A(W.bo.word_off, b->n);
  A(W.bo.status, b->n);
  A(W.bo.store, s.store_words);
  W.bo.store_cap = s.store_words;
  A(W.bm, (uint64_t)W.nqv * W.slot_words);
  A(W.ccount, (uint64_t)W.nqv * ipg);
  A(W.cscan, (uint64_t)W.nqv * ipg + 1);
  A(W.ascan, (uint64_t)W.nqv * ipg + 1);
  A(W.tlist, s.tlist); W.tlist_cap = s.tlist;
  A(W.alist, s.alist); W.alist_cap = s.alist;
  A(W.flist, s.flist); W.flist_cap = s.flist;
  A(W.flist_off, W.nqv);
  A(W.flist_len, W.nqv);
  A(W.ec_nkeys, W.nqe);
  A(W.ec_key_base, (uint64_t)W.nqe + 1);
  A(W.ec_cnt, s.ec_items); W.ec_items_cap = s.ec_items;
  A(W.ec_off, s.ec_items + 1);
  A(W.ec_vals, s.ec_vals); W.ec_vals_cap = s.ec_vals;
  A(W.lvl[0], s.lvl_words);
  A(W.lvl[1], s.lvl_words);
  W.lvl_words = s.lvl_words;
  W.row_cap = s.lvl_words;
  A(W.row_cnt, W.row_cap);
  A(W.row_scan, W.row_cap + 1);
  A(W.src, W.nq);
  A(W.out, s.out_words); W.out_words = s.out_words;
  A(W.out_q, s.out_rows);
  A(W.out_final, s.out_words);
  W.out_rows_cap = s.out_rows;
  for (int i = 0; i < 2; ++i) {
    A(W.skey[i], s.out_rows);
    A(W.sval[i], s.out_rows);
  }
  uint64_t tmpw = scan_tmp_words(std::max<uint64_t>({(uint64_t)W.nqv * ipg, (uint64_t)W.nqe, s.ec_items, W.row_cap}));
  tmpw = std::max(tmpw, radix_tmp_words(s.out_rows));
  A(b->scan_tmp, tmpw);
  A(b->type_count, G.T);
#undef A
  GS_CUDA(cudaMemsetAsync(W.bm, 0, sizeof(uint32_t) * (uint64_t)W.nqv * W.slot_words, b->stream));
  GS_CUDA(cudaMemsetAsync(W.ctrl, 0, sizeof(Ctrl), b->stream));
  GS_CUDA(cudaMemsetAsync(W.dq, 0, sizeof(DQuery) * (W.nq + 1), b->stream));
  uint64_t lens[3] = {(uint64_t)W.nq * ipg, (uint64_t)W.nqv * ipg, (uint64_t)W.nqe};
  GS_CUDA(cudaMemcpyAsync(W.ctrl->len, lens, sizeof(lens), cudaMemcpyHostToDevice, b->stream));
  GS_CUDA(cudaMemcpyAsync(b->type_count, b->g->type_count, sizeof(uint32_t) * G.T, cudaMemcpyHostToDevice, b->stream));
  GS_CUDA(cudaStreamSynchronize(b->stream));
  return GS_OK;
}

// Upload the packed queries and the wave table.
static gs_status batch_upload(gs_batch *b) {
  GS_CUDA(cudaMemcpyAsync(b->all_dq, b->hq.data(), sizeof(DQuery) * b->n, cudaMemcpyHostToDevice, b->stream));
  GS_CUDA(cudaMemcpyAsync(b->dwaves, b->waves.data(), sizeof(WaveDesc) * b->waves.size(), cudaMemcpyHostToDevice,
                          b->stream));
  return GS_OK;
}

// Greedy waves of consecutive queries within the slot capacities.
static void make_waves(gs_batch *b, uint32_t nq_s, uint32_t nqv_s, uint32_t nqe_s) {
  b->waves.clear();
  b->wave_k.clear();
  uint32_t i = 0, qv = 0, qe = 0;
  while (i < b->n) {
    WaveDesc w{i, 0, qv, 0, qe, 0};
    int K = 1;
    while (i < b->n && w.nq < nq_s) {
      const DQuery &d = b->hq[i];
      if (w.nq > 0 && (w.nqv + d.k > nqv_s || w.nqe + d.m > nqe_s)) break;
      b->hq[i].qv_base = qv;
      b->hq[i].qe_base = qe;
      w.nq++; w.nqv += d.k; w.nqe += d.m;
      qv += d.k; qe += d.m;
      K = std::max<int>(K, (int)d.k);
      ++i;
    }
    b->waves.push_back(w);
    b->wave_k.push_back(K);
  }
  if (b->waves.empty()) {
    b->waves.push_back(WaveDesc{0, 0, 0, 0, 0, 0});
    b->wave_k.push_back(1);
  }
}

// ------------------------------------------------------------ the pipeline
struct Rec {
  gs_batch *b;
  std::vector<gs_batch::Ev> *out;
  bool capture;
  int kind = -1;
  cudaEvent_t a = nullptr;
  void begin(int k) {
    if (!b->stats_on) return;
    kind = k;
    cudaEventCreate(&a);
    cudaEventRecordWithFlags(a, b->stream, capture ? cudaEventRecordExternal : cudaEventRecordDefault);
  }
  void end() {
    if (!b->stats_on || kind < 0) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecordWithFlags(e, b->stream, capture ? cudaEventRecordExternal : cudaEventRecordDefault);
    out->push_back({kind, a, e});
    kind = -1;
  }
};

void enqueue_wave(gs_batch *b, int K, bool capture, std::vector<gs_batch::Ev> *evs) {
  Wave &W = b->W;
  W.stats = b->stats_on ? 1 : 0;
  cudaStream_t s = b->stream;
  const int sms = b->sms, grp = b->group;
  const uint64_t ipg = W.G.ipg;
  Rec R{b, evs, capture};
  R.begin(KK_PLAN);
  launch_prologue(W, s, sms);
  launch_plan(W, b->type_count, s, sms);
  R.end();
  R.begin(KK_FILTER);
  launch_filter(W, s, sms);
  R.end();
  const int steps = K >= 2 ? K - 1 : 0;
  for (int step = 0; step < steps; ++step) {
    R.begin(KK_COMPACT);
    launch_compact_count(W, 0, step, s, sms);
    scan_u32(W.ccount, W.cscan, &W.ctrl->len[0], (uint64_t)W.nq * ipg, b->scan_tmp, s, sms);
    launch_compact_write(W, 0, step, W.cscan, W.tlist, W.tlist_cap, s, sms);
    R.end();
    R.begin(KK_EXPLORE);
    launch_explore(W, step, grp, s, sms);
    R.end();
  }
  R.begin(KK_COMPACT);
  launch_compact_count(W, 1, 0, s, sms);
  scan_u32(W.ccount, W.ascan, &W.ctrl->len[1], (uint64_t)W.nqv * ipg, b->scan_tmp, s, sms);
  launch_compact_write(W, 1, 0, W.ascan, W.alist, W.alist_cap, s, sms);
  R.end();
  R.begin(KK_REFINE);
  for (uint32_t r = 0; r < b->refine_rounds; ++r) launch_refine(W, r, grp, s, sms);
  R.end();
}

void enqueue_wave_tail(gs_batch *b, int K, bool capture, std::vector<gs_batch::Ev> *evs, int stop) {
  Wave &W = b->W;
  cudaStream_t s = b->stream;
  const int sms = b->sms, grp = b->group;
  const uint64_t ipg = W.G.ipg;
  Rec R{b, evs, capture};
  R.begin(KK_COMPACT);
  launch_compact_count(W, 1, 0, s, sms);
  scan_u32(W.ccount, W.cscan, &W.ctrl->len[1], (uint64_t)W.nqv * ipg, b->scan_tmp, s, sms);
  launch_compact_write(W, 1, 0, W.cscan, W.flist, W.flist_cap, s, sms);
  launch_list_table(W, s, sms);
  R.end();
  if (stop == 1) return;
  R.begin(KK_OTHER);
  launch_join_plan(W, s, sms);
  scan_u32(W.ec_nkeys, W.ec_key_base, &W.ctrl->len[2], W.nqe, b->scan_tmp, s, sms);
  launch_ec_limit(W, s, sms);
  R.end();
  R.begin(KK_EC_COUNT);
  launch_ec(W, false, grp, s, sms);
  R.end();
  R.begin(KK_SCAN);
  scan_u32(W.ec_cnt, W.ec_off, &W.ctrl->len[5], W.ec_items_cap, b->scan_tmp, s, sms);
  R.end();
  R.begin(KK_EC_WRITE);
  launch_ec(W, true, grp, s, sms);
  R.end();
  if (stop == 2) return;
  R.begin(KK_CLEAR);
  launch_clear(W, s, sms);
  R.end();
  R.begin(KK_OTHER);
  launch_join0(W, s, sms);
  R.end();
  for (int lvl = 0; lvl + 1 < K; ++lvl) {
    R.begin(KK_JOIN_COUNT);
    launch_join_count(W, lvl, grp, s, sms);
    R.end();
    R.begin(KK_SCAN);
    scan_u32(W.row_cnt, W.row_scan, &W.ctrl->len[3], W.row_cap, b->scan_tmp, s, sms);
    launch_join_totals(W, s, sms);
    launch_level_alloc(W, lvl + 1, s);
    R.end();
    R.begin(KK_JOIN_WRITE);
    launch_join_write(W, lvl, grp, s, sms);
    R.end();
  }
  R.begin(KK_SORT);
  launch_final_bases(W, s);
  bool rows_wanted = false;
  for (uint32_t i = 0; i < b->n; ++i)
    if (b->hstatus[i] == GS_OK && b->hq[i].mode != GS_COUNT_ONLY && b->hq[i].cap) rows_wanted = true;
  if (rows_wanted && W.out_rows_cap) {
    uint32_t *perm[2] = {W.sval[0], W.sval[1]};
    int cur = 0;
    launch_iota(W, perm[cur], s, sms);
    const int nb = bits_for(W.G.V ? W.G.V - 1 : 0);
    for (int col = K - 1; col >= 0; --col) {
      launch_sort_keys(W, perm[cur], W.skey[0], (uint32_t)col, s, sms);
      int r = radix_sort_pairs(W.skey[0], perm[cur], W.skey[1], perm[cur ^ 1], &W.ctrl->out_rows_total,
                               W.out_rows_cap, 0, nb, b->scan_tmp, s, sms);
      cur = r ? cur ^ 1 : cur;
    }
    if (W.nq > 1) {
      launch_sort_keys(W, perm[cur], W.skey[0], kMaxK, s, sms);
      int r = radix_sort_pairs(W.skey[0], perm[cur], W.skey[1], perm[cur ^ 1], &W.ctrl->out_rows_total,
                               W.out_rows_cap, 0, bits_for(W.nq - 1), b->scan_tmp, s, sms);
      cur = r ? cur ^ 1 : cur;
    }
    R.end();
    R.begin(KK_GATHER);
    launch_gather(W, perm[cur], s, sms);
  }
  R.end();
  R.begin(KK_OTHER);
  launch_epilogue(W, s, sms);
  R.end();
}

static gs_status capture_k(gs_batch *b, int K) {
  if (b->execs.count(K)) return GS_OK;
  cudaGraph_t graph;
  std::vector<gs_batch::Ev> evs;
  GS_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  enqueue_wave(b, K, true, &evs);
  enqueue_wave_tail(b, K, true, &evs, 0);
  cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t exec;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  b->execs[K] = exec;
  b->graph_evs[K] = evs;
  return GS_OK;
}

static void harvest_events(gs_batch *b, std::vector<gs_batch::Ev> &evs, bool destroy) {
  for (auto &ev : evs) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) {
      b->ms[ev.kind] += ms;
      b->launches[ev.kind] += 1;
    }
    if (destroy) {
      cudaEventDestroy(ev.a);
      cudaEventDestroy(ev.b);
    }
  }
  if (destroy) evs.clear();
}

// Host-driven refinement rounds until nothing changes (used when the graph
// is not captured and an exact fixpoint is asked for).
gs_status refine_to_fixpoint(gs_batch *b) {
  uint32_t changed[kMaxRounds];
  for (;;) {
    GS_CUDA(cudaMemcpyAsync(changed, b->W.ctrl->changed, sizeof(changed), cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaStreamSynchronize(b->stream));
    uint32_t last = b->refine_rounds - 1;
    if (!changed[last]) return GS_OK;
    GS_CUDA(cudaMemsetAsync(b->W.ctrl->changed, 0, sizeof(changed), b->stream));
    for (uint32_t r = 0; r < b->refine_rounds; ++r) launch_refine(b->W, r, b->group, b->stream, b->sms);
  }
}

gs_status run_waves(gs_batch *b) {
  GS_CUDA(cudaMemsetAsync(&b->W.ctrl->wave, 0, sizeof(uint32_t), b->stream));
  GS_CUDA(cudaMemsetAsync(&b->W.ctrl->store_top, 0, sizeof(uint64_t), b->stream));
  for (size_t w = 0; w < b->waves.size(); ++w) {
    const int K = b->wave_k[w];
    if (b->use_graph) {
      gs_status st = capture_k(b, K);
      if (st != GS_OK) return st;
      GS_CUDA(cudaGraphLaunch(b->execs[K], b->stream));
      if (b->stats_on) {
        GS_CUDA(cudaStreamSynchronize(b->stream));
        harvest_events(b, b->graph_evs[K], false);
      }
    } else {
      enqueue_wave(b, K, false, &b->evs);
      if (b->fixpoint) {
        gs_status st = refine_to_fixpoint(b);
        if (st != GS_OK) return st;
      }
      enqueue_wave_tail(b, K, false, &b->evs, 0);
      if (b->stats_on) {
        GS_CUDA(cudaStreamSynchronize(b->stream));
        harvest_events(b, b->evs, true);
      }
    }
  }
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

gs_status batch_create(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts, uint32_t wave_queries,
                       gs_batch **out) {
  *out = nullptr;
  gs_batch *b = new gs_batch();
  b->g = g;
  b->sms = g->num_sms;
  b->n = n;
  b->hq.resize(n);
  b->hstatus.resize(n);
  for (uint32_t i = 0; i < n; ++i) {
    gs_status st = pack_query(g->d, &qs[i], opts, &b->hq[i]);
    b->hstatus[i] = st;
    if (st != GS_OK) {
      memset(&b->hq[i], 0, sizeof(DQuery));
      b->hq[i].status = QS_INVALID;
    }
  }
  if (opts && opts->max_refine_rounds) {
    b->refine_rounds = std::min<uint32_t>(opts->max_refine_rounds, kMaxRounds);
    b->fixpoint = false;
  }
  const char *env_g = getenv("GS_GROUP");
  if (env_g) b->group = atoi(env_g);
  if (opts && opts->cuda_stream) {
    b->stream = static_cast<cudaStream_t>(opts->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(GS_ERR_CUDA, "cudaStreamCreate");
    }
    b->own_stream = true;
  }
  // waves: bounded by the candidate-bitmap budget
  const uint64_t slot_bytes = 4 * (((uint64_t)g->d.W0 + g->d.W1 + 31) / 32 * 32);
  const uint64_t bm_budget = 24ull << 30;
  uint64_t max_qv = std::max<uint64_t>(bm_budget / slot_bytes, kMaxK);
  uint32_t nq_s = wave_queries ? wave_queries : n;
  uint64_t tot_qv = 0, tot_qe = 0;
  for (uint32_t i = 0; i < n; ++i) { tot_qv += b->hq[i].k; tot_qe += b->hq[i].m; }
  uint32_t nqv_s = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(tot_qv, 1), max_qv);
  if (wave_queries) {
    uint32_t mk = 1, mm = 1;
    for (uint32_t i = 0; i < n; ++i) { mk = std::max(mk, b->hq[i].k); mm = std::max(mm, b->hq[i].m); }
    nqv_s = (uint32_t)std::min<uint64_t>((uint64_t)wave_queries * mk, max_qv);
    tot_qe = (uint64_t)wave_queries * mm;
  }
  uint32_t nqe_s = (uint32_t)std::max<uint64_t>(tot_qe, 1);
  nq_s = std::max<uint32_t>(nq_s, 1);
  make_waves(b, nq_s, nqv_s, nqe_s);
  uint32_t mq = 1, mqv = 1, mqe = 1;
  for (auto &w : b->waves) { mq = std::max(mq, w.nq); mqv = std::max(mqv, w.nqv); mqe = std::max(mqe, w.nqe); }
  b->nq_s = mq; b->nqv_s = mqv; b->nqe_s = mqe;
  gs_status st = batch_alloc(b, opts);
  if (st == GS_OK) st = batch_upload(b);
  if (st != GS_OK) {
    batch_destroy(b);
    return st;
  }
  *out = b;
  return GS_OK;
}

void batch_destroy(gs_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto &kv : b->execs) cudaGraphExecDestroy(kv.second);
  for (auto &kv : b->graph_evs) harvest_events(b, kv.second, true);
  harvest_events(b, b->evs, true);
  for (void *p : b->allocs) cudaFree(p);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

gs_status batch_finish(gs_batch *b) {
  if (!b->ran) return fail(GS_ERR_INVALID, "gs_batch_finish: nothing was run");
  GS_CUDA(cudaStreamSynchronize(b->stream));
  const uint32_t n = b->n;
  b->count.resize(n); b->fp.resize(n); b->nrows.resize(n); b->word_off.resize(n); b->status.resize(n);
  if (n) {
    GS_CUDA(cudaMemcpyAsync(b->count.data(), b->W.bo.count, 8ull * n, cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaMemcpyAsync(b->fp.data(), b->W.bo.fp, 8ull * n, cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaMemcpyAsync(b->nrows.data(), b->W.bo.nrows, 8ull * n, cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaMemcpyAsync(b->word_off.data(), b->W.bo.word_off, 8ull * n, cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaMemcpyAsync(b->status.data(), b->W.bo.status, 4ull * n, cudaMemcpyDeviceToHost, b->stream));
  }
  uint64_t top = 0;
  GS_CUDA(cudaMemcpyAsync(&top, &b->W.ctrl->store_top, 8, cudaMemcpyDeviceToHost, b->stream));
  GS_CUDA(cudaStreamSynchronize(b->stream));
  b->rows.resize(top);
  if (top) {
    GS_CUDA(cudaMemcpyAsync(b->rows.data(), b->W.bo.store, 4ull * top, cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaStreamSynchronize(b->stream));
  }
  b->fb_rows.assign(n, {});
  b->fb_done.assign(n, 0);
  for (uint32_t i = 0; i < n; ++i) {
    if (b->hstatus[i] != GS_OK) continue;
    if (b->status[i] == QS_OVERFLOW || b->status[i] == QS_TOPCAP) {
      gs_status st = fallback_query(b, i);
      if (st != GS_OK) return st;
    }
  }
  b->finished = true;
  return GS_OK;
}

gs_status batch_fetch(gs_batch *b, gs_result *outs) {
  if (!b->finished) return fail(GS_ERR_INVALID, "gs_batch_fetch: call gs_batch_finish first");
  for (uint32_t i = 0; i < b->n; ++i) {
    gs_result &r = outs[i];
    memset(&r, 0, sizeof(r));
    r.k = b->hq[i].k;
    if (b->hstatus[i] != GS_OK) {
      r.status = b->hstatus[i];
      continue;
    }
    const uint32_t st = b->status[i];
    r.count = b->count[i];
    r.fingerprint = b->fp[i];
    const uint64_t cap = b->hq[i].mode == GS_COUNT_ONLY ? 0 : b->hq[i].cap;
    r.truncated = r.count > cap ? 1 : 0;
    if (b->fb_done[i]) {
      r.num_rows = b->fb_rows[i].size() / (r.k ? r.k : 1);
      if (r.num_rows) {
        r.rows = static_cast<uint32_t *>(malloc(4 * b->fb_rows[i].size()));
        memcpy(r.rows, b->fb_rows[i].data(), 4 * b->fb_rows[i].size());
      }
      r.status = GS_OK;
      continue;
    }
    if (st == QS_OK || st == QS_EMPTY) {
      r.status = GS_OK;
      if (st == QS_EMPTY) { r.count = 0; r.fingerprint = 0; r.truncated = 0; }
      r.num_rows = b->nrows[i];
      if (r.num_rows) {
        const uint64_t words = r.num_rows * r.k;
        r.rows = static_cast<uint32_t *>(malloc(4 * words));
        memcpy(r.rows, b->rows.data() + b->word_off[i], 4 * words);
      }
    } else {
      r.status = GS_ERR_OOM;
    }
  }
  return GS_OK;
}

}  // namespace gs

// ------------------------------------------------------------ C ABI
extern "C" gs_status gs_batch_create(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                                     gs_batch **out) {
  if (!g || !out || (n && !qs)) return fail(GS_ERR_INVALID, "gs_batch_create: null argument");
  GS_CUDA(cudaSetDevice(g->device));
  return batch_create(g, qs, n, opts, 0, out);
}

// Waves of `wave_queries` queries each (1 = one query at a time).
extern "C" gs_status gs_batch_create_waves(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                                           uint32_t wave_queries, gs_batch **out) {
  if (!g || !out || (n && !qs)) return fail(GS_ERR_INVALID, "gs_batch_create_waves: null argument");
  GS_CUDA(cudaSetDevice(g->device));
  return batch_create(g, qs, n, opts, wave_queries, out);
}

extern "C" gs_status gs_batch_run(gs_batch *b) {
  if (!b) return fail(GS_ERR_INVALID, "gs_batch_run: null batch");
  gs_status st = run_waves(b);
  b->ran = st == GS_OK;
  b->finished = false;
  return st;
}

extern "C" gs_status gs_batch_finish(gs_batch *b) {
  if (!b) return fail(GS_ERR_INVALID, "gs_batch_finish: null batch");
  return batch_finish(b);
}

extern "C" gs_status gs_batch_fetch(gs_batch *b, gs_result *outs) {
  if (!b || !outs) return fail(GS_ERR_INVALID, "gs_batch_fetch: null argument");
  return batch_fetch(b, outs);
}

extern "C" void gs_batch_destroy(gs_batch *b) { batch_destroy(b); }

extern "C" gs_status gs_batch_set(gs_batch *b, int use_graph, int group, uint32_t refine_rounds) {
  if (!b) return fail(GS_ERR_INVALID, "gs_batch_set: null batch");
  if (group != 8 && group != 16 && group != 32) return fail(GS_ERR_INVALID, "group must be 8, 16 or 32");
  for (auto &kv : b->execs) cudaGraphExecDestroy(kv.second);
  b->execs.clear();
  for (auto &kv : b->graph_evs) harvest_events(b, kv.second, true);
  b->graph_evs.clear();
  b->use_graph = use_graph != 0;
  b->group = group;
  if (refine_rounds) {
    b->refine_rounds = std::min<uint32_t>(refine_rounds, kMaxRounds);
    b->fixpoint = false;
  } else {
    b->refine_rounds = 8;
    b->fixpoint = true;
  }
  return GS_OK;
}

extern "C" gs_status gs_match_batch(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                                    gs_result *outs) {
  if (!g || !outs || (n && !qs)) return fail(GS_ERR_INVALID, "gs_match_batch: null argument");
  gs_batch *b = nullptr;
  gs_status st = gs_batch_create(g, qs, n, opts, &b);
  if (st != GS_OK) return st;
  st = gs_batch_run(b);
  if (st == GS_OK) st = gs_batch_finish(b);
  if (st == GS_OK) st = gs_batch_fetch(b, outs);
  gs_batch_destroy(b);
  return st;
}

extern "C" gs_status gs_match(gs_graph *g, const gs_query *q, const gs_match_opts *opts, gs_result *out) {
  if (!g || !q || !out) return fail(GS_ERR_INVALID, "gs_match: null argument");
  gs_status st = gs_match_batch(g, q, 1, opts, out);
  if (st != GS_OK) return st;
  if (out->status != GS_OK) {
    gs_status qst = (gs_status)out->status;
    return fail(qst, qst == GS_ERR_INVALID ? "invalid query" : "query failed");
  }
  return GS_OK;
}

extern "C" void gs_result_free(gs_result *r) {
  if (!r) return;
  free(r->rows);
  r->rows = nullptr;
  r->num_rows = 0;
}

extern "C" gs_status gs_stats_enable(gs_batch *b, int on) {
  if (!b) return fail(GS_ERR_INVALID, "null batch");
  if ((on != 0) != b->stats_on) {
    for (auto &kv : b->execs) cudaGraphExecDestroy(kv.second);
    b->execs.clear();
    for (auto &kv : b->graph_evs) harvest_events(b, kv.second, true);
    b->graph_evs.clear();
  }
  b->stats_on = on != 0;
  return GS_OK;
}

static const char *kKindNames[GS_NUM_KERNEL_KINDS] = {
    "plan", "filter", "compact", "explore", "refine", "ec_count", "ec_write", "clear",
    "join_count", "join_write", "scan", "sort", "gather", "other", "", ""};

extern "C" gs_status gs_stats_get(gs_batch *b, gs_kernel_stats *out) {
  if (!b || !out) return fail(GS_ERR_INVALID, "null argument");
  memset(out, 0, sizeof(*out));
  uint64_t bytes[KK_N];
  GS_CUDA(cudaMemcpy(bytes, b->W.ctrl->bytes, sizeof(bytes), cudaMemcpyDeviceToHost));
  for (int i = 0; i < GS_NUM_KERNEL_KINDS; ++i) {
    out->name[i] = kKindNames[i];
    if (i < KK_N) {
      out->launches[i] = b->launches[i];
      out->ms[i] = b->ms[i];
      out->bytes[i] = bytes[i] - b->bytes_base[i];
    }
  }
  return GS_OK;
}

extern "C" gs_status gs_stats_reset(gs_batch *b) {
  if (!b) return fail(GS_ERR_INVALID, "null batch");
  GS_CUDA(cudaMemcpy(b->bytes_base, b->W.ctrl->bytes, sizeof(b->bytes_base), cudaMemcpyDeviceToHost));
  for (int i = 0; i < KK_N; ++i) { b->ms[i] = 0; b->launches[i] = 0; }
  return GS_OK;
}
