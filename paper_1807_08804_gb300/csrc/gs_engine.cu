// Host orchestration: query checks and packing, batches of waves, the
// captured pipeline graph, result transfer, and the C ABI entry points for
// matching (Algorithm "FilteringAndJoining", thesis Ch. 3).
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gs_engine.cuh"
#include "gs_host.h"

using namespace gs;

static void drop_graphs(gs_batch *b);

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
    if (r == kAny) r = kRelAny8;  // variable edge
    else if (r >= G.R) return fail(GS_ERR_INVALID, "query relation out of range");
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
    // degree needs per (direction, relation); variable edges count
    // distinct neighbours over all relations
    for (uint32_t i = 0; i < m; ++i) {
      int dir = d->esrc[i] == u ? 0 : (d->edst[i] == u ? 1 : -1);
      if (dir < 0) continue;
      uint16_t plane = (uint16_t)sig_plane(dir, d->erel[i], G.R);
      bool found = false;
      for (uint32_t t = d->need_begin[u]; t < nn; ++t)
        if (d->need_plane[t] == plane) { d->need_cnt[t]++; found = true; }
      if (!found) { d->need_plane[nn] = plane; d->need_cnt[nn] = 1; nn++; }
    }
  }
  d->inc_begin[k] = (uint8_t)ni;
  d->need_begin[k] = (uint8_t)nn;
  const uint32_t mode = o ? o->mode : GS_ENUMERATE;
  if (mode > GS_CHUNKED) return fail(GS_ERR_INVALID, "unknown match mode");
  if (mode == GS_CHUNKED && !o->on_chunk) return fail(GS_ERR_INVALID, "GS_CHUNKED needs an on_chunk callback");
  // a chunked query is counted by the batched pipeline and its embeddings
  // are streamed by the chunked join when the batch finishes
  d->mode = mode == GS_CHUNKED ? GS_COUNT_ONLY : mode;
  d->cap = o ? o->cap : 0;
  // projection (Section 3.5): output columns of the projected vertices
  const uint32_t pm = o ? o->project : 0;
  if (pm >> k) return fail(GS_ERR_INVALID, "projection names a vertex >= k");
  d->proj = pm == (1u << k) - 1 ? 0u : pm;
  if (d->proj && mode == GS_CHUNKED) return fail(GS_ERR_UNSUPPORTED, "projection with GS_CHUNKED");
  for (uint32_t u = 0; u < k; ++u)
    if (!d->proj || ((d->proj >> u) & 1u)) d->pu[d->kp++] = (uint8_t)u;
  // refinement variant
  const uint32_t rf = o ? o->refine : 0;
  if (rf & ~(GS_REFINE_OFF | GS_REFINE_REVERSED | GS_REFINE_BASELINE | GS_REFINE_LOW(0xFF)))
    return fail(GS_ERR_INVALID, "unknown refinement flags");
  d->refine_flags = (uint8_t)(((rf & GS_REFINE_OFF) ? kRefineOff : 0u) | ((rf & GS_REFINE_REVERSED) ? kRefineRev : 0u));
  if (rf & GS_REFINE_BASELINE) d->refine_flags = kRefineBase | kRefineOff;
  d->refine_low = (uint8_t)((rf >> 8) & 0xFFu);
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
  cudaError_t e = gs::dev_malloc(&q, sizeof(T) * (count ? count : 1));
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
  // Candidate lists and edge tables sized from upper bounds of the initial
  // candidate sets (a bound vertex: 1; a typed one: the vertices of its type;
  // an untyped one: V), per wave, capped; a query that needs more than the
  // caps finishes on the fallback path, which has pools of its own.
  auto clampu = [](uint64_t x, uint64_t lo, uint64_t hi) { return std::min(std::max(x, lo), hi); };
  auto est = [&](const DQuery &d, uint32_t u) -> uint64_t {
    if (d.vbind[u] != kUnbound) return 1;
    if (d.vtype[u] != kAny && d.vtype[u] < b->g->d.T) return b->g->type_count[d.vtype[u]];
    return V;
  };
  uint64_t w_t = 0, w_a = 0, w_e = 0;
  for (const auto &w : b->waves) {
    uint64_t t = 0, a = 0, e = 0;
    for (uint32_t i = w.q0; i < w.q0 + w.nq && i < b->n; ++i) {
      const DQuery &d = b->hq[i];
      uint64_t mx = 0;
      for (uint32_t u = 0; u < d.k; ++u) { a += est(d, u); mx = std::max(mx, est(d, u)); }
      t += mx;
      for (uint32_t j = 0; j < d.m; ++j) e += std::max(est(d, d.esrc[j]), est(d, d.edst[j]));
    }
    w_t = std::max(w_t, t); w_a = std::max(w_a, a); w_e = std::max(w_e, e);
  }
  s.tlist = clampu(w_t, 1ull << 20, 1ull << 28);
  s.alist = clampu(w_a, 1ull << 20, 1ull << 28);
  s.flist = s.alist;
  s.ec_items = clampu(w_e, 1ull << 20, 1ull << 28);
  s.ec_vals = clampu(4 * w_e, 1ull << 20, 1ull << 29);
  if (b->pool_hint) {  // capacity-created batches (serving slots): fixed pools
    s.tlist = s.alist = s.flist = s.ec_items = b->pool_hint;
    s.ec_vals = 4 * b->pool_hint;
  }
  uint64_t chunk = (o && o->chunk_bytes) ? o->chunk_bytes : (1ull << 30);
  s.lvl_words = std::max<uint64_t>(std::min<uint64_t>(chunk / 4 / 2, std::max<uint64_t>((uint64_t)b->nq_s << 16, 1ull << 22)), 1ull << 16);
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
  if (b->big) {  // the fallback context: large filtering pools, join buffers of its own
    s.tlist = std::min<uint64_t>((uint64_t)b->nq_s * V, 1ull << 28);
    s.alist = s.flist = std::min<uint64_t>((uint64_t)b->nqv_s * V, 1ull << 28);
    s.ec_items = std::min<uint64_t>((uint64_t)b->nqe_s * V, 1ull << 28);
    s.ec_vals = 1ull << 29;
    s.lvl_words = 1ull << 16;
    s.out_rows = s.out_words = s.store_words = 1ull << 10;
  }
  return s;
}

static gs_status batch_alloc(gs_batch *b, const gs_match_opts *o) {
  const DevGraph &G = b->g->d;
  Wave &W = b->W;
  W.G = G;
  W.nq = b->nq_s;
  W.nqv = b->nqv_s;
  W.nqe = b->nqe_s;
  const uint64_t cps = G.nchunks;  // chunks per set: one candidate count per chunk
  W.slot_words = ((uint64_t)G.W0 + G.W1 + G.ipg + 31) / 32 * 32;
  Sizing s = size_pools(b, o);
  gs_status st;
#define A(ptr, n) \
  if ((st = dalloc(b, &(ptr), (n))) != GS_OK) return st
  A(W.dq, W.nq + 1);
  A(W.qs, W.nq);
  A(W.ctrl, 1);
  A(W.qv_q, W.nqv);
  A(W.qe_q, W.nqe);
  A(b->all_dq, b->n_cap);
  A(b->dwaves, std::max<size_t>(b->n_cap, b->waves.size()));
  W.all_dq = b->all_dq;
  W.waves = b->dwaves;
  A(W.bo.count, b->n_cap);
  A(W.bo.fp, b->n_cap);
  A(W.bo.nrows, b->n_cap);
  A(W.bo.word_off, b->n_cap);
  A(W.bo.inter, b->n_cap);
  A(W.bo.peak, b->n_cap);
  A(W.bo.status, b->n_cap);
  A(W.bo.store, s.store_words);
  W.bo.store_cap = s.store_words;
  A(W.bm, (uint64_t)W.nqv * W.slot_words);
  A(W.ccount, (uint64_t)W.nqv * cps);
  A(W.cscan, (uint64_t)W.nqv * cps + 1);
  A(W.ascan, (uint64_t)W.nqv * cps + 1);
  A(W.tlist, s.tlist); W.tlist_cap = s.tlist;
  A(W.alist, s.alist); W.alist_cap = s.alist;
  A(W.tlist_q, s.tlist);
  A(W.alist_q, s.alist);
  A(W.fcnt, W.nq);
  if ((uint64_t)W.nqv * cps >= (1ull << 32)) return fail(GS_ERR_UNSUPPORTED, "batch too large for the chunk index");
  A(W.clist, (uint64_t)W.nqv * cps);
  A(W.fscan, (uint64_t)W.nq + 1);
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
  A(W.lsz, W.nq);
  A(W.out, s.out_words); W.out_words = s.out_words;
  A(W.out_q, s.out_rows);
  A(W.out_final, s.out_words);
  W.out_rows_cap = s.out_rows;
  for (int i = 0; i < 2; ++i) {
    A(W.skey[i], s.out_rows);
    A(W.sval[i], s.out_rows);
  }
  A(W.bkt_id, s.out_rows);
  // per tile of the large-output sort, with kBktPerTile bucket slots per tile
  A(W.msplit, kBktPerTile * (s.out_rows / kTileRows + W.nq + 1));
  A(W.bspl_key, kBktPerTile * (s.out_rows / kTileRows + W.nq + 1));
  A(W.bspl_key2, kBktPerTile * (s.out_rows / kTileRows + W.nq + 1));
  A(W.bspl_row, kBktPerTile * (s.out_rows / kTileRows + W.nq + 1));
  A(W.ptcount, kBktPerTile * (s.out_rows / kTileRows + W.nq + 1));
  A(W.ptscan, kBktPerTile * (s.out_rows / kTileRows + W.nq + 1) + 1);
  A(W.sel, W.nq);
  A(W.shist, (uint64_t)W.nq * 256);
  uint64_t tmpw = scan_tmp_words(std::max<uint64_t>(
      {(uint64_t)W.nqv * cps, (uint64_t)W.nqe, s.ec_items, W.row_cap, kBktPerTile * (s.out_rows / kTileRows + W.nq + 1)}));
  A(b->scan_tmp, tmpw);
  b->scan_tmp_words = tmpw;
  A(b->type_count, G.T);
#undef A
  GS_CUDA(cudaMemsetAsync(W.bm, 0, sizeof(uint32_t) * (uint64_t)W.nqv * W.slot_words, b->stream));
  GS_CUDA(cudaMemsetAsync(b->scan_tmp, 0, sizeof(uint64_t) * b->scan_tmp_words, b->stream));
  GS_CUDA(cudaMemsetAsync(W.shist, 0, sizeof(uint32_t) * (uint64_t)W.nq * 256, b->stream));
  GS_CUDA(cudaMemsetAsync(W.ctrl, 0, sizeof(Ctrl), b->stream));
  GS_CUDA(cudaMemsetAsync(W.dq, 0, sizeof(DQuery) * (W.nq + 1), b->stream));
  const uint64_t lens[3] = {(uint64_t)W.nq * cps, (uint64_t)W.nqv * cps, (uint64_t)W.nqe};
  GS_CUDA(cudaMemcpyAsync(W.ctrl->len, lens, sizeof(lens), cudaMemcpyHostToDevice, b->stream));
  const uint64_t nq = W.nq;
  GS_CUDA(cudaMemcpyAsync(&W.ctrl->len[8], &nq, sizeof(nq), cudaMemcpyHostToDevice, b->stream));
  GS_CUDA(cudaMemcpyAsync(b->type_count, b->g->type_count, sizeof(uint32_t) * G.T, cudaMemcpyHostToDevice, b->stream));
  GS_CUDA(cudaStreamSynchronize(b->stream));
  return GS_OK;
}

// Upload the packed queries and the wave table.
static gs_status batch_upload(gs_batch *b) {
  b->last_upload_bytes = sizeof(DQuery) * b->n + sizeof(WaveDesc) * b->waves.size();
  b->h2d_bytes += b->last_upload_bytes;
  if (b->n)
    GS_CUDA(cudaMemcpyAsync(b->all_dq, b->hq.data(), sizeof(DQuery) * b->n, cudaMemcpyHostToDevice, b->stream));
  GS_CUDA(cudaMemcpyAsync(b->dwaves, b->waves.data(), sizeof(WaveDesc) * b->waves.size(), cudaMemcpyHostToDevice,
                          b->stream));
  return GS_OK;
}

gs_status batch_set_wmasks(gs_batch *b, const uint64_t *wmask, uint32_t wstride, const uint32_t *wgroup) {
  for (uint32_t i = 0; i < b->n; ++i) {
    b->hq[i].wmask = wmask[i];
    b->hq[i].wstride = wstride;
    b->hq[i].wgroup = (uint64_t)(uintptr_t)wgroup;
  }
  return batch_upload(b);
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
// ------------------------------------------------------------ capture
// The pipeline of one wave is captured once per query size K as CUDA graphs
// (every launch is persistent over device-sized work, so one graph serves
// every wave): graph A runs plan through the one-block sort of small
// outputs; graph B, launched only when some query has more than 2,048
// output rows, sorts those outputs with the radix passes; graph C moves the
// wave's results to the batch store.  Kernels with no work for a wave return
// at once.
struct Pipe {
  gs_batch *b;
  std::vector<gs_batch::Ev> *evs;
  bool capture;      // inside stream capture
  cudaStream_t cur;  // stream receiving launches
  int kind = -1;
  cudaEvent_t ev0 = nullptr;

  void begin(int k) {
    if (!b->stats_on) return;
    kind = k;
    cudaEventCreate(&ev0);
    cudaEventRecordWithFlags(ev0, cur, capture ? cudaEventRecordExternal : cudaEventRecordDefault);
  }
  void end() {
    if (!b->stats_on || kind < 0) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecordWithFlags(e, cur, capture ? cudaEventRecordExternal : cudaEventRecordDefault);
    evs->push_back({kind, ev0, e});
    kind = -1;
  }
};

static bool rows_wanted(const gs_batch *b) {
  for (uint32_t i = 0; i < b->n; ++i)
    if (b->hstatus[i] == GS_OK && b->hq[i].mode != GS_COUNT_ONLY && b->hq[i].cap) return b->W.out_rows_cap > 0;
  return false;
}

// Refinement rounds of a wave: one launch per round, or, when a query asks
// for the reversed order, one launch per query vertex position per round.
void launch_refine_rounds(gs_batch *b, const Wave &W, int K, cudaStream_t s) {
  for (uint32_t r = 0; r < b->refine_rounds; ++r) {
    if (!b->has_rev) {
      launch_refine(W, r, kAllSub, b->group, s, b->sms);
      continue;
    }
    for (int j = 0; j < std::max(K, 1); ++j) launch_refine(W, r, (uint32_t)j, b->group, s, b->sms);
  }
}

void enqueue_front(Pipe &P, int K) {
  gs_batch *b = P.b;
  Wave &W = b->W;
  W.stats = b->stats_on ? 1 : 0;
  const int sms = b->sms, grp = b->group;
  const uint64_t cps = W.G.nchunks;  // chunks per set: one candidate count per chunk
  P.begin(KK_PLAN);
  launch_prologue(W, P.cur, sms);
  launch_plan(W, b->type_count, P.cur, sms);
  P.end();
  P.begin(KK_FILTER);
  scan_u32(W.fcnt, W.fscan, &W.ctrl->len[8], W.nq, b->scan_tmp, P.cur, sms);
  launch_filter(W, P.cur, sms);
  P.end();
  const int steps = K >= 2 ? K - 1 : 0;
  for (int step = 0; step < steps; ++step) {
    P.begin(KK_COMPACT);
    launch_compact_claim(W, step, P.cur, sms);
    P.end();
    P.begin(KK_EXPLORE);
    launch_explore(W, step, grp, P.cur, sms);
    P.end();
  }
  // the refinement work list (every candidate of every query vertex) is
  // needed only when some refinement round will run
  const bool refines = b->refine_rounds > 0 || (!b->use_graph && b->fixpoint);
  if (!refines) return;
  P.begin(KK_COMPACT_ALL);
  launch_compact_count(W, 1, 0, P.cur, sms);
  scan_u32(W.ccount, W.ascan, &W.ctrl->len[1], (uint64_t)W.nqv * cps, b->scan_tmp, P.cur, sms);
  launch_compact_write(W, 1, 0, W.ascan, W.alist, W.alist_q, W.alist_cap, HW_ALIST, P.cur, sms);
  P.end();
  P.begin(KK_REFINE);
  launch_refine_rounds(b, W, K, P.cur);
  P.end();
}

// stop: 0 = through the one-block sort, 1 = after the final candidate lists,
// 2 = after the candidate-edge tables.
void enqueue_back(Pipe &P, int K, int stop) {
  gs_batch *b = P.b;
  Wave &W = b->W;
  const int sms = b->sms, grp = b->group, jgrp = b->jgroup ? b->jgroup : b->group;
  const uint64_t cps = W.G.nchunks;  // chunks per set: one candidate count per chunk
  P.begin(KK_COMPACT_ALL);
  launch_compact_count(W, 1, 0, P.cur, sms);
  scan_u32(W.ccount, W.cscan, &W.ctrl->len[1], (uint64_t)W.nqv * cps, b->scan_tmp, P.cur, sms);
  launch_compact_write(W, 1, 0, W.cscan, W.flist, nullptr, W.flist_cap, HW_FLIST, P.cur, sms);
  launch_list_table(W, P.cur, sms);
  P.end();
  if (stop == 1) return;
  P.begin(KK_OTHER);
  launch_join_plan(W, P.cur, sms);
  scan_u32(W.ec_nkeys, W.ec_key_base, &W.ctrl->len[2], W.nqe, b->scan_tmp, P.cur, sms);
  launch_ec_limit(W, P.cur, sms);
  P.end();
  P.begin(KK_EC_COUNT);
  launch_ec(W, false, grp, P.cur, sms);
  P.end();
  P.begin(KK_SCAN);
  scan_u32(W.ec_cnt, W.ec_off, &W.ctrl->len[5], W.ec_items_cap, b->scan_tmp, P.cur, sms);
  P.end();
  P.begin(KK_EC_WRITE);
  launch_ec(W, true, grp, P.cur, sms);
  P.end();
  if (stop == 2) return;
  P.begin(KK_CLEAR);
  launch_clear(W, P.cur, sms);
  P.end();
  P.begin(KK_OTHER);
  launch_join0(W, P.cur, sms);
  P.end();
  for (int lvl = 0; lvl + 1 < K; ++lvl) {
    P.begin(KK_JOIN_COUNT);
    launch_join_count(W, lvl, jgrp, P.cur, sms);
    P.end();
    P.begin(KK_SCAN);
    scan_u32(W.row_cnt, W.row_scan, &W.ctrl->len[3], W.row_cap, b->scan_tmp, P.cur, sms);
    launch_level_alloc(W, lvl + 1, P.cur);
    P.end();
    P.begin(KK_JOIN_WRITE);
    launch_join_write(W, lvl, jgrp, P.cur, sms);
    P.end();
  }
  P.begin(KK_SORT);
  launch_final_bases(W, P.cur);
  if (rows_wanted(b)) launch_small_sort(W, P.cur, sms);
  P.end();
}

// Sort of the outputs above the one-block limit (launched directly: the
// host reads the largest output first): a sample sort into buckets of about
// one tile, each sorted in shared memory; a query with an overflowing bucket
// takes the tile sort and ceil(log2(largest / tile)) merge passes instead
// (those launches return at once when no query needs them).
// Launches of enqueue_large_sort for the largest output and the number of
// outputs cut at cap.
uint64_t large_sort_launches(uint64_t max_rows, uint64_t over_cap, bool proj) {
  uint64_t passes = 0;
  for (uint64_t run = kTileRows; run < max_rows; run *= 2) ++passes;
  return 3 + 8 + 2 * passes + (over_cap ? 3 + 2 * 3 : 0) + (proj ? 3 : 0);
}

void enqueue_large_sort(Pipe &P, uint64_t max_rows, uint64_t over_cap, bool proj) {
  gs_batch *b = P.b;
  Wave &W = b->W;
  const int sms = b->sms;
  uint32_t *perm[2] = {W.sval[0], W.sval[1]};
  SortKey *keys[2] = {W.skey[0], W.skey[1]};
  int cur = 0;
  P.begin(KK_SORT_LARGE);
  launch_sort_keys(W, perm[0], keys[0], P.cur, sms);
  int in = 0;
  if (over_cap) {  // cut the outputs above cap to about cap rows before sorting
    launch_select(W, perm[0], keys[0], perm[1], keys[1], P.cur, sms);
    in = 1;
  }
  const int x = in ^ 1;  // the scatter's target: the other buffer
  launch_bucket_sort(W, perm[in], keys[in], perm[x], keys[x], perm[0], keys[0], perm[1], keys[1], b->scan_tmp, P.cur,
                     sms);
  launch_tile_sort(W, perm[in], keys[in], perm[0], keys[0], P.cur, sms);
  for (uint64_t run = kTileRows; run < max_rows; run *= 2) {
    launch_merge_pass(W, perm[cur], keys[cur], perm[cur ^ 1], keys[cur ^ 1], run, P.cur, sms);
    cur ^= 1;
  }
  P.end();
  P.begin(KK_GATHER);
  launch_gather(W, perm[0], perm[1], P.cur, sms);
  if (proj)  // projected outputs: first row of each distinct tuple, first cap of them
    launch_project(W, perm[0], perm[1], keys[0], keys[1], W.out_rows_cap / kTileRows + W.nq + 1, b->scan_tmp, P.cur,
                   sms);
  P.end();
}

// Results of the wave into the batch store (graph C).
void enqueue_epilogue(Pipe &P) {
  P.begin(KK_OTHER);
  launch_epilogue(P.b->W, P.cur, P.b->sms);
  P.end();
}

void enqueue_wave(gs_batch *b, int K, bool capture, std::vector<gs_batch::Ev> *evs) {
  Pipe P{b, evs, capture, b->stream};
  enqueue_front(P, K);
}

void enqueue_wave_tail(gs_batch *b, int K, bool capture, std::vector<gs_batch::Ev> *evs, int stop) {
  Pipe P{b, evs, capture, b->stream};
  enqueue_back(P, K, stop);
}

// Capture one segment of the pipeline into an executable graph.
template <typename F>
static gs_status capture_one(gs_batch *b, F body, cudaGraphExec_t *exec, std::vector<gs_batch::Ev> *evs,
                             uint64_t *kernels) {
  cudaGraph_t graph;
  GS_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  Pipe P{b, evs, true, b->stream};
  body(P);
  cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline capture");
  size_t nn = 0;
  cudaGraphGetNodes(graph, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
  uint64_t kern = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) kern++;
  }
  *kernels = kern;
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return GS_OK;
}

static gs_status capture_k(gs_batch *b, int K) {
  if (b->execs.count(K)) return GS_OK;
  cudaGraphExec_t a = nullptr;
  std::vector<gs_batch::Ev> ea;
  uint64_t ka = 0;
  gs_status st = capture_one(b, [&](Pipe &P) { enqueue_front(P, K); enqueue_back(P, K, 0); }, &a, &ea, &ka);
  if (st != GS_OK) return st;
  if (!b->epi_exec) {
    st = capture_one(b, [&](Pipe &P) { enqueue_epilogue(P); }, &b->epi_exec, &b->epi_evs, &b->epi_kernels);
    if (st != GS_OK) return st;
  }
  b->execs[K] = a;
  b->graph_evs[K] = ea;
  b->kernels_per_exec[K] = ka;
  return GS_OK;
}

static void harvest_events(gs_batch *b, std::vector<gs_batch::Ev> &evs, bool destroy) {
  for (auto &ev : evs) {
    float ms = 0, t0 = 0, t1 = 0;
    if (cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) {
      b->ms[ev.kind] += ms;
      b->launches[ev.kind] += 1;
      if (b->anchor && cudaEventElapsedTime(&t0, b->anchor, ev.a) == cudaSuccess &&
          cudaEventElapsedTime(&t1, b->anchor, ev.b) == cudaSuccess)
        b->spans.push_back({b->run_id, ev.kind, t0, t1});
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
  if (b->refine_rounds == 0) {  // a batch set to skip refinement ran no round yet
    b->refine_rounds = 1;
    launch_refine_rounds(b, b->W, b->max_k, b->stream);
  }
  for (;;) {
    GS_CUDA(cudaMemcpyAsync(changed, b->W.ctrl->changed, sizeof(changed), cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaStreamSynchronize(b->stream));
    uint32_t last = b->refine_rounds - 1;
    if (!changed[last]) return GS_OK;
    GS_CUDA(cudaMemsetAsync(b->W.ctrl->changed, 0, sizeof(changed), b->stream));
    launch_refine_rounds(b, b->W, b->max_k, b->stream);
  }
}

// A run of a batch: every wave in two halves.  The first half launches the
// wave's pipeline and, when rows are wanted, copies the large-output flags
// to pinned host words; the second half, once those words have arrived,
// sorts the large outputs if there are any and moves the wave's results to
// the batch store.
static std::atomic<uint64_t> g_run_ids{0};

static gs_status run_reset(gs_batch *b) {
  if (b->stats_on && !b->shared_anchor) {
    if (!b->own_anchor) GS_CUDA(cudaEventCreate(&b->own_anchor));
    GS_CUDA(cudaEventRecord(b->own_anchor, b->stream));
    b->anchor = b->own_anchor;
    b->run_id = ++g_run_ids;
  }
  GS_CUDA(cudaMemsetAsync(b->W.ctrl->hw, 0, sizeof(b->W.ctrl->hw), b->stream));
  GS_CUDA(cudaMemsetAsync(&b->W.ctrl->wave, 0, sizeof(uint32_t), b->stream));
  GS_CUDA(cudaMemsetAsync(&b->W.ctrl->store_top, 0, sizeof(uint64_t), b->stream));
  if (!b->flag) GS_CUDA(cudaMallocHost((void **)&b->flag, 3 * sizeof(uint64_t)));
  b->sorting = rows_wanted(b);
  return GS_OK;
}

static gs_status wave_begin(gs_batch *b, size_t w) {
  const int K = b->wave_k[w];
  if (b->use_graph) {
    gs_status st = capture_k(b, K);
    if (st != GS_OK) return st;
    GS_CUDA(cudaGraphLaunch(b->execs[K], b->stream));
    b->kernel_launches += b->kernels_per_exec[K];
  } else {
    enqueue_wave(b, K, false, &b->evs);
    if (b->fixpoint) {
      gs_status st = refine_to_fixpoint(b);
      if (st != GS_OK) return st;
    }
    enqueue_wave_tail(b, K, false, &b->evs, 0);
  }
  if (b->sorting) {  // any output too large for the one-block sort?
    GS_CUDA(cudaMemcpyAsync(b->flag, &b->W.ctrl->len[6], sizeof(uint64_t), cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaMemcpyAsync(b->flag + 1, &b->W.ctrl->max_large_rows, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                            b->stream));
    GS_CUDA(cudaMemcpyAsync(b->flag + 2, &b->W.ctrl->over_cap, sizeof(uint64_t), cudaMemcpyDeviceToHost, b->stream));
  }
  return GS_OK;
}

// Read a finished wave's launch events (graph events are re-recorded by the
// next launch of their graph, so this comes before it).
static gs_status harvest_wave(gs_batch *b, int K) {
  GS_CUDA(cudaStreamSynchronize(b->stream));
  if (b->use_graph) {
    harvest_events(b, b->graph_evs[K], false);
    harvest_events(b, b->sort_evs_direct, true);
    harvest_events(b, b->epi_evs, false);
  } else {
    harvest_events(b, b->evs, true);
  }
  return GS_OK;
}

static gs_status wave_end(gs_batch *b, size_t w) {
  const int K = b->wave_k[w];
  if (b->sorting && b->flag[0] != 0) {
    Pipe P{b, &b->sort_evs_direct, false, b->stream};
    enqueue_large_sort(P, b->flag[1], b->flag[2], b->has_proj);
    b->kernel_launches += large_sort_launches(b->flag[1], b->flag[2], b->has_proj);
    b->large_sorts++;
  }
  if (b->use_graph) {
    GS_CUDA(cudaGraphLaunch(b->epi_exec, b->stream));
    b->kernel_launches += b->epi_kernels;
  } else {
    Pipe P{b, &b->evs, false, b->stream};
    enqueue_epilogue(P);
  }
  if (b->stats_on && !b->defer_harvest) return harvest_wave(b, K);
  return GS_OK;
}

gs_status run_waves(gs_batch *b) {
  gs_status st = run_reset(b);
  for (size_t w = 0; w < b->waves.size() && st == GS_OK; ++w) {
    st = wave_begin(b, w);
    if (st == GS_OK && b->sorting) GS_CUDA(cudaStreamSynchronize(b->stream));
    if (st == GS_OK) st = wave_end(b, w);
  }
  if (st != GS_OK) return st;
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

gs_status run_begin(gs_batch *b) {
  if (b->waves.size() != 1) return fail(GS_ERR_INVALID, "run_begin: one wave only");
  gs_status st = run_reset(b);
  if (st == GS_OK) st = wave_begin(b, 0);
  return st;
}

gs_status run_end(gs_batch *b) {
  gs_status st = wave_end(b, 0);
  if (st != GS_OK) return st;
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}

// Several batches at once, each on its own stream, after the work queued on
// `parent`: first halves of every batch (pipeline graphs), then, once each
// one's large-output flags are on the host, the second halves, so the
// batches' kernels overlap on the device and one batch's steps with few work
// items run beside another's bulk work; `parent` then waits for all of them.
gs_status run_batches(gs_batch *const *bs, uint32_t nb, cudaStream_t parent) {
  bool stats = false, multi = false;
  for (uint32_t i = 0; i < nb; ++i) {
    stats = stats || bs[i]->stats_on;
    multi = multi || bs[i]->waves.size() != 1;
  }
  cudaEvent_t ev = nullptr;  // the fork; with timing on, the run's shared anchor
  GS_CUDA(cudaEventCreateWithFlags(&ev, stats ? cudaEventDefault : cudaEventDisableTiming));
  gs_status st = GS_OK;
  if (cudaEventRecord(ev, parent) != cudaSuccess) st = fail(GS_ERR_CUDA, "run_batches: fork");
  const uint64_t run = stats ? ++g_run_ids : 0;
  for (uint32_t i = 0; i < nb && st == GS_OK; ++i) {
    if (cudaStreamWaitEvent(bs[i]->stream, ev, 0) != cudaSuccess) st = fail(GS_ERR_CUDA, "run_batches: wait");
    if (bs[i]->stats_on) {
      bs[i]->anchor = ev;
      bs[i]->shared_anchor = true;
      bs[i]->run_id = run;
      bs[i]->defer_harvest = !multi;
    }
  }
  for (uint32_t i = 0; i < nb && st == GS_OK; ++i) {
    bs[i]->ran = false;
    bs[i]->finished = false;
    st = multi ? run_waves(bs[i]) : run_begin(bs[i]);
  }
  for (uint32_t i = 0; i < nb && st == GS_OK && !multi; ++i)
    if (bs[i]->sorting && cudaStreamSynchronize(bs[i]->stream) != cudaSuccess) st = fail(GS_ERR_CUDA, "run_batches: sync");
  for (uint32_t i = 0; i < nb && st == GS_OK && !multi; ++i) st = run_end(bs[i]);
  // with timing on, each batch's events are read once all of them are queued,
  // so that the batches' launches still overlap
  for (uint32_t i = 0; i < nb; ++i) {
    gs_batch *b = bs[i];
    if (b->stats_on && b->defer_harvest && st == GS_OK) st = harvest_wave(b, b->wave_k[0]);
    if (b->anchor == ev) {
      b->anchor = nullptr;
      b->shared_anchor = false;
      b->defer_harvest = false;
    }
  }
  cudaEvent_t join = nullptr;
  if (st == GS_OK && cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess)
    st = fail(GS_ERR_CUDA, "run_batches: join event");
  for (uint32_t i = 0; i < nb && st == GS_OK; ++i) {
    bs[i]->ran = true;
    if (cudaEventRecord(join, bs[i]->stream) != cudaSuccess || cudaStreamWaitEvent(parent, join, 0) != cudaSuccess)
      st = fail(GS_ERR_CUDA, "run_batches: join");
  }
  if (join) cudaEventDestroy(join);
  cudaEventDestroy(ev);
  return st;
}

static void pack_all(gs_batch *b, const gs_query *qs, uint32_t n, const gs_match_opts *opts) {
  const bool had_rev = b->has_rev;
  b->n = n;
  b->hq.resize(n);  // pack_query clears each entry before filling it
  b->hstatus.assign(n, GS_OK);
  b->has_proj = b->has_rev = false;
  b->max_k = 1;
  // queries pack independently: large batches split over host threads
  auto pack_range = [&](uint32_t i0, uint32_t i1) {
    for (uint32_t i = i0; i < i1; ++i) {
      gs_status st = pack_query(b->g->d, &qs[i], opts, &b->hq[i]);
      b->hstatus[i] = st;
      if (st != GS_OK) {
        memset(&b->hq[i], 0, sizeof(DQuery));
        b->hq[i].status = QS_INVALID;
      }
    }
  };
  const uint32_t hw = std::max(1u, std::min(8u, std::thread::hardware_concurrency()));
  const uint32_t nt = n >= 2048 ? hw : 1;
  if (nt > 1) {
    std::vector<std::thread> th;
    for (uint32_t t = 0; t < nt; ++t)
      th.emplace_back(pack_range, (uint32_t)((uint64_t)n * t / nt), (uint32_t)((uint64_t)n * (t + 1) / nt));
    for (auto &x : th) x.join();
  } else {
    pack_range(0, n);
  }
  for (uint32_t i = 0; i < n; ++i) {
    b->has_proj = b->has_proj || b->hq[i].proj != 0;
    b->has_rev = b->has_rev || (b->hq[i].refine_flags & kRefineRev);
    b->max_k = std::max<uint32_t>(b->max_k, b->hq[i].k);
  }
  // the captured graphs launch refinement once per round, or once per query
  // vertex position per round for the reversed order: recapture on a change
  if (b->has_rev != had_rev) ::drop_graphs(b);
  b->ran = b->finished = false;
}

static void opts_key(gs_batch *b, const gs_match_opts *opts) {
  const bool chunked = opts && opts->mode == GS_CHUNKED;
  b->on_chunk = chunked ? opts->on_chunk : nullptr;
  b->chunk_user = chunked ? opts->user : nullptr;
  b->key_cap = opts ? opts->cap : 0;
  b->key_mode = opts ? opts->mode : 0;
  b->key_rounds = opts ? opts->max_refine_rounds : 0;
  b->key_chunk = opts ? opts->chunk_bytes : 0;
  b->key_stream = opts ? opts->cuda_stream : nullptr;
}

static bool opts_match(const gs_batch *b, const gs_match_opts *opts) {
  return b->key_cap == (opts ? opts->cap : 0) && b->key_mode == (opts ? opts->mode : 0) &&
         b->key_rounds == (opts ? opts->max_refine_rounds : 0) && b->key_chunk == (opts ? opts->chunk_bytes : 0) &&
         b->key_stream == (opts ? opts->cuda_stream : nullptr);
}

gs_status batch_create(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts, uint32_t wave_queries,
                       gs_batch **out, bool big) {
  *out = nullptr;
  gs_batch *b = new gs_batch();
  b->g = g;
  b->big = big;
  b->sms = g->num_sms;
  pack_all(b, qs, n, opts);
  b->n_cap = std::max<uint32_t>(n, 1);
  opts_key(b, opts);
  if (g->tuned_group) b->group = g->tuned_group;
  b->jgroup = (int)g->tuned_jgroup;
  if (g->tuned_rounds) b->refine_rounds = g->tuned_rounds == GS_ROUNDS_NONE ? 0 : g->tuned_rounds;
  if (opts && opts->max_refine_rounds) {
    b->refine_rounds = std::min<uint32_t>(opts->max_refine_rounds, kMaxRounds);
    b->fixpoint = false;
  }
  if (opts && opts->cuda_stream) {
    b->stream = static_cast<cudaStream_t>(opts->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(GS_ERR_CUDA, "cudaStreamCreate");
    }
    b->own_stream = true;
  }
  // waves: bounded by the candidate-bitmap budget, a quarter of the free
  // device memory (at least 4 GB, at most 64 GB), so that on a large GPU a
  // batch of thousands of queries runs as one wave
  const uint64_t slot_bytes = 4 * (((uint64_t)g->d.W0 + g->d.W1 + g->d.ipg + 31) / 32 * 32);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = 0;
  }
  const uint64_t bm_budget = std::min<uint64_t>(std::max<uint64_t>(free_b / 4, 4ull << 30), 64ull << 30);
  uint64_t max_qv = std::max<uint64_t>(bm_budget / slot_bytes, kMaxK);
  uint32_t nq_s = wave_queries ? wave_queries : n;
  uint64_t tot_qv = 0, tot_qe = 0;
  uint32_t mk = 1, mm = 1;
  for (uint32_t i = 0; i < n; ++i) {
    tot_qv += b->hq[i].k; tot_qe += b->hq[i].m;
    mk = std::max(mk, b->hq[i].k); mm = std::max(mm, b->hq[i].m);
  }
  uint32_t nqv_s = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(tot_qv, 1), max_qv);
  if (wave_queries) {
    nqv_s = (uint32_t)std::min<uint64_t>((uint64_t)wave_queries * mk, max_qv);
    tot_qe = (uint64_t)wave_queries * mm;
  }
  nqv_s = std::max<uint32_t>(nqv_s, mk);
  uint32_t nqe_s = (uint32_t)std::max<uint64_t>({tot_qe, (uint64_t)mm, 1});
  nq_s = std::max<uint32_t>(nq_s, 1);
  make_waves(b, nq_s, nqv_s, nqe_s);
  uint32_t mq = 1, mqv = 1, mqe = 1;
  for (auto &w : b->waves) { mq = std::max(mq, w.nq); mqv = std::max(mqv, w.nqv); mqe = std::max(mqe, w.nqe); }
  b->nq_s = mq; b->nqv_s = mqv; b->nqe_s = mqe;
  if (big) { b->nq_s = 1; b->nqv_s = kMaxK; b->nqe_s = kMaxM; }
  gs_status st = batch_alloc(b, opts);
  if (st == GS_OK) st = batch_upload(b);
  if (st != GS_OK) {
    batch_destroy(b);
    return st;
  }
  *out = b;
  return GS_OK;
}

// An empty batch with fixed capacities (queries come later through
// batch_rearm): n_cap queries, nqv_s query vertices and nqe_s query edges in
// one wave.
gs_status batch_create_capacity(gs_graph *g, const gs_match_opts *opts, uint32_t n_cap, uint32_t nqv_s, uint32_t nqe_s,
                                gs_batch **out) {
  *out = nullptr;
  gs_batch *b = new gs_batch();
  b->g = g;
  b->sms = g->num_sms;
  b->n_cap = std::max<uint32_t>(n_cap, 1);
  opts_key(b, opts);
  if (g->tuned_group) b->group = g->tuned_group;
  b->jgroup = (int)g->tuned_jgroup;
  if (g->tuned_rounds) b->refine_rounds = g->tuned_rounds == GS_ROUNDS_NONE ? 0 : g->tuned_rounds;
  if (opts && opts->max_refine_rounds) {
    b->refine_rounds = std::min<uint32_t>(opts->max_refine_rounds, kMaxRounds);
    b->fixpoint = false;
  }
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return fail(GS_ERR_CUDA, "cudaStreamCreate");
  }
  b->own_stream = true;
  b->n = 0;
  b->nq_s = b->n_cap;
  b->nqv_s = std::max<uint32_t>(nqv_s, kMaxK);
  b->nqe_s = std::max<uint32_t>(nqe_s, 1);
  // output pools sized for n_cap queries at the options' cap
  b->hq.assign(b->n_cap, DQuery{});
  b->hstatus.assign(b->n_cap, GS_OK);
  for (uint32_t i = 0; i < b->n_cap; ++i) {
    b->hq[i].k = kMaxK;
    b->hq[i].mode = opts ? opts->mode : GS_ENUMERATE;
    b->hq[i].cap = opts ? std::min<uint64_t>(opts->cap, 1u << 12) : 0;
  }
  b->n = b->n_cap;
  b->pool_hint = 1ull << 25;
  b->waves.assign(1, WaveDesc{0, b->n_cap, 0, b->nqv_s, 0, b->nqe_s});
  b->wave_k.assign(1, kMaxK);
  gs_status st = batch_alloc(b, opts);
  b->n = 0;
  b->waves.clear();
  b->wave_k.clear();
  if (st != GS_OK) {
    batch_destroy(b);
    return st;
  }
  *out = b;
  return GS_OK;
}

// Load new queries into an existing batch (same options, within its
// capacities).  Returns false when they do not fit.
bool batch_rearm(gs_batch *b, const gs_query *qs, uint32_t n, const gs_match_opts *opts) {
  if (n > b->n_cap || !opts_match(b, opts)) return false;
  for (uint32_t i = 0; i < n; ++i)
    if (qs[i].k > b->nqv_s || qs[i].m > b->nqe_s) return false;
  pack_all(b, qs, n, opts);
  for (uint32_t i = 0; i < n; ++i)
    if (b->hq[i].k > b->nqv_s || b->hq[i].m > b->nqe_s) return false;
  opts_key(b, opts);  // the same options, but a callback of this call's
  make_waves(b, b->nq_s, b->nqv_s, b->nqe_s);
  return batch_upload(b) == GS_OK;
}

void batch_destroy(gs_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto &kv : b->execs) cudaGraphExecDestroy(kv.second);
  if (b->epi_exec) cudaGraphExecDestroy(b->epi_exec);
  harvest_events(b, b->epi_evs, true);
  harvest_events(b, b->sort_evs_direct, true);
  if (b->flag) cudaFreeHost(b->flag);
  b->anchor = nullptr;
  if (b->own_anchor) cudaEventDestroy(b->own_anchor);
  for (auto &kv : b->graph_evs) harvest_events(b, kv.second, true);
  harvest_events(b, b->evs, true);
  for (void *p : b->allocs) cudaFree(p);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Replace one device pool by a larger one (contents are not kept).
template <typename T>
static gs_status regrow(gs_batch *b, T **p, uint64_t count) {
  void *old = *p;
  void *q = nullptr;
  cudaError_t e = gs::dev_malloc(&q, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GS_ERR_OOM;  // keep the old pool; overflowing queries keep taking the fallback path
  }
  cudaFree(old);
  for (auto &a : b->allocs)
    if (a == old) a = q;
  *p = static_cast<T *>(q);
  return GS_OK;
}

// After a run: enlarge every pool the run asked more of than it had, so the
// next run of a similar load stays on the device (this run's overflowing
// queries are finished on the fallback path as usual).  Graphs are captured
// again because pool pointers are kernel parameters.
gs_status grow_pools(gs_batch *b) {
  if (b->big) return GS_OK;
  uint64_t hw[HW_N];
  GS_CUDA(cudaMemcpy(hw, b->W.ctrl->hw, sizeof(hw), cudaMemcpyDeviceToHost));
  Wave &W = b->W;
  auto want = [](uint64_t need) { return need + need / 4 + 1024; };
  const uint64_t kMaxEntries = 1ull << 31;
  bool changed = false;
  auto grow32 = [&](uint32_t **p, uint64_t *cap, uint64_t need) {
    if (need <= *cap || need > kMaxEntries) return;
    const uint64_t n = want(need);
    if (regrow(b, p, n) == GS_OK) { *cap = n; changed = true; }
  };
  auto grow_owned = [&](uint32_t **p, uint32_t **owner, uint64_t *cap, uint64_t need) {
    if (need <= *cap || need > kMaxEntries) return;
    const uint64_t n = want(need);
    if (regrow(b, p, n) == GS_OK && regrow(b, owner, n) == GS_OK) { *cap = n; changed = true; }
  };
  grow_owned(&W.tlist, &W.tlist_q, &W.tlist_cap, hw[HW_TLIST]);
  grow_owned(&W.alist, &W.alist_q, &W.alist_cap, hw[HW_ALIST]);
  grow32(&W.flist, &W.flist_cap, hw[HW_FLIST]);
  grow32(&W.ec_vals, &W.ec_vals_cap, hw[HW_EC_VALS]);
  if (hw[HW_EC_ITEMS] > W.ec_items_cap && hw[HW_EC_ITEMS] <= kMaxEntries) {
    const uint64_t n = want(hw[HW_EC_ITEMS]);
    if (regrow(b, &W.ec_cnt, n) == GS_OK && regrow(b, &W.ec_off, n + 1) == GS_OK) { W.ec_items_cap = n; changed = true; }
  }
  const uint64_t need_words = std::max(hw[HW_LVL_WORDS], W.lvl_words), need_rows = std::max(hw[HW_ROWS], W.row_cap);
  if ((need_words > W.lvl_words || need_rows > W.row_cap) && need_words <= kMaxEntries && need_rows <= kMaxEntries) {
    const uint64_t nw = std::max(want(need_words), want(need_rows));  // rows of width 1 can fill a buffer
    if (regrow(b, &W.lvl[0], nw) == GS_OK && regrow(b, &W.lvl[1], nw) == GS_OK && regrow(b, &W.row_cnt, nw) == GS_OK &&
        regrow(b, &W.row_scan, nw + 1) == GS_OK) {
      W.lvl_words = W.row_cap = nw;
      changed = true;
    }
  }
  if (hw[HW_OUT_ROWS] > W.out_rows_cap && hw[HW_OUT_ROWS] <= kMaxEntries) {
    const uint64_t n = want(hw[HW_OUT_ROWS]);
    bool ok = regrow(b, &W.out_q, n) == GS_OK;
    for (int i = 0; i < 2 && ok; ++i) ok = regrow(b, &W.skey[i], n) == GS_OK && regrow(b, &W.sval[i], n) == GS_OK;
    ok = ok && regrow(b, &W.bkt_id, n) == GS_OK;
    ok = ok && regrow(b, &W.msplit, kBktPerTile * (n / kTileRows + W.nq + 1)) == GS_OK;
    ok = ok && regrow(b, &W.bspl_key, kBktPerTile * (n / kTileRows + W.nq + 1)) == GS_OK;
    ok = ok && regrow(b, &W.bspl_key2, kBktPerTile * (n / kTileRows + W.nq + 1)) == GS_OK;
    ok = ok && regrow(b, &W.bspl_row, kBktPerTile * (n / kTileRows + W.nq + 1)) == GS_OK;
    ok = ok && regrow(b, &W.ptcount, kBktPerTile * (n / kTileRows + W.nq + 1)) == GS_OK;
    ok = ok && regrow(b, &W.ptscan, kBktPerTile * (n / kTileRows + W.nq + 1) + 1) == GS_OK;
    if (ok) { W.out_rows_cap = n; changed = true; }
  }
  if (hw[HW_OUT_WORDS] > W.out_words && hw[HW_OUT_WORDS] <= kMaxEntries) {
    const uint64_t n = want(hw[HW_OUT_WORDS]);
    if (regrow(b, &W.out, n) == GS_OK && regrow(b, &W.out_final, n) == GS_OK) { W.out_words = n; changed = true; }
  }
  if (hw[HW_STORE] > W.bo.store_cap && hw[HW_STORE] <= kMaxEntries) {
    const uint64_t n = want(hw[HW_STORE]);
    if (regrow(b, &W.bo.store, n) == GS_OK) { W.bo.store_cap = n; changed = true; }
  }
  if (changed) {
    const uint64_t cps = W.G.nchunks;  // chunks per set: one candidate count per chunk
    uint64_t tmpw = scan_tmp_words(std::max<uint64_t>(
        {(uint64_t)W.nqv * cps, (uint64_t)W.nqe, W.ec_items_cap, W.row_cap, kBktPerTile * (W.out_rows_cap / kTileRows + W.nq + 1)}));
    if (regrow(b, &b->scan_tmp, tmpw) == GS_OK) {
      b->scan_tmp_words = tmpw;
      GS_CUDA(cudaMemsetAsync(b->scan_tmp, 0, sizeof(uint64_t) * tmpw, b->stream));
    }
    ::drop_graphs(b);
    b->regrows++;
  }
  return GS_OK;
}

void rows_from_pool(gs_batch *b, size_t words);

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
  uint32_t scan_err = 0;
  GS_CUDA(cudaMemcpyAsync(&top, &b->W.ctrl->store_top, 8, cudaMemcpyDeviceToHost, b->stream));
  GS_CUDA(cudaMemcpyAsync(&scan_err, scan_error_word(b->scan_tmp), 4, cudaMemcpyDeviceToHost, b->stream));
  GS_CUDA(cudaStreamSynchronize(b->stream));
  if (scan_err) {
    // the scans stayed exact (a wait that gives up sums its inputs directly),
    // but a bounded device wait ran out: report it and clear the record so
    // that later runs on this batch start clean
    GS_CUDA(cudaMemsetAsync(b->scan_tmp, 0, 4, b->stream));
    GS_CUDA(cudaStreamSynchronize(b->stream));
    return fail(GS_ERR_TIMEOUT, "a prefix scan's look-back wait reached its bound");
  }
  rows_from_pool(b, top);
  b->rows.resize(top);
  b->d2h_bytes += 36ull * n + 8 + 4ull * top;
  if (top) {
    GS_CUDA(cudaMemcpyAsync(b->rows.data(), b->W.bo.store, 4ull * top, cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaStreamSynchronize(b->stream));
  }
  gs_status gst = grow_pools(b);
  if (gst != GS_OK) return gst;
  b->fb_rows.assign(n, {});
  b->fb_done.assign(n, 0);
  b->fb_more.assign(n, 0);
  b->fallbacks = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (b->hstatus[i] != GS_OK) continue;
    // GS_CHUNKED: every query with embeddings streams them on the chunked
    // path; otherwise only the queries the device pools could not finish
    const bool stream = b->on_chunk && b->status[i] != QS_EMPTY && !(b->status[i] == QS_OK && b->count[i] == 0);
    if (stream || b->status[i] == QS_OVERFLOW || b->status[i] == QS_TOPCAP) {
      gs_status st = fallback_query(b, i);
      if (st != GS_OK) return st;
      b->fallbacks += stream ? 0 : 1;
    }
  }
  b->finished = true;
  return GS_OK;
}

gs_status batch_fetch(gs_batch *b, gs_result *outs) { return batch_fetch_views(b, outs, nullptr); }

// Results of a finished run; with `store` (the buffer that holds the run's
// rows as batch_finish copied them) the results' rows point into it
// (shared = 1) instead of being copied.
gs_status batch_fetch_views(gs_batch *b, gs_result *outs, uint32_t *store) {
  if (!b->finished) return fail(GS_ERR_INVALID, "gs_batch_fetch: call gs_batch_finish first");
  for (uint32_t i = 0; i < b->n; ++i) {
    gs_result &r = outs[i];
    memset(&r, 0, sizeof(r));
    r.k = b->hq[i].k;
    const bool proj = b->hq[i].proj != 0;
    if (b->hstatus[i] != GS_OK) {
      r.status = b->hstatus[i];
      continue;
    }
    const uint32_t st = b->status[i];
    r.count = b->count[i];
    r.fingerprint = b->fp[i];
    const uint64_t cap = b->hq[i].mode == GS_COUNT_ONLY ? 0 : b->hq[i].cap;
    r.truncated = !b->on_chunk && r.count > cap ? 1 : 0;  // GS_CHUNKED delivered every row
    if (proj) {  // rows of the projected vertices; truncated when distinct tuples exceed cap
      r.k = b->hq[i].kp;
      if (cap) r.truncated = 0;
    }
    if (b->fb_done[i]) {
      if (proj && cap) r.truncated = b->fb_more[i];
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
      r.num_rows = b->nrows[i] & ~kRowsMore;
      if (proj && cap && (b->nrows[i] & kRowsMore)) r.truncated = 1;
      if (r.num_rows && store) {
        r.rows = store + b->word_off[i];
        r.shared = 1;
      } else if (r.num_rows) {
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
extern "C" gs_status gs_memcpy_d2h(void *dst, const void *src, uint64_t bytes) {
  if (bytes && (!dst || !src)) return fail(GS_ERR_INVALID, "gs_memcpy_d2h: null pointer");
  GS_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
  return GS_OK;
}

extern "C" gs_status gs_batch_join_sizes(gs_batch *b, uint64_t *words_total, uint64_t *words_peak) {
  if (!b || !words_total || !words_peak) return fail(GS_ERR_INVALID, "gs_batch_join_sizes: null argument");
  if (!b->finished) return fail(GS_ERR_INVALID, "gs_batch_join_sizes: call gs_batch_finish first");
  GS_CUDA(cudaSetDevice(b->g->device));
  if (b->n) {
    GS_CUDA(cudaMemcpyAsync(words_total, b->W.bo.inter, 8ull * b->n, cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaMemcpyAsync(words_peak, b->W.bo.peak, 8ull * b->n, cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA(cudaStreamSynchronize(b->stream));
  }
  return GS_OK;
}

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

extern "C" gs_status gs_batch_run_all(gs_batch **bs, uint32_t nb, void *cuda_stream) {
  if (!bs || nb == 0) return fail(GS_ERR_INVALID, "gs_batch_run_all: no batches");
  for (uint32_t i = 0; i < nb; ++i) {
    if (!bs[i]) return fail(GS_ERR_INVALID, "gs_batch_run_all: null batch");
    for (uint32_t j = 0; j < i; ++j)
      if (bs[j] == bs[i] || bs[j]->stream == bs[i]->stream)
        return fail(GS_ERR_INVALID, "gs_batch_run_all: the batches need streams of their own");
  }
  return run_batches(bs, nb, static_cast<cudaStream_t>(cuda_stream));
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

// Forget captured graphs (their launch parameters changed).
static void drop_graphs(gs_batch *b) {
  for (auto &kv : b->execs) cudaGraphExecDestroy(kv.second);
  if (b->epi_exec) cudaGraphExecDestroy(b->epi_exec);
  b->execs.clear();
  b->epi_exec = nullptr;
  for (auto &kv : b->graph_evs) harvest_events(b, kv.second, true);
  harvest_events(b, b->epi_evs, true);
  b->graph_evs.clear();
}

extern "C" gs_status gs_batch_set(gs_batch *b, int use_graph, int group, uint32_t refine_rounds) {
  if (!b) return fail(GS_ERR_INVALID, "gs_batch_set: null batch");
  if (group != 4 && group != 8 && group != 16 && group != 32) return fail(GS_ERR_INVALID, "group must be 4, 8, 16 or 32");
  drop_graphs(b);
  b->use_graph = use_graph != 0;
  b->group = group;
  b->jgroup = 0;
  if (refine_rounds == GS_ROUNDS_NONE) {
    b->refine_rounds = 0;
    b->fixpoint = false;
  } else if (refine_rounds) {
    b->refine_rounds = std::min<uint32_t>(refine_rounds, kMaxRounds);
    b->fixpoint = false;
  } else {
    b->refine_rounds = 8;
    b->fixpoint = true;
  }
  return GS_OK;
}

extern "C" gs_status gs_batch_set_sort(gs_batch *b, uint32_t flags) {
  if (!b) return fail(GS_ERR_INVALID, "gs_batch_set_sort: null batch");
  if (flags & ~GS_SORT_MERGE_ONLY) return fail(GS_ERR_INVALID, "gs_batch_set_sort: unknown flags");
  b->W.merge_only = (flags & GS_SORT_MERGE_ONLY) ? 1u : 0u;
  return GS_OK;
}

extern "C" gs_status gs_batch_set_wait(gs_batch *b, uint32_t max_polls, uint32_t flags) {
  if (!b) return fail(GS_ERR_INVALID, "gs_batch_set_wait: null batch");
  if (flags & ~GS_WAIT_WITHHOLD_FIRST_TILE) return fail(GS_ERR_INVALID, "gs_batch_set_wait: unknown flags");
  return scan_set_wait(b->scan_tmp, max_polls, flags & GS_WAIT_WITHHOLD_FIRST_TILE, b->stream);
}

extern "C" void gs_debug_fail_alloc(int64_t after) { debug_fail_alloc(after); }

namespace gs {

// Batches kept per graph so that repeated gs_match / gs_match_batch calls
// reuse their device pools and captured graphs.
struct MatchCache {
  std::mutex mu;
  std::vector<gs_batch *> batches;
  uint64_t h2d = 0, d2h = 0;
};

static MatchCache *cache_of(gs_graph *g) {
  static std::mutex init_mu;
  std::lock_guard<std::mutex> lk(init_mu);
  if (!g->cache) g->cache = new MatchCache();
  return static_cast<MatchCache *>(g->cache);
}

// A batch of the cache re-armed with the queries, or a new one (the oldest
// of four is dropped).
static gs_status cached_batch(gs_graph *g, MatchCache *c, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                              gs_batch **out, gs_batch *const *taken = nullptr, uint32_t ntaken = 0) {
  auto is_taken = [&](const gs_batch *x) {
    for (uint32_t i = 0; i < ntaken; ++i)
      if (taken[i] == x) return true;
    return false;
  };
  for (gs_batch *x : c->batches)
    if (!is_taken(x) && batch_rearm(x, qs, n, opts)) {
      *out = x;
      return GS_OK;
    }
  gs_batch *b = nullptr;
  gs_status st = batch_create(g, qs, n, opts, 0, &b);
  if (st != GS_OK) return st;
  for (size_t i = 0; c->batches.size() >= 8 && i < c->batches.size();) {  // drop the oldest batch not in use
    if (is_taken(c->batches[i])) { ++i; continue; }
    batch_destroy(c->batches[i]);
    c->batches.erase(c->batches.begin() + i);
  }
  c->batches.push_back(b);
  *out = b;
  return GS_OK;
}

void release_cache(gs_graph *g) {
  if (!g->cache) return;
  MatchCache *c = static_cast<MatchCache *>(g->cache);
  for (gs_batch *b : c->batches) batch_destroy(b);
  delete c;
  g->cache = nullptr;
}

}  // namespace gs

extern "C" gs_status gs_match_batch(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                                    gs_result *outs) {
  if (!g || !outs || (n && !qs)) return fail(GS_ERR_INVALID, "gs_match_batch: null argument");
  if (n == 0) return GS_OK;
  GS_CUDA(cudaSetDevice(g->device));
  MatchCache *c = cache_of(g);
  std::lock_guard<std::mutex> lk(c->mu);
  gs_batch *b = nullptr;
  gs_status cst = cached_batch(g, c, qs, n, opts, &b);
  if (cst != GS_OK) return cst;
  const uint64_t d0 = b->d2h_bytes;
  c->h2d += b->last_upload_bytes;
  gs_status st = run_waves(b);
  b->ran = st == GS_OK;
  if (st == GS_OK) st = batch_finish(b);
  if (st == GS_OK) st = batch_fetch(b, outs);
  for (uint32_t i = 0; i < n && st == GS_OK; ++i) b->d2h_bytes += 4ull * outs[i].num_rows * outs[i].k;
  c->d2h += b->d2h_bytes - d0;
  return st;
}

extern "C" gs_status gs_graph_io_bytes(gs_graph *g, uint64_t *h2d, uint64_t *d2h) {
  if (!g) return fail(GS_ERR_INVALID, "null graph");
  MatchCache *c = cache_of(g);
  std::lock_guard<std::mutex> lk(c->mu);
  if (h2d) *h2d = c->h2d;
  if (d2h) *d2h = c->d2h;
  return GS_OK;
}

extern "C" gs_status gs_batch_counters(gs_batch *b, uint64_t *kernel_launches, uint64_t *h2d, uint64_t *d2h,
                                       uint64_t *fallback_queries) {
  if (!b) return fail(GS_ERR_INVALID, "null batch");
  if (fallback_queries) *fallback_queries = b->fallbacks;
  if (kernel_launches) *kernel_launches = b->kernel_launches;
  if (h2d) *h2d = b->h2d_bytes;
  if (d2h) *d2h = b->d2h_bytes;
  return GS_OK;
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
  if (!r->shared) free(r->rows);
  r->rows = nullptr;
  r->num_rows = 0;
}

// Page-locked result buffers handed out by gs_match_batch_shared, one per
// batch the call ran: a released buffer goes back to a small process-wide
// pool, from which a batch takes its next result buffer, so a steady stream
// of calls allocates no page-locked memory.
struct RowsBuf {
  uint32_t *p = nullptr;
  size_t cap = 0;      // words
  uint64_t words = 0;  // words written by the call
};
struct gs_rows {
  std::vector<RowsBuf> bufs;
};

namespace gs {
std::mutex g_rows_mu;
std::vector<RowsBuf> g_rows_pool;
constexpr size_t kRowsPoolMax = 16;

// Hand a finished batch's result buffer over to `blk`; the batch takes a
// pooled one when its next run has rows to copy out.
void take_rows(gs_batch *b, gs_rows *blk) {
  blk->bufs.push_back(RowsBuf{b->rows.p, b->rows.cap, b->rows.n});
  b->rows.p = nullptr;
  b->rows.cap = 0;
  b->rows.n = 0;
}

// A batch without a result buffer takes the smallest pooled one that holds
// `words`, else the largest (which then grows).
void rows_from_pool(gs_batch *b, size_t words) {
  if (b->rows.p || !words) return;
  std::lock_guard<std::mutex> pl(g_rows_mu);
  if (g_rows_pool.empty()) return;
  size_t best = 0;
  for (size_t i = 1; i < g_rows_pool.size(); ++i) {
    const size_t c = g_rows_pool[i].cap, bc = g_rows_pool[best].cap;
    if (bc >= words ? (c >= words && c < bc) : c > bc) best = i;
  }
  b->rows.p = g_rows_pool[best].p;
  b->rows.cap = g_rows_pool[best].cap;
  b->rows.n = 0;
  g_rows_pool.erase(g_rows_pool.begin() + best);
}
}  // namespace gs

extern "C" uint32_t gs_rows_count(const gs_rows *block) { return block ? (uint32_t)block->bufs.size() : 0; }
extern "C" const uint32_t *gs_rows_base(const gs_rows *block, uint32_t i) {
  return block && i < block->bufs.size() ? block->bufs[i].p : nullptr;
}
extern "C" uint64_t gs_rows_words(const gs_rows *block, uint32_t i) {
  return block && i < block->bufs.size() ? block->bufs[i].words : 0;
}

extern "C" void gs_rows_release(gs_rows *block) {
  if (!block) return;
  {
    std::lock_guard<std::mutex> lk(g_rows_mu);
    for (RowsBuf &r : block->bufs) {
      if (!r.p) continue;
      if (g_rows_pool.size() < kRowsPoolMax) {
        r.words = 0;
        g_rows_pool.push_back(r);
      } else {
        cudaFreeHost(r.p);
      }
    }
  }
  delete block;
}

// Batches of at least this many queries are matched as kSplitParts
// sub-batches running at once on their own streams (each sub-batch's steps
// with few work items left run beside the others' bulk work).
constexpr uint32_t kSplitMin = 4096, kSplitParts = 4;

extern "C" gs_status gs_match_batch_shared(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                                           gs_result *outs, gs_rows **block) {
  if (!block) return fail(GS_ERR_INVALID, "gs_match_batch_shared: null block");
  *block = nullptr;
  if (!g || !outs || (n && !qs)) return fail(GS_ERR_INVALID, "gs_match_batch_shared: null argument");
  if (n == 0) return GS_OK;
  GS_CUDA(cudaSetDevice(g->device));
  MatchCache *c = cache_of(g);
  std::lock_guard<std::mutex> lk(c->mu);
  const bool own_streams = !(opts && opts->cuda_stream);
  const uint32_t parts = n >= kSplitMin && own_streams ? kSplitParts : 1;
  std::vector<gs_batch *> bs(parts, nullptr);
  std::vector<uint32_t> lo(parts + 1);
  for (uint32_t p = 0; p <= parts; ++p) lo[p] = (uint32_t)((uint64_t)n * p / parts);
  gs_status st = GS_OK;
  for (uint32_t p = 0; p < parts && st == GS_OK; ++p)
    st = cached_batch(g, c, qs + lo[p], lo[p + 1] - lo[p], opts, &bs[p], bs.data(), p);
  if (st != GS_OK) return st;
  uint64_t d0 = 0;
  for (gs_batch *b : bs) {
    d0 += b->d2h_bytes;
    c->h2d += b->last_upload_bytes;
  }
  if (parts == 1) {
    st = run_waves(bs[0]);
    bs[0]->ran = st == GS_OK;
  } else {
    st = run_batches(bs.data(), parts, nullptr);
  }
  for (uint32_t p = 0; p < parts && st == GS_OK; ++p) st = batch_finish(bs[p]);
  if (st != GS_OK) return st;
  // the results point into the batches' result buffers, which the call hands over
  gs_rows *blk = new gs_rows();
  for (uint32_t p = 0; p < parts && st == GS_OK; ++p) {
    take_rows(bs[p], blk);
    st = batch_fetch_views(bs[p], outs + lo[p], blk->bufs.back().p);
  }
  uint64_t d1 = 0;
  for (uint32_t i = 0; i < n && st == GS_OK; ++i) bs[0]->d2h_bytes += 4ull * outs[i].num_rows * outs[i].k;
  for (gs_batch *b : bs) d1 += b->d2h_bytes;
  c->d2h += d1 - d0;
  bool any = false;
  for (uint32_t i = 0; i < n && st == GS_OK; ++i) any = any || outs[i].shared;
  if (st != GS_OK || !any) {
    gs_rows_release(blk);
    return st;
  }
  *block = blk;
  return GS_OK;
}

extern "C" gs_status gs_results_copy_rows(const gs_result *r, uint32_t n, uint32_t *dst) {
  if (n && (!r || !dst)) return fail(GS_ERR_INVALID, "gs_results_copy_rows: null pointer");
  uint64_t at = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const uint64_t words = r[i].num_rows * r[i].k;
    if (words && r[i].rows) memcpy(dst + at, r[i].rows, 4 * words);
    at += words;
  }
  return GS_OK;
}

extern "C" void gs_results_free(gs_result *r, uint32_t n) {
  if (!r) return;
  for (uint32_t i = 0; i < n; ++i) gs_result_free(&r[i]);
}

extern "C" gs_status gs_stats_enable(gs_batch *b, int on) {
  if (!b) return fail(GS_ERR_INVALID, "null batch");
  if ((on != 0) != b->stats_on) drop_graphs(b);
  b->stats_on = on != 0;
  return GS_OK;
}

static const char *kKindNames[GS_NUM_KERNEL_KINDS] = {
    "plan", "filter", "compact", "explore", "refine", "ec_count", "ec_write", "clear",
    "join_count", "join_write", "scan", "sort", "gather", "other", "compact_all", "sort_large"};

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
  b->spans.clear();
  return GS_OK;
}

extern "C" gs_status gs_stats_busy(gs_batch *const *bs, uint32_t nb, double *busy_ms) {
  if (!busy_ms || (nb && !bs)) return fail(GS_ERR_INVALID, "gs_stats_busy: null argument");
  std::vector<gs_batch::Span> all;
  for (uint32_t i = 0; i < nb; ++i) {
    if (!bs[i]) return fail(GS_ERR_INVALID, "gs_stats_busy: null batch");
    all.insert(all.end(), bs[i]->spans.begin(), bs[i]->spans.end());
  }
  for (int k = 0; k < GS_NUM_KERNEL_KINDS; ++k) busy_ms[k] = 0;
  std::sort(all.begin(), all.end(), [](const gs_batch::Span &x, const gs_batch::Span &y) {
    if (x.run != y.run) return x.run < y.run;
    if (x.kind != y.kind) return x.kind < y.kind;
    return x.t0 < y.t0;
  });
  // per run and kind, the length of the union of the launch intervals
  for (size_t i = 0; i < all.size();) {
    size_t j = i;
    double lo = all[i].t0, hi = all[i].t1, sum = 0;
    for (; j < all.size() && all[j].run == all[i].run && all[j].kind == all[i].kind; ++j) {
      if (all[j].t0 > hi) {
        sum += hi - lo;
        lo = all[j].t0;
      }
      hi = std::max(hi, (double)all[j].t1);
    }
    busy_ms[all[i].kind] += sum + (hi - lo);
    i = j;
  }
  return GS_OK;
}
