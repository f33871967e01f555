// Inspection of one query's candidate sets and candidate-edge tables, for
// per-kernel parity checks.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gs_host.h"

using namespace gs;

namespace {

// A one-query batch run step by step (no graph capture) with refinement
// looped to its fixpoint.
gs_status make_single(gs_graph *g, const gs_query *q, gs_batch **out) {
  gs_match_opts o;
  memset(&o, 0, sizeof(o));
  o.mode = GS_COUNT_ONLY;
  gs_status st = batch_create(g, q, 1, &o, 1, out);
  if (st != GS_OK) return st;
  if ((*out)->hstatus[0] != GS_OK) {
    gs_status qs = (gs_status)(*out)->hstatus[0];
    batch_destroy(*out);
    *out = nullptr;
    return fail(qs, "invalid query");
  }
  (*out)->use_graph = false;
  (*out)->fixpoint = true;
  return GS_OK;
}

template <typename T>
gs_status d2h(T *dst, const T *src, uint64_t n, cudaStream_t s) {
  if (!n) return GS_OK;
  GS_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
  return GS_OK;
}

}  // namespace

extern "C" gs_status gs_inspect_candidates(gs_graph *g, const gs_query *q, uint32_t stage, uint64_t *off, uint32_t *ids,
                                           uint64_t cap_ids, uint64_t *n_ids) {
  if (!g || !q || !off || !n_ids) return fail(GS_ERR_INVALID, "gs_inspect_candidates: null argument");
  if (stage != GS_STAGE_FILTER && stage != GS_STAGE_FIXPOINT) return fail(GS_ERR_INVALID, "unknown stage");
  GS_CUDA(cudaSetDevice(g->device));
  gs_batch *b = nullptr;
  gs_status st = make_single(g, q, &b);
  if (st != GS_OK) return st;
  const uint32_t k = b->hq[0].k;
  const cudaStream_t s = b->stream;
  const uint64_t cps = g->d.nchunks;
  std::vector<std::vector<uint32_t>> sets(k);
  if (stage == GS_STAGE_FILTER) {
    for (uint32_t u = 0; u < k && st == GS_OK; ++u) {
      b->hq[0].force_root = (uint8_t)u;
      GS_CUDA(cudaMemcpyAsync(b->all_dq, b->hq.data(), sizeof(DQuery), cudaMemcpyHostToDevice, s));
      GS_CUDA(cudaMemsetAsync(&b->W.ctrl->wave, 0, sizeof(uint32_t), s));
      launch_prologue(b->W, s, b->sms);
      launch_plan(b->W, b->type_count, s, b->sms);
      scan_u32(b->W.fcnt, b->W.fscan, &b->W.ctrl->len[8], b->W.nq, b->scan_tmp, s, b->sms);
      Wave wc = b->W;
      wc.c0_only = 1;  // the filter stage as Definition 3.3 defines it
      launch_filter(wc, s, b->sms);
      launch_compact_count(b->W, 0, 0, s, b->sms);
      scan_u32(b->W.ccount, b->W.cscan, &b->W.ctrl->len[0], (uint64_t)b->W.nq * cps, b->scan_tmp, s, b->sms);
      launch_compact_write(b->W, 0, 0, b->W.cscan, b->W.tlist, b->W.tlist_q, b->W.tlist_cap, HW_TLIST, s, b->sms);
      uint64_t total = 0;
      GS_CUDA(cudaMemcpyAsync(&total, b->W.cscan + (uint64_t)b->W.nq * cps, 8, cudaMemcpyDeviceToHost, s));
      GS_CUDA(cudaStreamSynchronize(s));
      sets[u].resize(total);
      st = d2h(sets[u].data(), b->W.tlist, total, s);
      launch_clear(b->W, s, b->sms);
      GS_CUDA(cudaStreamSynchronize(s));
    }
  } else {
    GS_CUDA(cudaMemsetAsync(&b->W.ctrl->wave, 0, sizeof(uint32_t), s));
    enqueue_wave(b, (int)k, false, &b->evs);
    st = refine_to_fixpoint(b);
    if (st == GS_OK) {
      enqueue_wave_tail(b, (int)k, false, &b->evs, 1);
      std::vector<uint64_t> lo(k);
      std::vector<uint32_t> ln(k);
      st = d2h(lo.data(), b->W.flist_off, k, s);
      if (st == GS_OK) st = d2h(ln.data(), b->W.flist_len, k, s);
      GS_CUDA(cudaStreamSynchronize(s));
      uint32_t qst = 0;
      GS_CUDA(cudaMemcpy(&qst, &b->W.dq[0].status, 4, cudaMemcpyDeviceToHost));
      if (qst == QS_OVERFLOW) st = fail(GS_ERR_OOM, "candidate lists overflowed");
      for (uint32_t u = 0; u < k && st == GS_OK; ++u) {
        sets[u].resize(ln[u]);
        st = d2h(sets[u].data(), b->W.flist + lo[u], ln[u], s);
      }
      GS_CUDA(cudaStreamSynchronize(s));
    }
  }
  if (st == GS_OK) {
    uint64_t tot = 0;
    for (uint32_t u = 0; u < k; ++u) {
      off[u] = tot;
      tot += sets[u].size();
    }
    off[k] = tot;
    *n_ids = tot;
    if (ids) {
      if (tot > cap_ids) {
        st = fail(GS_ERR_INVALID, "ids buffer too small");
      } else {
        for (uint32_t u = 0; u < k; ++u)
          if (!sets[u].empty()) memcpy(ids + off[u], sets[u].data(), 4 * sets[u].size());
      }
    }
  }
  batch_destroy(b);
  return st;
}

extern "C" gs_status gs_inspect_edge_table(gs_graph *g, const gs_query *q, uint32_t e, uint32_t from_src, uint32_t *keys,
                                           uint64_t *off, uint32_t *vals, uint64_t cap_keys, uint64_t cap_vals,
                                           uint64_t *nkeys, uint64_t *nvals) {
  if (!g || !q || !nkeys || !nvals) return fail(GS_ERR_INVALID, "gs_inspect_edge_table: null argument");
  if (e >= q->m) return fail(GS_ERR_INVALID, "edge index out of range");
  GS_CUDA(cudaSetDevice(g->device));
  gs_batch *b = nullptr;
  gs_status st = make_single(g, q, &b);
  if (st != GS_OK) return st;
  const DQuery &d = b->hq[0];
  const uint32_t rel = q->erel[e] == kAny ? kRelAny8 : q->erel[e];
  uint32_t j = 0;
  for (; j < d.m; ++j)
    if (d.esrc[j] == q->esrc[e] && d.edst[j] == q->edst[e] && d.erel[j] == rel) break;
  const uint32_t x = from_src ? d.esrc[j] : d.edst[j];
  b->hq[0].force_from_src = from_src ? 1 : 0;
  const cudaStream_t s = b->stream;
  GS_CUDA(cudaMemcpyAsync(b->all_dq, b->hq.data(), sizeof(DQuery), cudaMemcpyHostToDevice, s));
  GS_CUDA(cudaMemsetAsync(&b->W.ctrl->wave, 0, sizeof(uint32_t), s));
  enqueue_wave(b, (int)d.k, false, &b->evs);
  st = refine_to_fixpoint(b);
  if (st == GS_OK) {
    enqueue_wave_tail(b, (int)d.k, false, &b->evs, 2);
    uint64_t kb[2], lo = 0;
    uint32_t ln = 0, qst = 0;
    st = d2h(kb, b->W.ec_key_base + j, 2, s);
    if (st == GS_OK) st = d2h(&lo, b->W.flist_off + x, 1, s);
    if (st == GS_OK) st = d2h(&ln, b->W.flist_len + x, 1, s);
    GS_CUDA(cudaStreamSynchronize(s));
    GS_CUDA(cudaMemcpy(&qst, &b->W.dq[0].status, 4, cudaMemcpyDeviceToHost));
    if (st == GS_OK && qst == QS_OVERFLOW) st = fail(GS_ERR_OOM, "edge tables overflowed");
    const uint64_t nk = kb[1] - kb[0];  // 0 when some candidate set is empty
    std::vector<uint64_t> o(nk + 1, 0);
    if (st == GS_OK && nk) st = d2h(o.data(), b->W.ec_off + kb[0], nk + 1, s);
    GS_CUDA(cudaStreamSynchronize(s));
    const uint64_t base = nk ? o[0] : 0;
    const uint64_t nv = nk ? o[nk] - base : 0;
    *nkeys = nk;
    *nvals = nv;
    if (st == GS_OK && keys) {
      if (nk > cap_keys || nv > cap_vals || !off || !vals) {
        st = fail(GS_ERR_INVALID, "output buffers too small");
      } else {
        (void)ln;
        st = d2h(keys, b->W.flist + lo, nk, s);
        if (st == GS_OK) st = d2h(vals, b->W.ec_vals + base, nv, s);
        GS_CUDA(cudaStreamSynchronize(s));
        for (uint64_t i = 0; i <= nk; ++i) off[i] = o[i] - base;
      }
    }
  }
  batch_destroy(b);
  return st;
}
