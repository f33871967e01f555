// Serving: a request loop over a device-resident graph with continuous
// batching.  Requests queue on submit; a worker thread admits them into
// micro-batches whenever a slot is free and the working-set budget allows,
// so requests that arrive while others are on the GPU join the next
// micro-batch instead of waiting for the whole queue to drain.  Each slot has
// its own stream, so several micro-batches overlap on the device.  Results
// are kept per ticket until polled.
//
// Admission estimate per query (from candidate-set sizes): a bound vertex has
// one candidate; a free vertex has the expected size of its Definition 3.3
// set, from the graph's per-type signature statistics (the vertices of its
// type, or of any type, meeting each of its degree needs; exact for one
// need, a product of fractions for several); each candidate costs its list
// entry, its candidate-edge table entries and a bitmap slot share.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "gs_host.h"

using namespace gs;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  uint32_t k = 0, m = 0;
  std::vector<uint32_t> vtype, vbind, esrc, edst, erel;
  gs_match_opts opts{};
  Clock::time_point t_submit;
  uint64_t est = 0;
  gs_query view() const {
    return gs_query{k, m, vtype.data(), vbind.data(), esrc.data(), edst.data(), erel.data()};
  }
};

struct Done {
  gs_result r;
  double latency_s;
};

// A slot runs one micro-batch at a time in two halves on its own stream
// (phase 1: the pipeline graph and the copy of the large-output flags;
// phase 2: the large-output sort if needed and the epilogue), each ended by
// an event the worker polls, so that no slot blocks the others.
struct Slot {
  gs_batch *b = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  int phase = 0;
  std::vector<Req> reqs;
  uint64_t est = 0;
  gs_match_opts opts{};
};

bool same_opts(const gs_match_opts &a, const gs_match_opts &b) {
  return a.cap == b.cap && a.mode == b.mode && a.max_refine_rounds == b.max_refine_rounds &&
         a.chunk_bytes == b.chunk_bytes && a.project == b.project && a.refine == b.refine;
}

}  // namespace

struct gs_server {
  gs_graph *g = nullptr;
  gs_serve_opts o{};
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<Req> pending;
  std::unordered_map<uint64_t, Done> done;
  std::unordered_map<uint64_t, int> inflight;  // ticket -> slot
  std::unordered_set<uint64_t> live;           // submitted and not yet polled to completion
  uint64_t next_ticket = 1;
  uint64_t inflight_est = 0;
  std::vector<Slot> slots;
  std::thread worker;
  gs_status worker_error = GS_OK;
  std::string worker_msg;
};

namespace {

std::atomic<uint32_t> g_fail_waits{0};  // completion checks left to report a simulated CUDA error

// Completion check of a slot's event: cudaEventQuery, or a simulated failure
// armed by gs_debug_fail_serve_wait.
cudaError_t slot_query(cudaEvent_t ev) {
  uint32_t n = g_fail_waits.load(std::memory_order_relaxed);
  while (n > 0)
    if (g_fail_waits.compare_exchange_weak(n, n - 1)) return cudaErrorLaunchFailure;
  return cudaEventQuery(ev);
}

uint64_t estimate(const gs_graph *g, const DQuery &d) {
  const uint64_t slot_bytes = 4 * (((uint64_t)g->d.W0 + g->d.W1 + g->d.ipg + 31) / 32 * 32);
  const uint32_t T = g->d.T, P = 2 * g->d.R + 2;
  uint64_t est = 1 << 16;
  for (uint32_t u = 0; u < d.k; ++u) {
    double c = 1.0;
    if (d.vbind[u] == GS_UNBOUND) {
      const uint32_t t = d.vtype[u] == GS_ANY ? T : d.vtype[u];
      const double n = t == T ? (double)g->d.V : (double)g->type_count[t];
      c = n;
      for (uint32_t i = d.need_begin[u]; i < d.need_begin[u + 1] && n > 0; ++i)
        c *= (double)g->sigge_host[((uint64_t)t * P + d.need_plane[i]) * 16 + d.need_cnt[i]] / n;
    }
    const uint64_t deg = d.inc_begin[u + 1] - d.inc_begin[u];
    est += (uint64_t)(c + 1.0) * 4 * (2 + deg) + slot_bytes;
  }
  return est;
}

// Finish a slot whose micro-batch completed: results move to `done`.
void harvest(gs_server *s, Slot &sl) {
  gs_status st = batch_finish(sl.b);
  std::vector<gs_result> outs(sl.reqs.size());
  if (st == GS_OK) st = batch_fetch(sl.b, outs.data());
  const auto now = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    Done d;
    if (st == GS_OK) {
      d.r = outs[i];
    } else {
      memset(&d.r, 0, sizeof(d.r));
      d.r.status = st;
    }
    d.latency_s = std::chrono::duration<double>(now - sl.reqs[i].t_submit).count();
    s->inflight.erase(sl.reqs[i].ticket);
    s->done.emplace(sl.reqs[i].ticket, d);
  }
  s->inflight_est -= sl.est;
  sl.reqs.clear();
  sl.est = 0;
  sl.busy = false;
}

// Take the next micro-batch from the queue (FIFO, same options, within the
// budget; the head is always admitted when nothing is in flight).
std::vector<Req> admit(gs_server *s, uint64_t &est_sum) {
  std::vector<Req> take;
  est_sum = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  while (!s->pending.empty() && take.size() < s->o.max_batch) {
    Req &r = s->pending.front();
    if (!take.empty() && !same_opts(take.front().opts, r.opts)) break;
    const bool fits = s->inflight_est + est_sum + r.est <= s->o.budget_bytes;
    if (!fits && !(take.empty() && s->inflight_est == 0)) break;
    est_sum += r.est;
    take.push_back(std::move(r));
    s->pending.pop_front();
  }
  s->inflight_est += est_sum;
  return take;
}

// Start a micro-batch on a free slot.  The slot owns the requests from the
// start, so that a failure completes every one of them with the error.
gs_status launch(gs_server *s, Slot &sl, std::vector<Req> &&reqs, uint64_t est) {
  sl.reqs = std::move(reqs);
  sl.est = est;
  sl.busy = true;
  sl.phase = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &r : sl.reqs) s->inflight[r.ticket] = (int)(&sl - s->slots.data());
  }
  std::vector<gs_query> qs;
  qs.reserve(sl.reqs.size());
  for (auto &r : sl.reqs) qs.push_back(r.view());
  const gs_match_opts &o = sl.reqs.front().opts;
  if (!sl.b || !batch_rearm(sl.b, qs.data(), (uint32_t)qs.size(), &o)) {
    if (sl.b) batch_destroy(sl.b);
    sl.b = nullptr;
    gs_status st = batch_create_capacity(s->g, &o, s->o.max_batch, s->o.max_batch * 10, s->o.max_batch * 16, &sl.b);
    if (st != GS_OK) return st;
    if (!batch_rearm(sl.b, qs.data(), (uint32_t)qs.size(), &o)) return fail(GS_ERR_INVALID, "serving slot too small");
  }
  sl.opts = o;
  sl.b->ran = false;
  gs_status st = run_begin(sl.b);
  if (st != GS_OK) return st;
  GS_CUDA(cudaEventRecord(sl.ev, sl.b->stream));
  sl.phase = 1;
  return GS_OK;
}

// The pipeline half has completed (its flags are on the host): launch the tail.
gs_status launch_tail(Slot &sl) {
  gs_status st = run_end(sl.b);
  if (st != GS_OK) return st;
  sl.b->ran = true;
  GS_CUDA(cudaEventRecord(sl.ev, sl.b->stream));
  sl.phase = 2;
  return GS_OK;
}

// A slot whose micro-batch failed: wait until its stream has drained (at
// once after a real fault), drop its batch so that no later micro-batch
// reuses buffers that queued work may still touch, and complete its requests
// with the error.
void fail_slot(gs_server *s, Slot &sl, gs_status st) {
  const std::string msg = gs_last_error();
  if (sl.b) {
    cudaStreamSynchronize(sl.b->stream);
    cudaGetLastError();
    batch_destroy(sl.b);
    sl.b = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->worker_error = st;
  s->worker_msg = msg;
  for (auto &r : sl.reqs) {
    Done d;
    memset(&d.r, 0, sizeof(d.r));
    d.r.status = st;
    d.latency_s = 0;
    s->inflight.erase(r.ticket);
    s->done.emplace(r.ticket, d);
  }
  s->inflight_est -= sl.est;
  sl.reqs.clear();
  sl.busy = false;
  sl.phase = 0;
}

void worker_main(gs_server *s) {
  cudaSetDevice(s->g->device);
  for (Slot &sl : s->slots) cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
  for (;;) {
    bool worked = false;
    for (Slot &sl : s->slots) {
      if (!sl.busy) continue;
      const cudaError_t e = slot_query(sl.ev);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) {
        cudaGetLastError();
        fail_slot(s, sl, cuda_fail(e, "serving: micro-batch completion"));
        worked = true;
        continue;
      }
      if (sl.phase == 1) {
        gs_status st = launch_tail(sl);
        if (st != GS_OK) fail_slot(s, sl, st);
      } else {
        harvest(s, sl);
        sl.phase = 0;
      }
      worked = true;
    }
    for (Slot &sl : s->slots) {
      if (sl.busy) continue;
      uint64_t est = 0;
      std::vector<Req> reqs = admit(s, est);
      if (reqs.empty()) break;
      gs_status st = launch(s, sl, std::move(reqs), est);
      if (st != GS_OK) fail_slot(s, sl, st);
      worked = true;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    bool any_busy = false;
    for (Slot &sl : s->slots) any_busy |= sl.busy;
    if (s->stop && !any_busy) break;
    if (!worked) {
      if (any_busy) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      } else if (s->pending.empty()) {
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
      }
    }
  }
  for (Slot &sl : s->slots) {
    if (sl.b) batch_destroy(sl.b);
    sl.b = nullptr;
    if (sl.ev) cudaEventDestroy(sl.ev);
  }
}

}  // namespace

extern "C" gs_status gs_serve_create(gs_graph *g, const gs_serve_opts *opts, gs_server **out) {
  if (!g || !out) return fail(GS_ERR_INVALID, "gs_serve_create: null argument");
  *out = nullptr;
  gs_server *s = new gs_server();
  s->g = g;
  if (opts) s->o = *opts;
  if (!s->o.budget_bytes) s->o.budget_bytes = 40ull << 30;
  if (!s->o.slots) s->o.slots = 4;
  if (!s->o.max_batch) s->o.max_batch = 256;
  if (!s->o.queue_depth) s->o.queue_depth = 65536;
  if (s->o.slots > 64 || s->o.max_batch > 65536) {
    delete s;
    return fail(GS_ERR_INVALID, "serving options out of range");
  }
  s->slots.resize(s->o.slots);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return GS_OK;
}

extern "C" gs_status gs_serve_submit(gs_server *s, const gs_query *q, const gs_match_opts *opts, uint64_t *ticket) {
  if (!s || !q || !ticket) return fail(GS_ERR_INVALID, "gs_serve_submit: null argument");
  if (opts && opts->mode == GS_CHUNKED)
    return fail(GS_ERR_UNSUPPORTED, "GS_CHUNKED is not served (its callback would run on the serving thread)");
  // validate now so that a bad query fails at submit
  DQuery d;
  gs_status st = pack_query(s->g->d, q, opts, &d);
  if (st != GS_OK) return st;
  Req r;
  r.k = q->k;
  r.m = q->m;
  r.vtype.assign(q->vtype, q->vtype + q->k);
  r.vbind.assign(q->vbind, q->vbind + q->k);
  r.esrc.assign(q->esrc, q->esrc + q->m);
  r.edst.assign(q->edst, q->edst + q->m);
  r.erel.assign(q->erel, q->erel + q->m);
  if (opts) r.opts = *opts;
  r.opts.cuda_stream = nullptr;
  r.t_submit = Clock::now();
  r.est = estimate(s->g, d);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->pending.size() >= s->o.queue_depth) return fail(GS_ERR_BUSY, "serving queue full");
    r.ticket = s->next_ticket++;
    *ticket = r.ticket;
    s->live.insert(r.ticket);
    s->pending.push_back(std::move(r));
  }
  s->cv.notify_one();
  return GS_OK;
}

extern "C" gs_status gs_serve_poll(gs_server *s, uint64_t ticket, gs_result *out, double *latency_s) {
  if (!s || !out) return fail(GS_ERR_INVALID, "gs_serve_poll: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    if (!s->live.count(ticket)) return fail(GS_ERR_INVALID, "unknown or already collected ticket");
    return GS_ERR_NOT_READY;
  }
  *out = it->second.r;
  if (latency_s) *latency_s = it->second.latency_s;
  s->done.erase(it);
  s->live.erase(ticket);
  return GS_OK;
}

extern "C" void gs_debug_fail_serve_wait(uint32_t n) { g_fail_waits.store(n); }

extern "C" gs_status gs_serve_destroy(gs_server *s) {
  if (!s) return GS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto &kv : s->done) gs_result_free(&kv.second.r);
  delete s;
  return GS_OK;
}
