// The host-driven path for queries a batch could not finish on the device:
// partial embeddings that overflow the level budget, or more embeddings than
// `cap` (the smallest `cap` rows in lexicographic order are wanted).
//
// The join runs level by level as before (count, scan, write), but when the
// next level would not fit its buffer the current level is cut into chunks
// and each chunk is expanded depth first to the last level before the next
// chunk starts (a DFS over BFS chunks).  The last level is only counted
// (count and fingerprint accumulate in the count pass); when rows are
// wanted they are collected into a buffer of 2*cap rows that is sorted and
// cut back to cap whenever it fills.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "gs_host.h"

using namespace gs;

namespace gs {

namespace {

constexpr int kT = 256;

__global__ void k_iota_n(uint32_t *p, const uint64_t *d_n) {
  const uint64_t n = *d_n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = (uint32_t)i;
}

// key[i] = column `col` of row perm[i] (rows are k words wide)
__global__ void k_col_keys(const uint32_t *rows, uint32_t k, const uint32_t *perm, const uint64_t *d_n, uint32_t col,
                           uint32_t *key) {
  const uint64_t n = *d_n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    key[i] = rows[(uint64_t)perm[i] * k + col];
}

// out[i] = row perm[i] for i < keep, w columns taken in `order` (order[u] =
// source column of output column u).
struct ColOrder {
  uint8_t c[kMaxK];
};
__global__ void k_take_rows(const uint32_t *rows, uint32_t k, const uint32_t *perm, uint64_t keep, ColOrder order,
                            uint32_t w, uint32_t *out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < keep; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t *src = rows + (uint64_t)perm[i] * k;
    for (uint32_t u = 0; u < w; ++u) out[i * w + u] = src[order.c[u]];
  }
}

// Projection: flag[i] = 1 when row perm[i] starts a new tuple of the
// projected columns `cols` (rows sorted on them), i.e. differs from row
// perm[i-1] on one of them.
__global__ void k_proj_flags(const uint32_t *rows, uint32_t k, const uint32_t *perm, const uint64_t *d_n, ColOrder cols,
                             uint32_t ncols, uint32_t *flag) {
  const uint64_t n = *d_n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t f = 1;
    if (i > 0) {
      const uint32_t *a = rows + (uint64_t)perm[i] * k, *b = rows + (uint64_t)perm[i - 1] * k;
      f = 0;
      for (uint32_t j = 0; j < ncols; ++j) f |= a[cols.c[j]] != b[cols.c[j]];
    }
    flag[i] = f;
  }
}

// out[scan[i]] = row perm[i] (w columns in `order`) for every flagged i whose
// rank scan[i] is below keep.
__global__ void k_take_distinct(const uint32_t *rows, uint32_t k, const uint32_t *perm, const uint32_t *flag,
                                const uint64_t *scan, const uint64_t *d_n, uint64_t keep, ColOrder order, uint32_t w,
                                uint32_t *out) {
  const uint64_t n = *d_n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    if (!flag[i] || scan[i] >= keep) continue;
    const uint32_t *src = rows + (uint64_t)perm[i] * k;
    for (uint32_t u = 0; u < w; ++u) out[scan[i] * w + u] = src[order.c[u]];
  }
}

__device__ __forceinline__ uint64_t fb_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Fingerprint of one-vertex embeddings (v): the row hash folded over one id.
__global__ void k_list_fp(const uint32_t *lst, uint64_t n, unsigned long long *fp) {
  uint64_t acc = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    acc += fb_mix64((uint64_t)1 ^ ((uint64_t)lst[i] + 0x9E3779B97F4A7C15ull));
  for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(fp, (unsigned long long)acc);
}

// Chunk boundaries: bounds[j] = first row whose output starts at or after
// j*B (scan is the exclusive scan of per-row outputs, n+1 entries).
__global__ void k_chunk_bounds(const uint64_t *scan, uint64_t n, uint64_t B, uint64_t nb, uint64_t *bounds) {
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j <= nb; j += (uint64_t)gridDim.x * blockDim.x) {
    if (j == nb) { bounds[j] = n; continue; }
    const uint64_t key = j * B;
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
      uint64_t mid = (lo + hi) >> 1;
      if (scan[mid] < key) lo = mid + 1; else hi = mid;
    }
    bounds[j] = lo;
  }
}

// Lay out the one query of the fallback context for the next launch.
__global__ void k_set_state(QState *S, Ctrl *c, uint64_t cur_rows, uint64_t out_word_base, uint64_t out_rows,
                            SrcRows src, uint64_t len3, uint64_t len4) {
  S->cur_row_base = 0;
  S->cur_rows = cur_rows;
  S->cur_word_base = 0;
  S->out_row_base = 0;
  S->out_rows = out_rows;
  S->out_word_base = out_word_base;
  *reinterpret_cast<SrcRows *>(c->fb_src) = src;
  c->len[3] = len3;
  c->len[4] = len4;
}

__global__ void k_copy_src(Wave W) {
  if (threadIdx.x == 0 && blockIdx.x == 0) W.src[0] = *reinterpret_cast<const SrcRows *>(W.ctrl->fb_src);
}

unsigned grid_n(uint64_t n, int sms) {
  uint64_t b = (n + kT - 1) / kT;
  if (b == 0) b = 1;
  return (unsigned)std::min<uint64_t>(b, (uint64_t)sms * 8);
}

}  // namespace

struct Fallback {
  gs_batch *fb = nullptr;
  uint64_t depth_words = 1ull << 25;  // words per level buffer
  uint64_t depth_rows = 1ull << 23;   // rows per level chunk (count/scan arrays)
  uint32_t *buf[kMaxK] = {};
  uint64_t *rscan[kMaxK] = {};
  uint32_t *cnt = nullptr;
  uint64_t *bounds = nullptr;
  uint64_t bounds_cap = 1 << 20;
  uint64_t *d_n = nullptr;
  uint64_t *tmp = nullptr;   // radix sort scratch (zeroed when allocated)
  uint64_t *stmp = nullptr;  // scan scratch (zeroed when allocated)
  // rows of queries with more than cap embeddings
  uint32_t *top = nullptr, *top2 = nullptr, *perm[2] = {}, *key[2] = {};
  uint32_t *pflag = nullptr;                     // projection: run starts [top_rows]
  uint64_t *pscan = nullptr, *ptmp = nullptr;    //   their scan [top_rows + 1] and scan scratch
  uint64_t top_rows = 0;  // capacity in rows
  uint32_t top_k = 0;
  std::vector<void *> allocs;
  ~Fallback() {
    if (fb) batch_destroy(fb);
    for (void *p : allocs) cudaFree(p);
  }
};

void release_fallback(gs_graph *g) {
  delete static_cast<Fallback *>(g->fallback);
  g->fallback = nullptr;
}

template <typename T>
static gs_status falloc(Fallback *f, T **p, uint64_t n) {
  void *q = nullptr;
  cudaError_t e = gs::dev_malloc(&q, sizeof(T) * (n ? n : 1));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (fallback buffers)");
  f->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return GS_OK;
}

static gs_status fallback_ctx(gs_graph *g, Fallback **out) {
  if (g->fallback) {
    *out = static_cast<Fallback *>(g->fallback);
    return GS_OK;
  }
  Fallback *f = new Fallback();
  // Level-buffer sizes can be shrunk (tests exercise the chunking this way).
  if (const char *e = getenv("GS_FALLBACK_DEPTH_WORDS")) f->depth_words = std::max<uint64_t>(strtoull(e, nullptr, 10), 64);
  if (const char *e = getenv("GS_FALLBACK_DEPTH_ROWS")) f->depth_rows = std::max<uint64_t>(strtoull(e, nullptr, 10), 64);
  // A one-query context sized for any query shape.
  std::vector<uint32_t> vt(kMaxK, kAny), vb(kMaxK, kUnbound), es, ed, er;
  for (uint32_t i = 1; i < kMaxK; ++i) { es.push_back(i - 1); ed.push_back(i); er.push_back(0); }
  gs_query q{kMaxK, kMaxK - 1, vt.data(), vb.data(), es.data(), ed.data(), er.data()};
  gs_match_opts o;
  memset(&o, 0, sizeof(o));
  o.mode = GS_COUNT_ONLY;
  gs_status st = batch_create(g, &q, 1, &o, 1, &f->fb, true);
  if (st != GS_OK) {
    delete f;
    return st;
  }
  f->fb->use_graph = false;
  f->fb->fixpoint = true;
  for (uint32_t d = 0; d < kMaxK && st == GS_OK; ++d) {
    st = falloc(f, &f->buf[d], f->depth_words);
    if (st == GS_OK) st = falloc(f, &f->rscan[d], f->depth_rows + 1);
  }
  if (st == GS_OK) st = falloc(f, &f->cnt, f->depth_rows);
  if (st == GS_OK) st = falloc(f, &f->bounds, f->bounds_cap + 1);
  if (st == GS_OK) st = falloc(f, &f->d_n, 1);
  if (st == GS_OK) st = falloc(f, &f->tmp, radix_tmp_words(1));
  if (st == GS_OK) st = falloc(f, &f->stmp, scan_tmp_words(f->depth_rows));
  if (st == GS_OK && (cudaMemset(f->tmp, 0, sizeof(uint64_t) * radix_tmp_words(1)) != cudaSuccess ||
                      cudaMemset(f->stmp, 0, sizeof(uint64_t) * scan_tmp_words(f->depth_rows)) != cudaSuccess))
    st = fail(GS_ERR_CUDA, "cudaMemset (fallback scratch)");
  if (st != GS_OK) {
    delete f;
    return st;
  }
  g->fallback = f;
  *out = f;
  return GS_OK;
}

static gs_status ensure_top(Fallback *f, uint64_t rows, uint32_t k) {
  if (f->top && f->top_rows >= rows && f->top_k >= k) return GS_OK;
  for (void *p : {(void *)f->top, (void *)f->top2, (void *)f->perm[0], (void *)f->perm[1], (void *)f->key[0],
                  (void *)f->key[1], (void *)f->pflag, (void *)f->pscan, (void *)f->ptmp}) {
    if (!p) continue;
    cudaFree(p);
    f->allocs.erase(std::remove(f->allocs.begin(), f->allocs.end(), p), f->allocs.end());
  }
  f->top = f->top2 = f->perm[0] = f->perm[1] = f->key[0] = f->key[1] = f->pflag = nullptr;
  f->pscan = f->ptmp = nullptr;
  gs_status st = falloc(f, &f->top, rows * k);
  if (st == GS_OK) st = falloc(f, &f->top2, rows * k);
  for (int i = 0; i < 2 && st == GS_OK; ++i) {
    st = falloc(f, &f->perm[i], rows);
    if (st == GS_OK) st = falloc(f, &f->key[i], rows);
  }
  if (st == GS_OK) st = falloc(f, &f->pflag, rows);
  if (st == GS_OK) st = falloc(f, &f->pscan, rows + 1);
  if (st == GS_OK) st = falloc(f, &f->ptmp, scan_tmp_words(rows));
  if (st == GS_OK && cudaMemset(f->ptmp, 0, sizeof(uint64_t) * scan_tmp_words(rows)) != cudaSuccess)
    st = fail(GS_ERR_CUDA, "cudaMemset (fallback projection scratch)");
  if (st != GS_OK) return st;
  // radix scratch for `rows` items
  void *t = nullptr;
  cudaError_t e = gs::dev_malloc(&t, sizeof(uint64_t) * radix_tmp_words(rows));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (fallback sort scratch)");
  e = cudaMemset(t, 0, sizeof(uint64_t) * radix_tmp_words(rows));
  if (e != cudaSuccess) {
    cudaFree(t);
    return cuda_fail(e, "cudaMemset (fallback sort scratch)");
  }
  f->allocs.erase(std::remove(f->allocs.begin(), f->allocs.end(), (void *)f->tmp), f->allocs.end());
  cudaFree(f->tmp);
  f->tmp = static_cast<uint64_t *>(t);
  f->allocs.push_back(t);
  f->top_rows = rows;
  f->top_k = k;
  return GS_OK;
}

namespace {

struct FbRun {
  Fallback *f;
  gs_batch *fb;
  Wave W0;
  cudaStream_t s;
  int sms, grp;
  uint32_t k;
  uint8_t pos[kMaxK];
  bool rows;
  uint64_t cap;
  uint64_t top_n = 0;
  int nbits;
  // GS_CHUNKED: final rows go to the callback instead of a running top-cap
  gs_chunk_cb cb = nullptr;
  void *user = nullptr;
  uint32_t query = 0;
  // output columns: the projected vertices pu[0..kp) (every vertex when not
  // projecting); more: more distinct projected tuples than cap were seen
  uint32_t kp = 0;
  uint8_t pu[kMaxK] = {};
  bool proj = false, more = false;
  uint64_t kept = 0;  // rows the last sort kept
};

template <typename T>
gs_status d2h1(T *dst, const T *src, cudaStream_t s) {
  GS_CUDA(cudaMemcpyAsync(dst, src, sizeof(T), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  return GS_OK;
}

// Sort the collected rows (join-order columns) lexicographically on the
// output columns in query-vertex order and keep the first `keep` (for a
// projection: the first row of each distinct projected tuple, the first
// `keep` of those); if `final`, write the output columns in query-vertex
// order into top2, else keep whole rows in top.
gs_status sort_top(FbRun &R, uint64_t keep, bool final) {
  Fallback *f = R.f;
  const uint64_t n = R.top_n;
  R.kept = 0;
  if (n == 0) return GS_OK;
  GS_CUDA(cudaMemcpyAsync(f->d_n, &n, sizeof(n), cudaMemcpyHostToDevice, R.s));
  k_iota_n<<<grid_n(n, R.sms), kT, 0, R.s>>>(f->perm[0], f->d_n);
  int cur = 0;
  for (int c = (int)R.kp - 1; c >= 0; --c) {  // least significant column first (stable passes)
    k_col_keys<<<grid_n(n, R.sms), kT, 0, R.s>>>(f->top, R.k, f->perm[cur], f->d_n, R.pos[R.pu[c]], f->key[0]);
    int r = radix_sort_pairs(f->key[0], f->perm[cur], f->key[1], f->perm[cur ^ 1], f->d_n, f->top_rows, 0, R.nbits,
                             f->tmp, R.s, R.sms);
    cur = r ? cur ^ 1 : cur;
  }
  const uint32_t w = final ? R.kp : R.k;
  ColOrder ord;
  for (uint32_t u = 0; u < w; ++u) ord.c[u] = final ? R.pos[R.pu[u]] : (uint8_t)u;
  if (R.proj) {
    ColOrder cols;
    for (uint32_t c = 0; c < R.kp; ++c) cols.c[c] = R.pos[R.pu[c]];
    k_proj_flags<<<grid_n(n, R.sms), kT, 0, R.s>>>(f->top, R.k, f->perm[cur], f->d_n, cols, R.kp, f->pflag);
    scan_u32(f->pflag, f->pscan, f->d_n, f->top_rows, f->ptmp, R.s, R.sms);
    uint64_t d = 0;
    gs_status st = d2h1(&d, f->pscan + n, R.s);
    if (st != GS_OK) return st;
    if (d > R.cap) R.more = true;
    keep = std::min(keep, d);
    k_take_distinct<<<grid_n(n, R.sms), kT, 0, R.s>>>(f->top, R.k, f->perm[cur], f->pflag, f->pscan, f->d_n, keep, ord,
                                                       w, f->top2);
  } else {
    keep = std::min(keep, n);
    k_take_rows<<<grid_n(keep, R.sms), kT, 0, R.s>>>(f->top, R.k, f->perm[cur], keep, ord, w, f->top2);
  }
  if (!final) {
    GS_CUDA(cudaMemcpyAsync(f->top, f->top2, 4ull * keep * R.k, cudaMemcpyDeviceToDevice, R.s));
    R.top_n = keep;
  }
  R.kept = keep;
  GS_CUDA(cudaStreamSynchronize(R.s));
  return GS_OK;
}

// GS_CHUNKED: the collected final rows, in query-vertex column order, to the
// callback; the buffer starts over.
gs_status flush_chunk(FbRun &R) {
  Fallback *f = R.f;
  const uint64_t n = R.top_n;
  if (n == 0) return GS_OK;
  GS_CUDA(cudaMemcpyAsync(f->d_n, &n, sizeof(n), cudaMemcpyHostToDevice, R.s));
  k_iota_n<<<grid_n(n, R.sms), kT, 0, R.s>>>(f->perm[0], f->d_n);
  ColOrder ord;
  for (uint32_t u = 0; u < R.k; ++u) ord.c[u] = R.pos[u];
  k_take_rows<<<grid_n(n, R.sms), kT, 0, R.s>>>(f->top, R.k, f->perm[0], n, ord, R.k, f->top2);
  GS_CUDA(cudaStreamSynchronize(R.s));
  R.cb(f->top2, n, R.k, R.query, R.user);
  R.top_n = 0;
  return GS_OK;
}

void set_state(FbRun &R, uint64_t cur_rows, uint64_t out_word_base, uint64_t out_rows, SrcRows src, uint64_t len3,
               uint64_t len4) {
  k_set_state<<<1, 1, 0, R.s>>>(R.W0.qs, R.W0.ctrl, cur_rows, out_word_base, out_rows, src, len3, len4);
  k_copy_src<<<1, 32, 0, R.s>>>(R.W0);
}

// Expand the n rows of level s held in buf[s] to the last level.
gs_status expand(FbRun &R, uint32_t s, uint64_t n) {
  Fallback *f = R.f;
  Wave W = R.W0;
  W.lvl[s & 1] = f->buf[s];
  if (s + 1 < kMaxK) W.lvl[(s + 1) & 1] = f->buf[s + 1];
  W.row_cnt = f->cnt;
  W.row_scan = f->rscan[s];
  set_state(R, n, 0, 0, SrcRows{0, 0, 0}, n, 0);
  launch_join_count(W, s, R.grp, R.s, R.sms);
  scan_u32(f->cnt, f->rscan[s], &W.ctrl->len[3], f->depth_rows, f->stmp, R.s, R.sms);
  uint64_t T = 0;
  gs_status st = d2h1(&T, f->rscan[s] + n, R.s);
  if (st != GS_OK) return st;
  const bool final = s + 2 == R.k;
  if (T == 0 || (final && !R.rows)) return GS_OK;
  const uint64_t width = s + 2;
  uint64_t B = final ? f->top_rows / 4 : std::min(f->depth_rows, f->depth_words / width) / 2;
  B = std::max<uint64_t>(B, 1);
  const uint64_t nb = (T + B - 1) / B;
  std::vector<uint64_t> bounds(nb + 1), scan_at(nb + 1);
  if (nb == 1) {
    bounds[0] = 0;
    bounds[1] = n;
  } else {
    if (nb > f->bounds_cap) return fail(GS_ERR_OOM, "chunked join: too many chunks");
    k_chunk_bounds<<<grid_n(nb + 1, R.sms), kT, 0, R.s>>>(f->rscan[s], n, B, nb, f->bounds);
    GS_CUDA(cudaMemcpyAsync(bounds.data(), f->bounds, 8 * (nb + 1), cudaMemcpyDeviceToHost, R.s));
    GS_CUDA(cudaStreamSynchronize(R.s));
  }
  for (uint64_t j = 0; j < nb; ++j) {
    const uint64_t a = bounds[j], b = bounds[j + 1];
    if (a >= b) continue;
    uint64_t sa = 0, sb = 0;
    if ((st = d2h1(&sa, f->rscan[s] + a, R.s)) != GS_OK) return st;
    if ((st = d2h1(&sb, f->rscan[s] + b, R.s)) != GS_OK) return st;
    const uint64_t out = sb - sa;
    if (out == 0) continue;
    Wave Wc = W;
    Wc.row_scan = f->rscan[s] + a;
    const SrcRows src{0, b - a, a * (s + 1)};
    if (final) {
      if (R.top_n + out > f->top_rows) {
        if ((st = R.cb ? flush_chunk(R) : sort_top(R, R.cap, false)) != GS_OK) return st;
        if (R.top_n + out > f->top_rows) return fail(GS_ERR_OOM, "chunked join: row buffer too small");
      }
      Wc.out = f->top;
      Wc.out_q = nullptr;
      set_state(R, 0, R.top_n * R.k, 1, src, 0, b - a);
      launch_join_write(Wc, s, R.grp, R.s, R.sms);
      R.top_n += out;
    } else {
      set_state(R, 0, 0, 0, src, 0, b - a);
      launch_join_write(Wc, s, R.grp, R.s, R.sms);
      if ((st = expand(R, s + 1, out)) != GS_OK) return st;
    }
  }
  return GS_OK;
}

}  // namespace

static std::mutex g_fallback_mu;  // one chunked join at a time (the context is shared)

gs_status fallback_query(gs_batch *b, uint32_t i) {
  std::lock_guard<std::mutex> lk(g_fallback_mu);
  Fallback *f = nullptr;
  gs_status st = fallback_ctx(b->g, &f);
  if (st != GS_OK) return st;
  gs_batch *fb = f->fb;
  const DQuery &src = b->hq[i];
  // load the packed query
  fb->hq.resize(1);
  fb->hq[0] = src;
  fb->hq[0].qv_base = 0;
  fb->hq[0].qe_base = 0;
  fb->hq[0].status = QS_OK;
  fb->hstatus.assign(1, GS_OK);
  fb->n = 1;
  fb->has_rev = (src.refine_flags & kRefineRev) != 0;
  fb->max_k = src.k;
  fb->waves.assign(1, WaveDesc{0, 1, 0, src.k, 0, src.m});
  fb->wave_k.assign(1, (int)src.k);
  cudaStream_t s = fb->stream;
  GS_CUDA(cudaMemcpyAsync(fb->all_dq, fb->hq.data(), sizeof(DQuery), cudaMemcpyHostToDevice, s));
  GS_CUDA(cudaMemcpyAsync(fb->dwaves, fb->waves.data(), sizeof(WaveDesc), cudaMemcpyHostToDevice, s));
  GS_CUDA(cudaMemsetAsync(&fb->W.ctrl->wave, 0, sizeof(uint32_t), s));
  enqueue_wave(fb, (int)src.k, false, &fb->evs);
  st = refine_to_fixpoint(fb);
  if (st != GS_OK) return st;
  enqueue_wave_tail(fb, (int)src.k, false, &fb->evs, 2);
  DQuery dq;
  GS_CUDA(cudaMemcpyAsync(&dq, fb->W.dq, sizeof(DQuery), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  const bool stream = b->on_chunk != nullptr;  // GS_CHUNKED: every embedding to the callback
  const bool want_rows = stream || (src.mode != GS_COUNT_ONLY && src.cap > 0);
  // rows per streamed chunk: the chunk budget (default 1 GiB) over the row width
  const uint64_t chunk_rows =
      std::max<uint64_t>((b->key_chunk ? b->key_chunk : (1ull << 30)) / (4ull * std::max<uint32_t>(src.k, 1)), 4096);
  std::vector<uint32_t> rows;
  uint64_t count = 0, fp = 0;
  bool more = false;
  if (dq.status == QS_OK) {
    FbRun R{f, fb, fb->W, s, fb->sms, fb->group, src.k};
    memcpy(R.pos, dq.pos, sizeof(R.pos));
    R.rows = want_rows;
    R.cap = src.cap;
    R.kp = src.kp;
    memcpy(R.pu, src.pu, sizeof(R.pu));
    R.proj = src.proj != 0;
    if (stream) {
      R.cb = b->on_chunk;
      R.user = b->chunk_user;
      R.query = i;
    }
    int nb = 1;
    while (nb < 32 && ((uint64_t)(b->g->d.V - 1) >> nb)) ++nb;
    R.nbits = nb;
    if (want_rows) {
      st = ensure_top(f, stream ? chunk_rows : 2 * std::max<uint64_t>(src.cap, 1ull << 16), src.k);
      if (st != GS_OK) return st;
    }
    uint32_t len = 0;
    uint64_t off = 0;
    GS_CUDA(cudaMemcpyAsync(&len, fb->W.flist_len + dq.join[0], 4, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaMemcpyAsync(&off, fb->W.flist_off + dq.join[0], 8, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    if (src.k == 1) {
      k_list_fp<<<grid_n(len, R.sms), kT, 0, s>>>(fb->W.flist + off, len,
                                                  reinterpret_cast<unsigned long long *>(&fb->W.qs[0].fp));
      GS_CUDA(cudaMemsetAsync(&fb->W.qs[0].count, 0, 8, s));
      uint64_t c = len;
      GS_CUDA(cudaMemcpyAsync(&fb->W.qs[0].count, &c, 8, cudaMemcpyHostToDevice, s));
      if (stream) {  // the rows are the candidates themselves
        GS_CUDA(cudaStreamSynchronize(s));
        for (uint64_t a = 0; a < len; a += chunk_rows)
          R.cb(fb->W.flist + off + a, std::min<uint64_t>(chunk_rows, len - a), 1, i, R.user);
      } else if (want_rows) {
        const uint64_t keep = std::min<uint64_t>(len, src.cap);
        rows.resize(keep);
        if (keep) GS_CUDA(cudaMemcpyAsync(rows.data(), fb->W.flist + off, 4 * keep, cudaMemcpyDeviceToHost, s));
      }
      GS_CUDA(cudaStreamSynchronize(s));
    } else {
      // level 0 = the candidates of join[0], in chunks of the level buffer
      const uint64_t step = std::min(f->depth_rows, f->depth_words);
      for (uint64_t a = 0; a < len && st == GS_OK; a += step) {
        const uint64_t m = std::min<uint64_t>(step, len - a);
        GS_CUDA(cudaMemcpyAsync(f->buf[0], fb->W.flist + off + a, 4 * m, cudaMemcpyDeviceToDevice, s));
        st = expand(R, 0, m);
      }
      if (st == GS_OK && stream) {
        st = flush_chunk(R);
      } else if (st == GS_OK && want_rows && R.top_n) {
        st = sort_top(R, src.cap, true);
        if (st == GS_OK) {
          rows.resize(R.kept * R.kp);
          GS_CUDA(cudaMemcpyAsync(rows.data(), f->top2, 4 * rows.size(), cudaMemcpyDeviceToHost, s));
          GS_CUDA(cudaStreamSynchronize(s));
        }
      }
    }
    if (st != GS_OK) {
      launch_clear(fb->W, s, fb->sms);
      cudaStreamSynchronize(s);
      return st;
    }
    GS_CUDA(cudaMemcpyAsync(&count, &fb->W.qs[0].count, 8, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaMemcpyAsync(&fp, &fb->W.qs[0].fp, 8, cudaMemcpyDeviceToHost, s));
    more = R.more;
  }
  launch_clear(fb->W, s, fb->sms);
  GS_CUDA(cudaStreamSynchronize(s));
  if (dq.status == QS_OVERFLOW) return GS_OK;  // still too large: reported as GS_ERR_OOM
  b->count[i] = dq.status == QS_OK ? count : 0;
  b->fp[i] = dq.status == QS_OK ? fp : 0;
  b->status[i] = dq.status == QS_EMPTY ? QS_EMPTY : QS_OK;
  b->fb_rows[i] = std::move(rows);
  b->fb_more[i] = more ? 1 : 0;
  b->fb_done[i] = 1;
  return GS_OK;
}

}  // namespace gs
