// Domain-graph exploration (Ch. 5, "Domain-specific knowledge graph
// generation"): the concepts within a few hops of a set of seed concepts,
// found level by level the way the filtering phase explores (warps over the
// frontier vertices' coalesced adjacency rows).
//
// State: level[V] (uint8, 255 = not reached), a visited bitmap claimed with
// atomicOr, and two frontier lists.  A level step reads the frontier size
// from device memory, so the whole exploration runs without a host sync.
// The last level needs neither the bitmap nor a frontier.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kKT = 256;  // threads per block
constexpr uint32_t kFullMask = 0xFFFFFFFFu;

struct KhopArgs {
  const uint64_t *off[2];
  const uint32_t *adj[2];
  uint32_t dirs;           // bit 0: follow edges forwards, bit 1: backwards
  uint32_t relmask[8];     // relations followed (bit r)
  uint32_t all_rels;       // every relation: skip the mask test
  uint32_t V;
  uint8_t *level;
  uint32_t *vis;           // visited bitmap [ceil(V/32)]
  uint32_t *front[2];      // frontier lists [V]
  unsigned long long *cnt; // vertices per level [levels + 2]
  unsigned long long *grab;  // per level: frontier entries handed out to warps so far
  unsigned long long *edges;  // adjacency entries scanned
  uint32_t *err;           // bit 0: a seed out of range
};

__device__ __forceinline__ bool claim(const KhopArgs &A, uint32_t v) {
  const uint32_t bit = 1u << (v & 31);
  if (A.vis[v >> 5] & bit) return false;
  return !(atomicOr(&A.vis[v >> 5], bit) & bit);
}

// Seeds: level 0, frontier 0 (repeated seeds claimed once).
__global__ void k_khop_seeds(KhopArgs A, const uint32_t *seeds, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t s = seeds[i];
    if (s >= A.V) {
      atomicOr(A.err, 1u);
      continue;
    }
    if (claim(A, s)) {
      A.level[s] = 0;
      A.front[0][atomicAdd(&A.cnt[0], 1ull)] = s;
    }
  }
}

// One level: the frontier vertices of level l (front[l & 1], cnt[l] of
// them) scan their rows in the followed directions; each neighbour over a
// followed relation that is not yet visited gets level l + 1.  Load
// balanced: a warp takes up to 32 frontier vertices at a time from a shared
// counter (fewer when the frontier is small, and when it is smaller than the
// grid several warps share one vertex's rows), scans their row lengths,
// and walks the concatenated rows 32 entries per step, each lane finding the
// vertex and row of its entry by a search over the scan held in registers.
// Below the last level a neighbour is claimed in the visited bitmap and
// appended to the next frontier (one atomic per warp and step).  The last
// level builds no frontier: an unreached neighbour's level is written
// without atomics (every writer writes the same value) and counted after.
// Entry t of a warp's concatenated rows: the owner lane (a search over the
// inclusive counts held in registers) and the adjacency entry itself.
__device__ __forceinline__ uint32_t row_entry(const KhopArgs &A, uint32_t incl, uint32_t n0, uint32_t n1, uint64_t b0,
                                              uint64_t b1, uint32_t t, uint32_t total, bool &valid) {
  int owner = 0;
  for (int step = 16; step; step >>= 1) {
    const uint32_t c = __shfl_sync(kFullMask, incl, owner + step - 1);
    if (c <= t) owner += step;
  }
  const uint32_t on0 = __shfl_sync(kFullMask, n0, owner);
  const uint32_t before = __shfl_sync(kFullMask, incl, owner) - on0 - __shfl_sync(kFullMask, n1, owner);
  const uint64_t ob0 = __shfl_sync(kFullMask, b0, owner), ob1 = __shfl_sync(kFullMask, b1, owner);
  valid = t < total;
  if (!valid) return 0;
  const uint32_t k = t - before;  // entry k of the owner's rows: forward first, then backward
  return k < on0 ? A.adj[0][ob0 + k] : A.adj[1][ob1 + (k - on0)];
}

__device__ __forceinline__ bool follow(const KhopArgs &A, uint32_t x) {
  const uint32_t r = x >> kNbrBits;
  return A.all_rels || ((A.relmask[r >> 5] >> (r & 31)) & 1u);
}

template <bool LAST>
__global__ void __launch_bounds__(kKT, 6) k_khop_level(KhopArgs A, uint32_t l) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nfront = A.cnt[l];
  const uint32_t *front = A.front[l & 1];
  uint32_t *next = A.front[(l + 1) & 1];
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  // work units: vpw frontier vertices per warp when the frontier is large;
  // when it is smaller than the grid, wpv warps share each vertex's rows
  const uint64_t per_warp = (nfront + nwarps - 1) / nwarps;
  const uint32_t vpw = per_warp >= 32 ? 32u : (per_warp ? (uint32_t)per_warp : 1u);
  const uint32_t wpv = nfront && nfront < nwarps ? (uint32_t)min((uint64_t)32, nwarps / nfront) : 1u;
  const bool fw = A.dirs & 1u, bw = (A.dirs >> 1) & 1u;
  uint64_t scanned = 0;
  for (;;) {
    // the next unit, taken from a shared counter so that warps that drew
    // short rows take more
    unsigned long long g = 0;
    if (lane == 0) g = atomicAdd(&A.grab[l], (unsigned long long)(wpv > 1 ? 1u : vpw));
    g = __shfl_sync(kFullMask, g, 0);
    const uint64_t i0 = wpv > 1 ? g / wpv : g;
    const uint32_t sub = wpv > 1 ? (uint32_t)(g % wpv) : 0u;
    if (i0 >= nfront) break;
    // this lane's frontier vertex: its forward and backward row ranges
    uint64_t b0 = 0, b1 = 0;
    uint32_t n0 = 0, n1 = 0;
    if (lane < vpw && i0 + lane < nfront) {
      const uint32_t u = front[i0 + lane];
      if (fw) { b0 = A.off[0][u]; n0 = (uint32_t)(A.off[0][u + 1] - b0); }
      if (bw) { b1 = A.off[1][u]; n1 = (uint32_t)(A.off[1][u + 1] - b1); }
    }
    // inclusive scan of the lanes' entry counts
    uint32_t incl = n0 + n1;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(kFullMask, incl, 31);
    if (sub == 0) scanned += total;
    const uint32_t stride = 32 * wpv;
    if (LAST) {
      // two entries per lane and step: independent loads in flight
      for (uint32_t t0 = 32 * sub; t0 < total; t0 += 2 * stride) {
        bool v0, v1;
        const uint32_t x0 = row_entry(A, incl, n0, n1, b0, b1, t0 + lane, total, v0);
        const uint32_t x1 = row_entry(A, incl, n0, n1, b0, b1, t0 + stride + lane, total, v1);
        const uint32_t w0 = x0 & kNbrMask, w1 = x1 & kNbrMask;
        const bool f0 = v0 && follow(A, x0), f1 = v1 && follow(A, x1);
        const uint8_t l0 = f0 ? A.level[w0] : 0, l1 = f1 ? A.level[w1] : 0;
        if (f0 && l0 == 255) A.level[w0] = (uint8_t)(l + 1);
        if (f1 && l1 == 255) A.level[w1] = (uint8_t)(l + 1);
      }
      continue;
    }
    for (uint32_t t0 = 32 * sub; t0 < total; t0 += stride) {
      bool valid;
      const uint32_t x = row_entry(A, incl, n0, n1, b0, b1, t0 + lane, total, valid);
      const uint32_t w = x & kNbrMask;
      const bool mine = valid && follow(A, x) && claim(A, w);
      const uint32_t m = __ballot_sync(kFullMask, mine);
      if (m) {
        unsigned long long base = 0;
        const int leader = __ffs(m) - 1;
        if (lane == leader) base = atomicAdd(&A.cnt[l + 1], (unsigned long long)__popc(m));
        base = __shfl_sync(kFullMask, base, leader);
        if (mine) {
          A.level[w] = (uint8_t)(l + 1);
          next[base + __popc(m & ((1u << lane) - 1))] = w;
        }
      }
    }
  }
  if (lane == 0 && scanned) atomicAdd(A.edges, (unsigned long long)scanned);
}

// Vertices whose level is l (the last level's count), four level bytes per
// load where aligned.
__global__ void k_count_level(KhopArgs A, uint32_t l) {
  uint32_t c = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < A.V; i += (uint64_t)gridDim.x * blockDim.x)
    c += A.level[i] == l;
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFullMask, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&A.cnt[l], (unsigned long long)c);
}

__global__ void k_fill_u8(uint8_t *p, uint64_t n, uint8_t v) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

}  // namespace

// Per-graph buffers of the exploration, made on first use.
struct Khop {
  uint8_t *level = nullptr;
  uint32_t *vis = nullptr, *front[2] = {}, *seeds = nullptr, *err = nullptr;
  unsigned long long *cnt = nullptr, *edges = nullptr;
  uint32_t seeds_cap = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  ~Khop() {
    for (void *p : {(void *)level, (void *)vis, (void *)front[0], (void *)front[1], (void *)seeds, (void *)err,
                    (void *)cnt, (void *)edges})
      if (p) cudaFree(p);
    if (stream) cudaStreamDestroy(stream);
  }
};

void release_khop(gs_graph *g) {
  delete static_cast<Khop *>(g->khop);
  g->khop = nullptr;
}

static std::mutex g_khop_ctx_mu;  // first use on a graph from several threads

static gs_status khop_ctx(gs_graph *g, Khop **out) {
  std::lock_guard<std::mutex> lk(g_khop_ctx_mu);
  if (g->khop) {
    *out = static_cast<Khop *>(g->khop);
    return GS_OK;
  }
  Khop *k = new Khop();
  const uint64_t V = g->d.V, words = (V + 31) / 32;
  cudaError_t e = gs::dev_malloc(&k->level, V);
  if (e == cudaSuccess) e = gs::dev_malloc(&k->vis, 4 * words);
  if (e == cudaSuccess) e = gs::dev_malloc(&k->front[0], 4 * V);
  if (e == cudaSuccess) e = gs::dev_malloc(&k->front[1], 4 * V);
  if (e == cudaSuccess) e = gs::dev_malloc(&k->err, 4);
  if (e == cudaSuccess) e = gs::dev_malloc(&k->cnt, 8 * 512);  // counts [0, 256), hand-out counters [256, 512)
  if (e == cudaSuccess) e = gs::dev_malloc(&k->edges, 8);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&k->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete k;
    return cuda_fail(e, "gs_khop buffers");
  }
  g->khop = k;
  *out = k;
  return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_khop(gs_graph *g, const uint32_t *seeds, uint32_t nseeds, const gs_khop_opts *opts,
                             uint8_t *level_out, uint64_t *counts, uint64_t *edges_scanned) {
  if (!g || !opts || !level_out || !counts || (nseeds && !seeds)) return fail(GS_ERR_INVALID, "gs_khop: null argument");
  if (opts->levels > 254) return fail(GS_ERR_INVALID, "gs_khop: levels must be at most 254");
  if (opts->directions == 0 || opts->directions > (GS_KHOP_OUT | GS_KHOP_IN))
    return fail(GS_ERR_INVALID, "gs_khop: directions must be GS_KHOP_OUT, GS_KHOP_IN or both");
  if (opts->nrels && !opts->rels) return fail(GS_ERR_INVALID, "gs_khop: null relation list");
  KhopArgs A;
  memset(&A, 0, sizeof(A));
  A.all_rels = opts->rels ? 0u : 1u;
  for (uint32_t i = 0; opts->rels && i < opts->nrels; ++i) {
    const uint32_t r = opts->rels[i];
    if (r >= g->d.R) return fail(GS_ERR_INVALID, "gs_khop: relation out of range");
    A.relmask[r >> 5] |= 1u << (r & 31);
  }
  const bool on_dev = (opts->flags & GS_DEVICE_PTRS) != 0;
  if (!on_dev)
    for (uint32_t i = 0; i < nseeds; ++i)
      if (seeds[i] >= g->d.V) return fail(GS_ERR_INVALID, "gs_khop: seed out of range");
  GS_CUDA(cudaSetDevice(g->device));
  Khop *k = nullptr;
  gs_status st = khop_ctx(g, &k);
  if (st != GS_OK) return st;
  std::lock_guard<std::mutex> lk(k->mu);
  const cudaStream_t s = opts->cuda_stream ? static_cast<cudaStream_t>(opts->cuda_stream) : k->stream;
  const uint32_t V = g->d.V, L = opts->levels;
  const uint32_t *dseeds = seeds;
  if (!on_dev && nseeds) {
    if (nseeds > k->seeds_cap) {
      if (k->seeds) cudaFree(k->seeds);
      k->seeds = nullptr;
      k->seeds_cap = 0;
      GS_CUDA(gs::dev_malloc(&k->seeds, 4ull * nseeds));
      k->seeds_cap = nseeds;
    }
    GS_CUDA(cudaMemcpyAsync(k->seeds, seeds, 4ull * nseeds, cudaMemcpyHostToDevice, s));
    dseeds = k->seeds;
  }
  A.off[0] = g->d.off[0]; A.off[1] = g->d.off[1];
  A.adj[0] = g->d.adj[0]; A.adj[1] = g->d.adj[1];
  A.dirs = opts->directions;
  A.V = V;
  A.level = on_dev ? level_out : k->level;
  A.vis = k->vis;
  A.front[0] = k->front[0]; A.front[1] = k->front[1];
  A.cnt = k->cnt;
  A.grab = k->cnt + 256;
  A.edges = k->edges;
  A.err = k->err;
  const unsigned fill_grid = (unsigned)std::min<uint64_t>((V + kKT - 1) / kKT, (uint64_t)g->num_sms * 8);
  k_fill_u8<<<fill_grid, kKT, 0, s>>>(A.level, V, 255);
  GS_CUDA(cudaMemsetAsync(A.vis, 0, 4ull * ((V + 31) / 32), s));
  GS_CUDA(cudaMemsetAsync(A.cnt, 0, 8ull * (L + 2), s));
  GS_CUDA(cudaMemsetAsync(A.grab, 0, 8ull * (L + 1), s));
  GS_CUDA(cudaMemsetAsync(A.edges, 0, 8, s));
  GS_CUDA(cudaMemsetAsync(A.err, 0, 4, s));
  if (nseeds) {
    const unsigned sg = (unsigned)std::min<uint64_t>((nseeds + kKT - 1) / kKT, (uint64_t)g->num_sms * 4);
    k_khop_seeds<<<sg, kKT, 0, s>>>(A, dseeds, nseeds);
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_khop_level<false>, kKT, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const unsigned grid = (unsigned)(g->num_sms * std::min(per_sm, 8));
  for (uint32_t l = 0; l + 1 < L; ++l) k_khop_level<false><<<grid, kKT, 0, s>>>(A, l);
  if (L > 0) {
    k_khop_level<true><<<grid, kKT, 0, s>>>(A, L - 1);
    k_count_level<<<fill_grid, kKT, 0, s>>>(A, L);
  }
  GS_CUDA(cudaGetLastError());
  std::vector<unsigned long long> c(L + 1);
  uint32_t err = 0;
  unsigned long long ed = 0;
  GS_CUDA(cudaMemcpyAsync(c.data(), A.cnt, 8ull * (L + 1), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaMemcpyAsync(&err, A.err, 4, cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaMemcpyAsync(&ed, A.edges, 8, cudaMemcpyDeviceToHost, s));
  if (!on_dev) GS_CUDA(cudaMemcpyAsync(level_out, A.level, V, cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (err & 1u) return fail(GS_ERR_INVALID, "gs_khop: seed out of range");
  for (uint32_t l = 0; l <= L; ++l) counts[l] = c[l];
  if (edges_scanned) *edges_scanned = ed;
  return GS_OK;
}
