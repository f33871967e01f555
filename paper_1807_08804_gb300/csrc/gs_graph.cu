// Data-graph storage (Section 3.3.1: a "nodes array" of row offsets and an
// "edges array" of neighbours, plus node- and edge-label arrays) built in
// both directions (Section 3.5: "incoming and outgoing graph
// representations"), canonicalised on the device:
//   - each row sorted by (relation, neighbour) and packed rel << 24 | nbr, so
//     a relation's neighbours form one ascending run found by binary search;
//   - repeated (src, rel, dst) triples dropped;
//   - per direction, a second CSR of the distinct neighbours over all
//     relations (ascending), read by variable edges;
//   - per-vertex, per-(direction, relation) distinct-neighbour counts kept
//     as 4-bit signatures for the candidate test (Definition 3.3's degree
//     condition, read per direction and relation, plus one plane per
//     direction over all relations).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "gs_internal.h"

namespace gs {

static thread_local std::string t_last_error;

void set_error(const std::string &msg) { t_last_error = msg; }
gs_status fail(gs_status st, const std::string &msg) {
  set_error(msg);
  return st;
}
namespace {
std::atomic<int64_t> g_fail_alloc_after{-1};  // allocations left before the armed failure; -1 = none
}

void debug_fail_alloc(int64_t after) { g_fail_alloc_after.store(after < 0 ? -1 : after); }

cudaError_t dev_malloc_bytes(void **p, size_t bytes) {
  int64_t left = g_fail_alloc_after.load(std::memory_order_relaxed);
  while (left >= 0) {
    if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
      if (left == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

gs_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA;
}

namespace {

constexpr int kT = 256;

inline unsigned blocks_for(uint64_t n, int per = kT, unsigned cap = 1u << 20) {
  uint64_t b = (n + per - 1) / per;
  if (b == 0) b = 1;
  return (unsigned)(b < cap ? b : cap);
}

// Validation: bit 0 offsets, bit 1 target, bit 2 relation, bit 3 type.
__global__ void k_validate(uint32_t V, uint64_t E, const uint64_t *ro, const uint32_t *col, const uint32_t *rel,
                           const uint32_t *vt, uint32_t T, uint32_t R, uint32_t *err) {
  uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = tid; v < V; v += stride) {
    if (ro[v] > ro[v + 1]) atomicOr(err, 1u);
    if (vt[v] >= T) atomicOr(err, 8u);
  }
  if (tid == 0 && (ro[0] != 0 || ro[V] != E)) atomicOr(err, 1u);
  for (uint64_t e = tid; e < E; e += stride) {
    if (col[e] >= V) atomicOr(err, 2u);
    if (rel[e] >= R) atomicOr(err, 4u);
  }
}

// Expand rows to triples: key = rel << 24 | dst, val = src.
__global__ void k_expand(uint32_t V, const uint64_t *ro, const uint32_t *col, const uint32_t *rel, uint32_t *key,
                         uint32_t *val) {
  uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = tid; v < V; v += stride)
    for (uint64_t e = ro[v]; e < ro[v + 1]; ++e) {
      key[e] = (rel[e] << kNbrBits) | col[e];
      val[e] = (uint32_t)v;
    }
}

// After sorting by (row, packed): keep[i] = first occurrence.
__global__ void k_mark_first(uint64_t n, const uint32_t *row, const uint32_t *packed, uint32_t *keep) {
  uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < n; i += stride)
    keep[i] = (i == 0 || row[i] != row[i - 1] || packed[i] != packed[i - 1]) ? 1u : 0u;
}

__global__ void k_compact_triples(uint64_t n, const uint32_t *row, const uint32_t *packed, const uint32_t *keep,
                                  const uint64_t *pos, uint32_t *out_row, uint32_t *out_packed) {
  uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < n; i += stride)
    if (keep[i]) {
      out_row[pos[i]] = row[i];
      out_packed[pos[i]] = packed[i];
    }
}

// Row lengths by counting; rows are contiguous after the sort.
__global__ void k_row_count(uint64_t n, const uint32_t *row, uint32_t *cnt) {
  uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < n; i += stride) atomicAdd(&cnt[row[i]], 1u);
}

// Re-key kept triples for the incoming direction: key = rel << 24 | src, val = dst.
__global__ void k_rekey_in(uint64_t n, const uint32_t *src, const uint32_t *packed, uint32_t *key, uint32_t *val) {
  uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < n; i += stride) {
    key[i] = (packed[i] & ~kNbrMask) | src[i];
    val[i] = packed[i] & kNbrMask;
  }
}

// Any-relation rows: key = neighbour (relation field 0), val = row vertex.
__global__ void k_strip_rel(uint64_t n, const uint32_t *packed, const uint32_t *row, uint32_t *key, uint32_t *val) {
  uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < n; i += stride) {
    key[i] = packed[i] & kNbrMask;
    val[i] = row[i];
  }
}

// Signatures: one thread per vertex of one adjacency plane walks its sorted
// row and ORs each relation's saturated count into plane plane0 + relation.
__global__ void k_signatures(uint32_t V, const uint64_t *off, const uint32_t *adj, uint32_t plane0, uint32_t *sig,
                             uint64_t sig_words) {
  uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = tid; v < V; v += stride) {
    uint64_t b = off[v], e = off[v + 1];
    uint64_t i = b;
    while (i < e) {
      uint32_t r = adj[i] >> kNbrBits;
      uint64_t j = i;
      while (j < e && (adj[j] >> kNbrBits) == r) ++j;
      uint32_t c = (uint32_t)((j - i) > 15 ? 15 : (j - i));
      atomicOr(&sig[(uint64_t)(plane0 + r) * sig_words + (v >> 3)], c << ((v & 7) * 4));
      i = j;
    }
  }
}

// Vertices per (type, signature plane, nibble value): one block per (plane,
// vertex chunk), counts gathered in shared memory first.  hist holds
// (T + 1) * P * 16 counters; row T counts every vertex (the untyped case).
__global__ void __launch_bounds__(256) k_sig_hist(uint32_t V, uint32_t T, uint32_t P, const uint8_t *vtype,
                                                  const uint32_t *sig, uint64_t sig_words, uint32_t *hist) {
  __shared__ uint32_t h[257 * 16];
  const uint32_t p = blockIdx.y;
  for (uint32_t i = threadIdx.x; i < (T + 1) * 16; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t *plane = sig + (uint64_t)p * sig_words;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t n = (plane[v >> 3] >> ((v & 7) * 4)) & 15u;
    atomicAdd(&h[vtype[v] * 16 + n], 1u);
    atomicAdd(&h[T * 16 + n], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < (T + 1) * 16; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[((uint64_t)(i >> 4) * P + p) * 16 + (i & 15)], h[i]);
}

// Neighbour-type masks: for each vertex v and each relation of one adjacency
// plane, the OR of 1 << (type mod 32) over v's neighbours over that relation,
// stored in mask plane plane0 + relation.
__global__ void k_type_masks(uint32_t V, const uint64_t *off, const uint32_t *adj, uint32_t plane0,
                             const uint8_t *vtype, uint32_t *tmask) {
  uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = tid; v < V; v += stride) {
    const uint64_t b = off[v], e = off[v + 1];
    uint64_t i = b;
    while (i < e) {
      const uint32_t r = adj[i] >> kNbrBits;
      uint32_t m = 0;
      for (; i < e && (adj[i] >> kNbrBits) == r; ++i) m |= 1u << (vtype[adj[i] & kNbrMask] & 31u);
      tmask[(uint64_t)(plane0 + r) * V + v] = m;
    }
  }
}

// Type-ordered copies of the signature planes and neighbour-type masks:
// entry x of a plane belongs to vertex tvid[x], so a filter that walks a
// type's list reads them contiguously.  One thread per 8 list entries (one
// signature word) and plane.
__global__ void k_type_order(uint32_t V, uint32_t P, const uint32_t *tvid, const uint32_t *sig, uint64_t sig_words,
                             const uint32_t *tmask, uint32_t *sig_t, uint32_t *tmask_t) {
  const uint64_t words = (V + 7) / 8;
  const uint64_t n = words * P;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t p = i / words, wd = i % words;
    uint32_t out = 0;
    for (uint32_t e = 0; e < 8; ++e) {
      const uint64_t x = wd * 8 + e;
      if (x >= V) break;
      const uint32_t v = tvid[x];
      out |= ((sig[p * sig_words + (v >> 3)] >> ((v & 7) * 4)) & 15u) << (e * 4);
      tmask_t[p * V + x] = tmask[p * V + v];
    }
    sig_t[p * sig_words + wd] = out;
  }
}

__global__ void k_iota(uint32_t n, uint32_t *out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)i;
}

__global__ void k_types(uint32_t V, const uint32_t *vt, uint8_t *out, uint32_t *hist) {
  uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = tid; v < V; v += stride) {
    out[v] = (uint8_t)vt[v];
    atomicAdd(&hist[vt[v]], 1u);
  }
}

int bits_for(uint64_t maxval) {
  int b = 1;
  while (b < 32 && (maxval >> b)) ++b;
  return b;
}

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  template <typename T>
  T *as() const { return static_cast<T *>(p); }
};

}  // namespace

// Build one direction: given (row, packed) pairs, sort by (row, packed),
// drop repeats, and produce off[V+1], adj[n'].  Returns kept count.
static gs_status build_direction(uint32_t V, uint32_t R, uint64_t n, uint32_t *key, uint32_t *val, uint32_t *k1,
                                 uint32_t *v1, uint64_t *scan_buf, uint64_t *tmp, uint64_t *stmp, uint64_t *d_n,
                                 cudaStream_t s,
                                 int sms, uint64_t **off_out, uint32_t **adj_out, uint32_t **row_out, uint64_t *kept) {
  // (1) by packed key (carry row), (2) stably by row (carry packed)
  int cur = radix_sort_pairs(key, val, k1, v1, d_n, n, 0, kNbrBits + bits_for(R ? R - 1 : 0), tmp, s, sms);
  uint32_t *pk = cur ? k1 : key, *rw = cur ? v1 : val;
  uint32_t *pk_alt = cur ? key : k1, *rw_alt = cur ? val : v1;
  cur = radix_sort_pairs(rw, pk, rw_alt, pk_alt, d_n, n, 0, bits_for(V ? V - 1 : 0), tmp, s, sms);
  uint32_t *row = cur ? rw_alt : rw, *packed = cur ? pk_alt : pk;
  uint32_t *frow = cur ? rw : rw_alt, *fpacked = cur ? pk : pk_alt;  // free buffers
  // de-duplicate
  uint32_t *keep = frow;  // reuse as flags
  k_mark_first<<<blocks_for(n), kT, 0, s>>>(n, row, packed, keep);
  scan_u32(keep, scan_buf, d_n, n, stmp, s, sms);
  uint64_t total = 0;
  GS_CUDA(cudaMemcpyAsync(&total, scan_buf + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  DevBuf adj_b, crow_b, off_b;  // freed on an early return, handed out at the end
  GS_CUDA(gs::dev_malloc(&adj_b.p, sizeof(uint32_t) * (total ? total : 1)));
  GS_CUDA(gs::dev_malloc(&crow_b.p, sizeof(uint32_t) * (total ? total : 1)));
  uint32_t *adj = adj_b.as<uint32_t>(), *crow = crow_b.as<uint32_t>();
  k_compact_triples<<<blocks_for(n), kT, 0, s>>>(n, row, packed, keep, scan_buf, crow, adj);
  (void)fpacked;
  // offsets
  uint32_t *cnt = frow;  // keep flags no longer needed after compaction
  GS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (V + 1), s));
  k_row_count<<<blocks_for(total), kT, 0, s>>>(total, crow, cnt);
  GS_CUDA(gs::dev_malloc(&off_b.p, sizeof(uint64_t) * (V + 1)));
  uint64_t *off = off_b.as<uint64_t>();
  uint64_t nv = V;
  GS_CUDA(cudaMemcpyAsync(d_n, &nv, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  scan_u32(cnt, off, d_n, V, stmp, s, sms);
  GS_CUDA(cudaStreamSynchronize(s));
  GS_CUDA(cudaMemcpyAsync(d_n, &n, sizeof(uint64_t), cudaMemcpyHostToDevice, s));  // restore
  *off_out = off;
  *adj_out = adj;
  *row_out = crow;
  off_b.p = adj_b.p = crow_b.p = nullptr;
  *kept = total;
  return GS_OK;
}

}  // namespace gs

using namespace gs;

static gs_status build_graph(gs_graph *g, uint32_t V, uint64_t E, uint32_t T, uint32_t R, uint64_t nmax,
                             cudaStream_t s, int sms, DevBuf &ro, DevBuf &col, DevBuf &rel, DevBuf &vt, DevBuf &k0,
                             DevBuf &v0, DevBuf &k1, DevBuf &v1, DevBuf &scanb, DevBuf &tmpb, DevBuf &stmpb,
                             DevBuf &dn);

extern "C" gs_status gs_graph_load(const gs_graph_desc *desc, gs_graph **out) {
  if (!desc || !out) return fail(GS_ERR_INVALID, "gs_graph_load: null argument");
  *out = nullptr;
  const uint32_t V = desc->num_vertices;
  const uint64_t E = desc->num_edges;
  if (V == 0 || V > (1u << kNbrBits)) return fail(GS_ERR_INVALID, "num_vertices must be in [1, 2^24]");
  if (desc->num_types == 0 || desc->num_types > 256) return fail(GS_ERR_INVALID, "num_types must be in [1, 256]");
  if (desc->num_rels == 0 || desc->num_rels > 255) return fail(GS_ERR_INVALID, "num_rels must be in [1, 255]");
  if (E >= (1ull << 32)) return fail(GS_ERR_UNSUPPORTED, "num_edges must be < 2^32");
  if (!desc->row_offsets || !desc->vertex_type || (E && (!desc->col_targets || !desc->edge_rel)))
    return fail(GS_ERR_INVALID, "gs_graph_load: null array");
  cudaStream_t s = static_cast<cudaStream_t>(desc->cuda_stream);
  int dev = 0, sms = 0;
  GS_CUDA(cudaGetDevice(&dev));
  GS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const bool on_dev = desc->flags & GS_DEVICE_PTRS;
  const uint32_t T = desc->num_types, R = desc->num_rels;
  const uint64_t En = E ? E : 1;

  DevBuf ro, col, rel, vt, k0, v0, k1, v1, scanb, tmpb, stmpb, dn, err;
  GS_CUDA(gs::dev_malloc(&ro.p, sizeof(uint64_t) * (V + 1)));
  GS_CUDA(gs::dev_malloc(&col.p, sizeof(uint32_t) * En));
  GS_CUDA(gs::dev_malloc(&rel.p, sizeof(uint32_t) * En));
  GS_CUDA(gs::dev_malloc(&vt.p, sizeof(uint32_t) * V));
  cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  GS_CUDA(cudaMemcpyAsync(ro.p, desc->row_offsets, sizeof(uint64_t) * (V + 1), kind, s));
  if (E) {
    GS_CUDA(cudaMemcpyAsync(col.p, desc->col_targets, sizeof(uint32_t) * E, kind, s));
    GS_CUDA(cudaMemcpyAsync(rel.p, desc->edge_rel, sizeof(uint32_t) * E, kind, s));
  }
  GS_CUDA(cudaMemcpyAsync(vt.p, desc->vertex_type, sizeof(uint32_t) * V, kind, s));
  GS_CUDA(gs::dev_malloc(&err.p, sizeof(uint32_t)));
  GS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(uint32_t), s));
  k_validate<<<blocks_for(V > E ? V : E), kT, 0, s>>>(V, E, ro.as<uint64_t>(), col.as<uint32_t>(), rel.as<uint32_t>(),
                                                       vt.as<uint32_t>(), T, R, err.as<uint32_t>());
  uint32_t herr = 0;
  GS_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  if (herr & 1) return fail(GS_ERR_INVALID, "row_offsets must start at 0, be non-decreasing and end at num_edges");
  if (herr & 2) return fail(GS_ERR_INVALID, "col_targets holds an id >= num_vertices");
  if (herr & 4) return fail(GS_ERR_INVALID, "edge_rel holds a relation >= num_rels");
  if (herr & 8) return fail(GS_ERR_INVALID, "vertex_type holds a type >= num_types");

  const uint64_t nmax = En > V + 1 ? En : V + 1;
  GS_CUDA(gs::dev_malloc(&k0.p, sizeof(uint32_t) * nmax));
  GS_CUDA(gs::dev_malloc(&v0.p, sizeof(uint32_t) * nmax));
  GS_CUDA(gs::dev_malloc(&k1.p, sizeof(uint32_t) * nmax));
  GS_CUDA(gs::dev_malloc(&v1.p, sizeof(uint32_t) * nmax));
  GS_CUDA(gs::dev_malloc(&scanb.p, sizeof(uint64_t) * (nmax + 1)));
  uint64_t tw = radix_tmp_words(nmax);
  uint64_t sw = scan_tmp_words(nmax);
  GS_CUDA(gs::dev_malloc(&tmpb.p, sizeof(uint64_t) * tw));   // radix sort scratch
  GS_CUDA(gs::dev_malloc(&stmpb.p, sizeof(uint64_t) * sw));  // scan scratch
  GS_CUDA(cudaMemsetAsync(tmpb.p, 0, sizeof(uint64_t) * tw, s));
  GS_CUDA(cudaMemsetAsync(stmpb.p, 0, sizeof(uint64_t) * sw, s));
  GS_CUDA(gs::dev_malloc(&dn.p, sizeof(uint64_t)));
  GS_CUDA(cudaMemcpyAsync(dn.p, &E, sizeof(uint64_t), cudaMemcpyHostToDevice, s));

  gs_graph *g = new gs_graph();
  memset(g, 0, sizeof(*g));
  g->device = dev;
  g->num_sms = sms;
  gs_status st = build_graph(g, V, E, T, R, nmax, s, sms, ro, col, rel, vt, k0, v0, k1, v1, scanb, tmpb, stmpb, dn);
  if (st != GS_OK) {
    gs_graph_free(g);  // frees whatever the build had attached to g
    return st;
  }
  *out = g;
  return GS_OK;
}

// Tables derived from the signature planes and neighbour-type masks: the
// same planes in type-list order (sig_t, tmask_t; needs the type lists) and
// the signature statistics of the plan, sigge[(t * P + p) * 16 + c] =
// vertices of type t (t = T: any type) whose count in plane p is at least c.
// With alloc the three arrays are allocated (graph load), else rewritten in
// place (after the signatures were replaced).
static gs_status derive_sig_tables(gs_graph *g, uint32_t V, uint32_t T, uint64_t P, uint64_t sig_words, cudaStream_t s,
                                   bool alloc) {
  if (alloc && (gs::dev_malloc(&g->sig_t, sizeof(uint32_t) * sig_words * P) != cudaSuccess ||
                gs::dev_malloc(&g->tmask_t, sizeof(uint32_t) * (uint64_t)V * P) != cudaSuccess))
    return fail(GS_ERR_OOM, "type-ordered planes");
  GS_CUDA(cudaMemsetAsync(g->sig_t, 0, sizeof(uint32_t) * sig_words * P, s));
  k_type_order<<<blocks_for((V + 7) / 8 * P), kT, 0, s>>>(V, (uint32_t)P, g->tvid, g->sig, sig_words, g->tmask,
                                                         g->sig_t, g->tmask_t);
  const uint64_t nh = (uint64_t)(T + 1) * P * 16;
  DevBuf dh_b;
  GS_CUDA(gs::dev_malloc(&dh_b.p, sizeof(uint32_t) * nh));
  uint32_t *dh = dh_b.as<uint32_t>();
  GS_CUDA(cudaMemsetAsync(dh, 0, sizeof(uint32_t) * nh, s));
  const dim3 grid((unsigned)std::min<uint64_t>((V + 255) / 256, 64), (unsigned)P);
  k_sig_hist<<<grid, 256, 0, s>>>(V, T, (uint32_t)P, g->vtype, g->sig, sig_words, dh);
  std::vector<uint32_t> hh(nh);
  GS_CUDA(cudaMemcpyAsync(hh.data(), dh, sizeof(uint32_t) * nh, cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  for (uint64_t row = 0; row < (uint64_t)(T + 1) * P; ++row)
    for (int c = 14; c >= 0; --c) hh[row * 16 + c] += hh[row * 16 + c + 1];
  if (alloc && gs::dev_malloc(&g->sigge, sizeof(uint32_t) * nh) != cudaSuccess)
    return fail(GS_ERR_OOM, "signature statistics");
  if (!g->sigge_host) g->sigge_host = new uint32_t[nh];
  memcpy(g->sigge_host, hh.data(), sizeof(uint32_t) * nh);
  GS_CUDA(cudaMemcpyAsync(g->sigge, hh.data(), sizeof(uint32_t) * nh, cudaMemcpyHostToDevice, s));
  GS_CUDA(cudaStreamSynchronize(s));
  return GS_OK;
}

gs_status gs::graph_set_signatures(gs_graph *g, const uint8_t *counts) {
  const DevGraph &d = g->d;
  const uint64_t P = 2ull * d.R + 2, V = d.V;
  std::vector<uint32_t> words(P * d.sig_words, 0);
  for (uint64_t p = 0; p < P; ++p)
    for (uint64_t v = 0; v < V; ++v) {
      const uint32_t c = counts[p * V + v] > 15 ? 15u : counts[p * V + v];
      words[p * d.sig_words + (v >> 3)] |= c << ((v & 7) * 4);
    }
  GS_CUDA(cudaMemcpy(g->sig, words.data(), sizeof(uint32_t) * words.size(), cudaMemcpyHostToDevice));
  return derive_sig_tables(g, d.V, d.T, P, d.sig_words, nullptr, false);
}

// Everything after the inputs are validated and the work buffers exist:
// on an error return, g holds only buffers gs_graph_free releases, and every
// temporary is released here.
static gs_status build_graph(gs_graph *g, uint32_t V, uint64_t E, uint32_t T, uint32_t R, uint64_t nmax,
                             cudaStream_t s, int sms, DevBuf &ro, DevBuf &col, DevBuf &rel, DevBuf &vt, DevBuf &k0,
                             DevBuf &v0, DevBuf &k1, DevBuf &v1, DevBuf &scanb, DevBuf &tmpb, DevBuf &stmpb,
                             DevBuf &dn) {
  auto cleanup = [](gs_status st) { return st; };
  k_expand<<<blocks_for(V), kT, 0, s>>>(V, ro.as<uint64_t>(), col.as<uint32_t>(), rel.as<uint32_t>(), k0.as<uint32_t>(),
                                        v0.as<uint32_t>());
  DevBuf src_rows_b, dst_rows_b;
  uint32_t *src_rows = nullptr;
  uint64_t kept = 0;
  gs_status st = build_direction(V, R, E, k0.as<uint32_t>(), v0.as<uint32_t>(), k1.as<uint32_t>(), v1.as<uint32_t>(),
                                 scanb.as<uint64_t>(), tmpb.as<uint64_t>(), stmpb.as<uint64_t>(), dn.as<uint64_t>(), s, sms, &g->off_out,
                                 &g->adj_out, &src_rows, &kept);
  src_rows_b.p = src_rows;
  if (st != GS_OK) return cleanup(st);
  // incoming direction from the kept triples
  GS_CUDA(cudaMemcpyAsync(dn.p, &kept, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  k_rekey_in<<<blocks_for(kept), kT, 0, s>>>(kept, src_rows, g->adj_out, k0.as<uint32_t>(), v0.as<uint32_t>());
  uint32_t *dst_rows = nullptr;
  uint64_t kept_in = 0;
  st = build_direction(V, R, kept, k0.as<uint32_t>(), v0.as<uint32_t>(), k1.as<uint32_t>(), v1.as<uint32_t>(),
                       scanb.as<uint64_t>(), tmpb.as<uint64_t>(), stmpb.as<uint64_t>(), dn.as<uint64_t>(), s, sms, &g->off_in, &g->adj_in,
                       &dst_rows, &kept_in);
  dst_rows_b.p = dst_rows;
  // distinct neighbours over all relations, per direction
  for (int d = 0; d < 2 && st == GS_OK; ++d) {
    const uint64_t n = d == 0 ? kept : kept_in;
    GS_CUDA(cudaMemcpyAsync(dn.p, &n, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    k_strip_rel<<<blocks_for(n), kT, 0, s>>>(n, d == 0 ? g->adj_out : g->adj_in, d == 0 ? src_rows : dst_rows,
                                             k0.as<uint32_t>(), v0.as<uint32_t>());
    uint32_t *rows = nullptr;
    uint64_t kept_any = 0;
    st = build_direction(V, 1, n, k0.as<uint32_t>(), v0.as<uint32_t>(), k1.as<uint32_t>(), v1.as<uint32_t>(),
                         scanb.as<uint64_t>(), tmpb.as<uint64_t>(), stmpb.as<uint64_t>(), dn.as<uint64_t>(), s, sms,
                         d == 0 ? &g->off_aout : &g->off_ain, d == 0 ? &g->adj_aout : &g->adj_ain, &rows, &kept_any);
    cudaFree(rows);
  }
  if (st != GS_OK) return cleanup(st);
  const uint64_t P = 2ull * R + 2;  // signature / mask planes

  // Planes hold whole 16-byte groups (32 vertices) so the filter can read
  // them as aligned uint4 vectors up to the last partial group.
  const uint64_t sig_words = ((V + 7) / 8 + 3) / 4 * 4;
  if (gs::dev_malloc(&g->sig, sizeof(uint32_t) * sig_words * P) != cudaSuccess)
    return cleanup(fail(GS_ERR_OOM, "signature planes"));
  GS_CUDA(cudaMemsetAsync(g->sig, 0, sizeof(uint32_t) * sig_words * P, s));
  k_signatures<<<blocks_for(V), kT, 0, s>>>(V, g->off_out, g->adj_out, 0, g->sig, sig_words);
  k_signatures<<<blocks_for(V), kT, 0, s>>>(V, g->off_in, g->adj_in, R, g->sig, sig_words);
  k_signatures<<<blocks_for(V), kT, 0, s>>>(V, g->off_aout, g->adj_aout, 2 * R, g->sig, sig_words);
  k_signatures<<<blocks_for(V), kT, 0, s>>>(V, g->off_ain, g->adj_ain, 2 * R + 1, g->sig, sig_words);
  const uint64_t vt_bytes = ((uint64_t)V + 127) / 128 * 128;  // whole 32-vertex groups, zero padded
  if (gs::dev_malloc(&g->vtype, vt_bytes) != cudaSuccess) return cleanup(fail(GS_ERR_OOM, "types"));
  GS_CUDA(cudaMemsetAsync(g->vtype, 0, vt_bytes, s));
  DevBuf hist_b;
  GS_CUDA(gs::dev_malloc(&hist_b.p, sizeof(uint32_t) * T));
  uint32_t *hist = hist_b.as<uint32_t>();
  GS_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * T, s));
  k_types<<<blocks_for(V), kT, 0, s>>>(V, vt.as<uint32_t>(), g->vtype, hist);
  g->type_count = new uint32_t[T];
  GS_CUDA(cudaMemcpyAsync(g->type_count, hist, sizeof(uint32_t) * T, cudaMemcpyDeviceToHost, s));
  // content hash for the tuning cache: sizes plus a sample of rows
  std::vector<uint32_t> sample(1024, 0);
  uint64_t ns = kept < 1024 ? kept : 1024;
  if (ns) GS_CUDA(cudaMemcpyAsync(sample.data(), g->adj_out + (kept - ns), ns * 4, cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  // Vertices grouped by type (stable radix sort of (type, id) pairs keeps
  // the ids ascending within a type); run starts from the type counts.
  {
    std::vector<uint32_t> toff(T + 1, 0);
    for (uint32_t t = 0; t < T; ++t) toff[t + 1] = toff[t] + g->type_count[t];
    if (gs::dev_malloc(&g->toff, sizeof(uint32_t) * (T + 1)) != cudaSuccess ||
        gs::dev_malloc(&g->tvid, sizeof(uint32_t) * V) != cudaSuccess)
      return cleanup(fail(GS_ERR_OOM, "type lists"));
    GS_CUDA(cudaMemcpyAsync(g->toff, toff.data(), sizeof(uint32_t) * (T + 1), cudaMemcpyHostToDevice, s));
    uint64_t nv = V;
    GS_CUDA(cudaMemcpyAsync(dn.p, &nv, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    GS_CUDA(cudaMemcpyAsync(k0.p, vt.p, sizeof(uint32_t) * V, cudaMemcpyDeviceToDevice, s));
    k_iota<<<blocks_for(V), kT, 0, s>>>(V, v0.as<uint32_t>());
    int tb = 1;
    while (tb < 8 && ((T - 1) >> tb)) ++tb;
    const int res = radix_sort_pairs(k0.as<uint32_t>(), v0.as<uint32_t>(), k1.as<uint32_t>(), v1.as<uint32_t>(),
                                     dn.as<uint64_t>(), nmax, 0, tb, tmpb.as<uint64_t>(), s, sms);
    GS_CUDA(cudaMemcpyAsync(g->tvid, res ? v1.p : v0.p, sizeof(uint32_t) * V, cudaMemcpyDeviceToDevice, s));
    GS_CUDA(cudaStreamSynchronize(s));
  }
  // neighbour-type masks (zero where a vertex has no neighbour in a plane)
  if (gs::dev_malloc(&g->tmask, sizeof(uint32_t) * (uint64_t)V * P) != cudaSuccess)
    return cleanup(fail(GS_ERR_OOM, "neighbour-type masks"));
  GS_CUDA(cudaMemsetAsync(g->tmask, 0, sizeof(uint32_t) * (uint64_t)V * P, s));
  k_type_masks<<<blocks_for(V), kT, 0, s>>>(V, g->off_out, g->adj_out, 0, g->vtype, g->tmask);
  k_type_masks<<<blocks_for(V), kT, 0, s>>>(V, g->off_in, g->adj_in, R, g->vtype, g->tmask);
  k_type_masks<<<blocks_for(V), kT, 0, s>>>(V, g->off_aout, g->adj_aout, 2 * R, g->vtype, g->tmask);
  k_type_masks<<<blocks_for(V), kT, 0, s>>>(V, g->off_ain, g->adj_ain, 2 * R + 1, g->vtype, g->tmask);
  st = derive_sig_tables(g, V, T, P, sig_words, s, true);
  if (st != GS_OK) return cleanup(st);
  uint64_t h = 1469598103934665603ull;
  auto mixin = [&](uint64_t x) { h = (h ^ x) * 1099511628211ull; };
  mixin(V); mixin(kept); mixin(T); mixin(R);
  for (uint64_t i = 0; i < ns; ++i) mixin(sample[i]);
  g->hash = h;

  DevGraph &d = g->d;
  d.V = V; d.T = T; d.R = R; d.E = kept;
  d.off[0] = g->off_out; d.off[1] = g->off_in; d.off[2] = g->off_aout; d.off[3] = g->off_ain;
  d.adj[0] = g->adj_out; d.adj[1] = g->adj_in; d.adj[2] = g->adj_aout; d.adj[3] = g->adj_ain;
  d.vtype = g->vtype;
  d.tvid = g->tvid;
  d.toff = g->toff;
  d.sigge = g->sigge;
  d.tmask = g->tmask;
  d.sig_t = g->sig_t;
  d.tmask_t = g->tmask_t;
  d.sig = g->sig;
  d.sig_words = sig_words;
  d.W0 = (V + 31) / 32;
  d.W1 = (d.W0 + 31) / 32;
  d.nchunks = (d.W1 + 31) / 32;
  d.ipg = (d.nchunks + 31) / 32;
  d.idbits = 1;
  while (d.idbits < 32 && ((V - 1) >> d.idbits)) ++d.idbits;
  return GS_OK;
}

extern "C" void gs_graph_free(gs_graph *g) {
  if (!g) return;
  gs::release_cache(g);
  gs::release_fallback(g);
  gs::release_khop(g);
  cudaFree(g->off_out);
  cudaFree(g->off_in);
  cudaFree(g->adj_out);
  cudaFree(g->adj_in);
  cudaFree(g->off_aout);
  cudaFree(g->off_ain);
  cudaFree(g->adj_aout);
  cudaFree(g->adj_ain);
  cudaFree(g->vtype);
  cudaFree(g->tvid);
  cudaFree(g->toff);
  cudaFree(g->sigge);
  cudaFree(g->tmask);
  cudaFree(g->sig_t);
  cudaFree(g->tmask_t);
  cudaFree(g->sig);
  delete[] g->type_count;
  delete[] g->sigge_host;
  delete g;
}

extern "C" uint64_t gs_graph_num_edges(const gs_graph *g) { return g ? g->d.E : 0; }

extern "C" gs_status gs_graph_export(const gs_graph *g, uint32_t plane, uint64_t *off, uint32_t *adj, uint64_t *n,
                                     uint8_t *sig) {
  if (!g || plane > 3 || !off || !n) return fail(GS_ERR_INVALID, "gs_graph_export: bad argument");
  GS_CUDA(cudaSetDevice(g->device));
  const uint64_t V = g->d.V;
  GS_CUDA(cudaMemcpy(off, g->d.off[plane], sizeof(uint64_t) * (V + 1), cudaMemcpyDeviceToHost));
  *n = off[V];
  if (adj && off[V]) GS_CUDA(cudaMemcpy(adj, g->d.adj[plane], sizeof(uint32_t) * off[V], cudaMemcpyDeviceToHost));
  if (sig) {
    const uint64_t P = 2ull * g->d.R + 2;
    std::vector<uint32_t> words(P * g->d.sig_words);
    GS_CUDA(cudaMemcpy(words.data(), g->d.sig, sizeof(uint32_t) * words.size(), cudaMemcpyDeviceToHost));
    for (uint64_t p = 0; p < P; ++p)
      for (uint64_t v = 0; v < V; ++v) sig[p * V + v] = (words[p * g->d.sig_words + (v >> 3)] >> ((v & 7) * 4)) & 15u;
  }
  return GS_OK;
}

extern "C" const char *gs_last_error(void) { return gs::t_last_error.c_str(); }
