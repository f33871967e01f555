// Candidate filter for one query vertex that allocates no memory.
//
// Some callers cannot let this library allocate: a serving process that
// reserved its whole device memory budget at start-up, or a caller whose own
// allocator owns the device, must not see cudaMalloc/cudaFree (both can also
// stall the whole device while they run).  For them this entry point does
// the filtering step (binding, type and per-direction, per-relation degree
// test over every data vertex) and compacts the result into the caller's
// output buffer, using only a fixed scratch area compiled into the library.
//
// Scratch: one array in device memory, kStaticScratchBytes long, shared by
// every call on a device and kept until the process exits.  It holds one
// count per 1,024-vertex chunk and the chunk offsets, so it bounds the graph
// size to kStaticMaxVertices.  Calls that overlap on the GPU (two streams,
// or two threads) race on it; callers serialise them.  Every scratch word a
// call reads is written earlier in that call, so nothing needs clearing.
#include <cstring>
#include <mutex>

#include "gs_host.h"

using namespace gs;

namespace {

constexpr uint32_t kStaticMaxVertices = 1u << 24;
constexpr uint32_t kStaticChunk = 1024;  // vertices per count
constexpr uint32_t kStaticMaxChunks = kStaticMaxVertices / kStaticChunk;
constexpr size_t kStaticScratchBytes = sizeof(uint32_t) * kStaticMaxChunks + sizeof(uint64_t) * (kStaticMaxChunks + 1);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// The test one query vertex applies, passed by value.
struct VertexTest {
  uint32_t type, bind, nneeds;
  uint16_t plane[2 * kMaxM];
  uint8_t cnt[2 * kMaxM];
};

// One 32-vertex word of the candidate test (bit j = vertex v0 + j passes).
__device__ __forceinline__ uint32_t test_word(const DevGraph &G, const VertexTest &t, uint32_t w0) {
  const uint32_t v0 = w0 * 32;
  if (v0 >= G.V) return 0;
  uint32_t ok = 0xFFFFFFFFu;
  if (t.bind != kUnbound) {
    ok = (t.bind >= v0 && t.bind < v0 + 32) ? (1u << (t.bind - v0)) : 0u;
  }
  if (ok && t.type != kAny) {
    uint32_t m = 0;
    for (int j = 0; j < 32; ++j) m |= (G.vtype[v0 + j] == t.type ? 1u : 0u) << j;
    ok &= m;
  }
  for (uint32_t i = 0; i < t.nneeds && ok; ++i) {
    const uint32_t *p = G.sig + (uint64_t)t.plane[i] * G.sig_words + (uint64_t)w0 * 4;
    uint32_t m = 0;
    for (int j = 0; j < 32; ++j) m |= (((p[j >> 3] >> ((j & 7) * 4)) & 15u) >= t.cnt[i] ? 1u : 0u) << j;
    ok &= m;
  }
  if (v0 + 32 > G.V) ok &= (1u << (G.V - v0)) - 1;
  return ok;
}

// Pass 1: candidates per chunk (one warp per 1,024-vertex chunk).
__global__ void k_static_count(DevGraph G, VertexTest t, uint32_t *counts, uint32_t nchunks) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * blockDim.x / 32;
  for (uint64_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; c < nchunks; c += warps) {
    uint32_t n = __popc(test_word(G, t, (uint32_t)c * 32 + lane));
    for (int o = 16; o; o >>= 1) n += __shfl_down_sync(0xFFFFFFFFu, n, o);
    if (lane == 0) counts[c] = n;
  }
}

// Pass 2 (one block): exclusive scan of the chunk counts; total to *d_count.
__global__ void k_static_scan(const uint32_t *counts, uint64_t *offs, uint32_t nchunks, uint64_t *d_count) {
  __shared__ uint64_t warp_tot[32];
  __shared__ uint64_t carry;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < nchunks; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint64_t v = i < nchunks ? counts[i] : 0;
    uint64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = lane < blockDim.x / 32 ? warp_tot[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
        if (lane >= o) w += y;
      }
      warp_tot[lane] = w;
    }
    __syncthreads();
    if (i < nchunks) offs[i] = carry + (warp ? warp_tot[warp - 1] : 0) + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[blockDim.x / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    offs[nchunks] = carry;
    *d_count = carry;
  }
}

// Pass 3: ids in ascending order; ids past cap_ids are not written.
__global__ void k_static_write(DevGraph G, VertexTest t, const uint64_t *offs, uint32_t nchunks, uint32_t *ids,
                               uint64_t cap_ids) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * blockDim.x / 32;
  for (uint64_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; c < nchunks; c += warps) {
    const uint32_t w0 = (uint32_t)c * 32 + lane;
    uint32_t x = test_word(G, t, w0);
    uint32_t n = __popc(x), incl = n;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    uint64_t p = offs[c] + incl - n;
    while (x) {
      const int b = __ffs(x) - 1;
      x &= x - 1;
      if (p < cap_ids) ids[p] = w0 * 32 + b;
      ++p;
    }
  }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_static_mu;
void *g_static_ptr[256];

gs_status static_scratch(void **out) {
  int dev = 0;
  GS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(GS_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (static filter scratch)");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return GS_OK;
}

}  // namespace

extern "C" gs_status gs_filter_candidates_static(gs_graph *g, const gs_query *q, uint32_t u, uint32_t *d_ids,
                                                 uint64_t cap_ids, uint64_t *d_count, void *cuda_stream) {
  if (!g || !q || !d_count || (cap_ids && !d_ids))
    return fail(GS_ERR_INVALID, "gs_filter_candidates_static: null argument");
  if (g->d.V > kStaticMaxVertices)
    return fail(GS_ERR_INVALID, "gs_filter_candidates_static: the graph has more than 2^24 vertices, the most its "
                                "fixed scratch covers");
  DQuery d;
  gs_status st = pack_query(g->d, q, nullptr, &d);
  if (st != GS_OK) return st;
  if (u >= d.k) return fail(GS_ERR_INVALID, "gs_filter_candidates_static: query vertex out of range");
  GS_CUDA(cudaSetDevice(g->device));
  void *scratch = nullptr;
  if ((st = static_scratch(&scratch)) != GS_OK) return st;
  VertexTest t;
  memset(&t, 0, sizeof(t));
  t.type = d.vtype[u];
  t.bind = d.vbind[u];
  t.nneeds = d.need_begin[u + 1] - d.need_begin[u];
  for (uint32_t i = 0; i < t.nneeds; ++i) {
    t.plane[i] = d.need_plane[d.need_begin[u] + i];
    t.cnt[i] = d.need_cnt[d.need_begin[u] + i];
  }
  const uint32_t nchunks = (g->d.V + kStaticChunk - 1) / kStaticChunk;
  uint32_t *counts = static_cast<uint32_t *>(scratch);
  uint64_t *offs = reinterpret_cast<uint64_t *>(static_cast<unsigned char *>(scratch) +
                                                sizeof(uint32_t) * kStaticMaxChunks);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const unsigned grid = (unsigned)std::min<uint64_t>((nchunks + 7) / 8, (uint64_t)g->num_sms * 8);
  k_static_count<<<grid, 256, 0, s>>>(g->d, t, counts, nchunks);
  k_static_scan<<<1, 1024, 0, s>>>(counts, offs, nchunks, d_count);
  k_static_write<<<grid, 256, 0, s>>>(g->d, t, offs, nchunks, d_ids, cap_ids);
  GS_CUDA(cudaGetLastError());
  return GS_OK;
}
