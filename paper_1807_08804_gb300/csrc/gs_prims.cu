// Device primitives: exclusive scan (the prefix-sum step of the two-step
// output scheme, Section 3.3.4, and of stream compaction, Section 3.3.3
// "kernel_collect") and a stable LSD radix sort (graph canonicalisation and
// the final ordering of embeddings).
//
// Sizes are read from device memory so that a whole pipeline can be captured
// once in a CUDA graph and replayed: each kernel is persistent over tiles and
// learns how many tiles exist from *d_n.
#include <algorithm>

#include "gs_internal.h"

namespace gs {

namespace {

constexpr int kScanThreads = 256;
constexpr uint64_t kScanMaxTiles = 8192;

// Tile of the scan: 1,024 items while that gives at most 8,192 tiles (short
// serial chains for the small scans of the pipeline), larger beyond.  Every
// kernel of one scan derives it from the same n.
__device__ __forceinline__ uint64_t scan_rounds(uint64_t n) {
  uint64_t r = (n + kScanThreads * kScanMaxTiles - 1) / (kScanThreads * kScanMaxTiles);
  return r < 4 ? 4 : r;
}

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixRounds = 4;
constexpr uint64_t kRadixTile = kRadixThreads * kRadixRounds;  // 1024
constexpr int kRadixBins = 256;

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *total, uint64_t *smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < kScanThreads / 32 ? smem[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) smem[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  uint64_t before = warp ? smem[warp - 1] : 0;
  *total = smem[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T *in, const uint64_t *d_n, uint64_t *tile_sums) {
  __shared__ uint64_t red[kScanThreads / 32];
  const uint64_t n = *d_n;
  const uint64_t rounds = scan_rounds(n), tile = rounds * kScanThreads;
  const uint64_t ntiles = (n + tile - 1) / tile;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint64_t s = 0;
    const uint64_t base = t * tile;
#pragma unroll 4
    for (uint64_t j = 0; j < rounds; ++j) {
      uint64_t i = base + (uint64_t)j * kScanThreads + threadIdx.x;
      if (i < n) s += (uint64_t)in[i];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t tot = 0;
      for (int w = 0; w < kScanThreads / 32; ++w) tot += red[w];
      tile_sums[t] = tot;
    }
    __syncthreads();
  }
}

// One block: exclusive scan of the tile sums in place; out[n] = grand total.
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(uint64_t *tile_sums, const uint64_t *d_n, uint64_t *out) {
  __shared__ uint64_t smem[kScanThreads / 32];
  const uint64_t n = *d_n;
  const uint64_t tile = scan_rounds(n) * kScanThreads;
  const uint64_t ntiles = (n + tile - 1) / tile;
  uint64_t carry = 0;
  for (uint64_t base = 0; base < ntiles; base += kScanThreads) {
    uint64_t i = base + threadIdx.x;
    uint64_t v = i < ntiles ? tile_sums[i] : 0, tot;
    uint64_t ex = block_exclusive_scan(v, &tot, smem);
    if (i < ntiles) tile_sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) out[n] = carry;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const T *in, const uint64_t *d_n, const uint64_t *tile_sums,
                                                             uint64_t *out) {
  __shared__ uint64_t smem[kScanThreads / 32];
  const uint64_t n = *d_n;
  const uint64_t rounds = scan_rounds(n), tile = rounds * kScanThreads;
  const uint64_t ntiles = (n + tile - 1) / tile;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint64_t carry = tile_sums[t];
    const uint64_t base = t * tile;
    for (uint64_t j = 0; j < rounds; ++j) {
      uint64_t i = base + (uint64_t)j * kScanThreads + threadIdx.x;
      uint64_t v = i < n ? (uint64_t)in[i] : 0, tot;
      uint64_t ex = block_exclusive_scan(v, &tot, smem);
      if (i < n) out[i] = carry + ex;
      carry += tot;
    }
  }
}

template <typename T>
void scan_impl(const T *in, uint64_t *out, const uint64_t *d_n, uint64_t max_n, uint64_t *tmp, cudaStream_t s,
               int num_sms) {
  uint64_t tiles = std::min<uint64_t>((max_n + 1023) / 1024, kScanMaxTiles);
  unsigned grid = (unsigned)(tiles < (uint64_t)num_sms * 8 ? (tiles ? tiles : 1) : (uint64_t)num_sms * 8);
  k_scan_reduce<T><<<grid, kScanThreads, 0, s>>>(in, d_n, tmp);
  k_scan_partials<<<1, kScanThreads, 0, s>>>(tmp, d_n, out);
  k_scan_down<T><<<grid, kScanThreads, 0, s>>>(in, d_n, tmp, out);
}

// ------------------------------------------------------------ radix sort
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const uint32_t *keys, const uint64_t *d_n, int shift,
                                                               uint32_t *counts, uint64_t *d_len) {
  __shared__ uint32_t cnt[kRadixBins];
  const uint64_t n = *d_n;
  const uint64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
  if (blockIdx.x == 0 && threadIdx.x == 0) *d_len = (uint64_t)kRadixBins * ntiles;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = t * kRadixTile;
    for (int j = 0; j < kRadixRounds; ++j) {
      uint64_t i = base + (uint64_t)j * kRadixThreads + threadIdx.x;
      if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    counts[(uint64_t)threadIdx.x * ntiles + t] = cnt[threadIdx.x];
    __syncthreads();
  }
}

// Stable scatter: each warp ranks its 512 consecutive items in order with
// __match_any_sync, warps are ordered by an exclusive scan of their digit
// counts, and tiles by the digit-major global scan of the histograms.
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(const uint32_t *kin, const uint32_t *vin,
                                                                  uint32_t *kout, uint32_t *vout,
                                                                  const uint64_t *d_n, int shift,
                                                                  const uint64_t *offs) {
  __shared__ uint32_t wcnt[kRadixWarps][kRadixBins];
  __shared__ uint64_t goff[kRadixBins];
  const uint64_t n = *d_n;
  const uint64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (int i = threadIdx.x; i < kRadixWarps * kRadixBins; i += kRadixThreads) (&wcnt[0][0])[i] = 0;
    goff[threadIdx.x] = offs[(uint64_t)threadIdx.x * ntiles + t];
    __syncthreads();
    uint32_t key[kRadixRounds], val[kRadixRounds], rank[kRadixRounds];
    const uint64_t base = t * kRadixTile + (uint64_t)warp * (kRadixRounds * 32);
#pragma unroll
    for (int j = 0; j < kRadixRounds; ++j) {
      uint64_t i = base + (uint64_t)j * 32 + lane;
      bool valid = i < n;
      key[j] = valid ? kin[i] : 0;
      val[j] = valid ? vin[i] : 0;
      uint32_t d = valid ? ((key[j] >> shift) & 0xFF) : (kRadixBins + lane);
      uint32_t peers = __match_any_sync(kFull, d);
      uint32_t before = valid ? wcnt[warp][d] : 0;
      __syncwarp();
      if (valid && (__ffs(peers) - 1) == lane) wcnt[warp][d] = before + __popc(peers);
      __syncwarp();
      rank[j] = valid ? before + __popc(peers & lt) : 0xFFFFFFFFu;
    }
    __syncthreads();
    {
      uint32_t run = 0;
      for (int w = 0; w < kRadixWarps; ++w) {
        uint32_t c = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = run;
        run += c;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRadixRounds; ++j) {
      if (rank[j] != 0xFFFFFFFFu) {
        uint32_t d = (key[j] >> shift) & 0xFF;
        uint64_t dst = goff[d] + wcnt[warp][d] + rank[j];
        kout[dst] = key[j];
        vout[dst] = val[j];
      }
    }
    __syncthreads();
  }
}

}  // namespace

uint64_t scan_tmp_words(uint64_t max_n) { return std::min<uint64_t>((max_n + 1023) / 1024, kScanMaxTiles) + 1; }

void scan_u32(const uint32_t *in, uint64_t *out, const uint64_t *d_n, uint64_t max_n, uint64_t *tmp, cudaStream_t s,
              int num_sms) {
  scan_impl<uint32_t>(in, out, d_n, max_n, tmp, s, num_sms);
}
void scan_u64(const uint64_t *in, uint64_t *out, const uint64_t *d_n, uint64_t max_n, uint64_t *tmp, cudaStream_t s,
              int num_sms) {
  scan_impl<uint64_t>(in, out, d_n, max_n, tmp, s, num_sms);
}

static uint64_t radix_tiles(uint64_t max_n) {
  uint64_t t = (max_n + kRadixTile - 1) / kRadixTile;
  return t ? t : 1;
}
uint64_t radix_tmp_words(uint64_t max_n) {
  uint64_t bins = (uint64_t)kRadixBins * radix_tiles(max_n);
  // counts (uint32, rounded to words) + offsets (bins+1) + scan tmp + length
  return (bins + 1) / 2 + (bins + 1) + scan_tmp_words(bins) + 1;
}
int radix_passes(int nbits) { return (nbits + 7) / 8; }

int radix_sort_pairs(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const uint64_t *d_n, uint64_t max_n,
                     int bit_lo, int nbits, uint64_t *tmp, cudaStream_t s, int num_sms) {
  const uint64_t bins = (uint64_t)kRadixBins * radix_tiles(max_n);
  uint32_t *counts = reinterpret_cast<uint32_t *>(tmp);
  uint64_t *offs = tmp + (bins + 1) / 2;
  uint64_t *stmp = offs + bins + 1;
  uint64_t *d_len = stmp + scan_tmp_words(bins);
  uint64_t tiles = radix_tiles(max_n);
  unsigned grid = (unsigned)(tiles < (uint64_t)num_sms * 4 ? tiles : (uint64_t)num_sms * 4);
  int cur = 0;
  uint32_t *ks[2] = {k0, k1}, *vs[2] = {v0, v1};
  for (int p = 0; p < radix_passes(nbits); ++p) {
    int shift = bit_lo + 8 * p;
    k_radix_hist<<<grid, kRadixThreads, 0, s>>>(ks[cur], d_n, shift, counts, d_len);
    scan_u32(counts, offs, d_len, bins, stmp, s, num_sms);
    k_radix_scatter<<<grid, kRadixThreads, 0, s>>>(ks[cur], vs[cur], ks[cur ^ 1], vs[cur ^ 1], d_n, shift, offs);
    cur ^= 1;
  }
  return cur;
}

}  // namespace gs
