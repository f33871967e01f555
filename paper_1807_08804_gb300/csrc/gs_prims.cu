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

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixRounds = 4;
constexpr uint64_t kRadixTile = kRadixThreads * kRadixRounds;  // 1024
constexpr int kRadixBins = 256;

// ------------------------------------------------------------ scan
// Single-pass exclusive scan with decoupled look-back (Merrill and Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016).
// Blocks claim tiles in order from an atomic counter; each publishes its
// tile's aggregate, then sums the aggregates of the tiles before it (a warp
// reads 32 predecessors at a time) until it meets one that has published
// its inclusive prefix, and publishes its own.  A block only waits on tiles
// claimed before its own, by blocks that are already running, so the waits
// end; each is bounded all the same and records an error when the bound is
// hit: a wait that gives up records the event in the scratch's error word
// and takes its prefix directly, as the sum of every input before its tile,
// so the scan's result stays exact either way.  Descriptors carry the scan's
// 62-bit epoch, so the scratch needs zeroing only once, when it is
// allocated; the last block to finish resets the tile counter and advances
// the epoch for the next scan on the same scratch.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;  // 2048
constexpr uint32_t kLookbackLimit = 1u << 22;

struct ScanState {  // the first 32 bytes of the scratch
  uint32_t err;       // a look-back wait hit its bound (kept until the host clears it)
  uint32_t tiles;     // next tile to claim
  uint32_t done;      // blocks finished
  uint32_t limit;     // polls before a look-back wait gives up (0 = kLookbackLimit); set by the host
  uint64_t epoch;     // scans completed on this scratch
  uint32_t withhold;  // test setting: tile 0 of a multi-tile scan publishes nothing
  uint32_t pad;
};
struct __align__(32) ScanDesc {
  uint64_t agg;   // the tile's total
  uint64_t incl;  // prefix through the tile
  uint64_t flag;  // (epoch << 2) | 1 (aggregate) or 2 (inclusive)
  uint64_t pad;
};
static_assert(sizeof(ScanState) == 32 && sizeof(ScanDesc) == 32, "scan scratch layout");

__device__ __forceinline__ uint64_t block_scan_excl(uint64_t v, uint64_t *total, uint64_t *smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < kScanThreads / 32 ? smem[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) smem[lane] = w;
  }
  __syncthreads();
  const uint64_t before = warp ? smem[warp - 1] : 0;
  *total = smem[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan(const T *in, const uint64_t *d_n, uint64_t *out, ScanState *st,
                                                        ScanDesc *desc) {
  gdc_wait();
  __shared__ uint64_t vals[kScanTile];
  __shared__ uint64_t red[kScanThreads / 32];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_prefix;
  const uint64_t n = *d_n;
  const uint64_t ntiles = (n + kScanTile - 1) / kScanTile;
  const uint64_t tag = *reinterpret_cast<volatile uint64_t *>(&st->epoch) << 2;
  const uint32_t limit = st->limit ? st->limit : kLookbackLimit;
  const bool withhold = st->withhold != 0 && ntiles > 1;
  const int lane = threadIdx.x & 31;
  if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&st->tiles, 1u);
    __syncthreads();
    const uint64_t t = s_tile;
    if (t >= ntiles) break;  // block-uniform
    const uint64_t base = t * kScanTile;
    // striped loads (coalesced), then each thread owns 8 consecutive items
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      const uint64_t i = base + (uint64_t)j * kScanThreads + threadIdx.x;
      vals[j * kScanThreads + threadIdx.x] = i < n ? (uint64_t)in[i] : 0;
    }
    __syncthreads();
    uint64_t loc[kScanItems], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      loc[j] = sum;
      sum += vals[threadIdx.x * kScanItems + j];
    }
    uint64_t agg;
    const uint64_t ex = block_scan_excl(sum, &agg, red);
    if (threadIdx.x == 0) {
      ScanDesc &d = desc[t];
      if (t == 0) {
        if (!withhold) {
          __stcg(&d.incl, agg);
          __threadfence();
          __stcg(&d.flag, tag | 2u);
        }
      } else {
        __stcg(&d.agg, agg);
        __threadfence();
        __stcg(&d.flag, tag | 1u);
      }
    }
    if (threadIdx.x < 32) {  // look-back
      uint64_t prefix = 0;
      if (t > 0) {
        int64_t pos = (int64_t)t - 1;
        uint32_t spins = 0;
        for (;;) {
          const int64_t p = pos - lane;
          uint32_t status = 2;  // before tile 0: an inclusive prefix of 0
          if (p >= 0) {
            const uint64_t f = __ldcg(&desc[p].flag);
            status = (f & ~3ull) == tag ? (uint32_t)(f & 3u) : 0u;
          }
          const uint32_t incl_mask = __ballot_sync(kFull, status == 2);
          const uint32_t zero_mask = __ballot_sync(kFull, status == 0);
          const int first = incl_mask ? __ffs(incl_mask) - 1 : 32;
          const uint32_t need = first >= 31 ? kFull : ((2u << first) - 1);
          if ((zero_mask & need) && ++spins < limit) continue;
          if (zero_mask & need) {  // bound hit: record it, then sum the inputs before this tile
            if (lane == 0) atomicExch(&st->err, 1u);
            uint64_t v = 0;
            for (uint64_t i = lane; i < base; i += 32) v += (uint64_t)in[i];
#pragma unroll
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            prefix = v;
            break;
          }
          __threadfence();
          uint64_t v = 0;
          if (p >= 0 && status != 0 && lane <= first) v = lane < first ? __ldcg(&desc[p].agg) : __ldcg(&desc[p].incl);
#pragma unroll
          for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
          prefix += v;
          if (first < 32) break;
          pos -= 32;
        }
        if (lane == 0) {
          ScanDesc &d = desc[t];
          __stcg(&d.incl, prefix + agg);
          __threadfence();
          __stcg(&d.flag, tag | 2u);
        }
      }
      if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    const uint64_t pre = s_prefix + ex;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) vals[threadIdx.x * kScanItems + j] = pre + loc[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      const uint64_t i = base + (uint64_t)j * kScanThreads + threadIdx.x;
      if (i < n) out[i] = vals[j * kScanThreads + threadIdx.x];
    }
    if (t == ntiles - 1 && threadIdx.x == 0) out[n] = s_prefix + agg;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&st->done, 1u) == gridDim.x - 1) {  // every block has stopped claiming tiles
      st->tiles = 0;
      st->done = 0;
      st->epoch = (tag >> 2) + 1;
      __threadfence();
    }
  }
}

int scan_resident(const void *fn) {
  static int cached[2] = {0, 0};
  const int slot = fn == (const void *)k_scan<uint32_t> ? 0 : 1;
  if (!cached[slot]) {
    int r = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, fn, kScanThreads, 0) != cudaSuccess || r < 1) {
      cudaGetLastError();
      r = 1;
    }
    cached[slot] = r;
  }
  return cached[slot];
}

template <typename T>
void scan_impl(const T *in, uint64_t *out, const uint64_t *d_n, uint64_t max_n, uint64_t *tmp, cudaStream_t s,
               int num_sms) {
  const uint64_t tiles = std::max<uint64_t>((max_n + kScanTile - 1) / kScanTile, 1);
  // at most two blocks per SM: every block claims one tile past the end and
  // counts itself done with an atomic, so a small scan sized for a large
  // max_n stays cheap; large scans loop over tiles
  const uint64_t cap = (uint64_t)num_sms * std::min(2, scan_resident((const void *)k_scan<T>));
  const unsigned grid = (unsigned)std::min(tiles, cap);
  ScanState *st = reinterpret_cast<ScanState *>(tmp);
  ScanDesc *desc = reinterpret_cast<ScanDesc *>(tmp + 4);  // 32 bytes in
  pdl(k_scan<T>, grid, kScanThreads, 0, s, in, d_n, out, st, desc);
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

gs_status scan_set_wait(uint64_t *tmp, uint32_t max_polls, uint32_t withhold_first_tile, cudaStream_t s) {
  ScanState *st = reinterpret_cast<ScanState *>(tmp);
  const uint32_t w = withhold_first_tile ? 1u : 0u;
  GS_CUDA(cudaMemcpyAsync(&st->limit, &max_polls, 4, cudaMemcpyHostToDevice, s));
  GS_CUDA(cudaMemcpyAsync(&st->withhold, &w, 4, cudaMemcpyHostToDevice, s));
  return GS_OK;
}

uint64_t scan_tmp_words(uint64_t max_n) {
  const uint64_t tiles = std::max<uint64_t>((max_n + kScanTile - 1) / kScanTile, 1);
  return 4 + 4 * tiles;  // state (padded to 32 bytes) + one 32-byte descriptor per tile
}

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
