// Internal declarations shared by the engine's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "../../include/gs.h"

namespace gs {

constexpr uint32_t kMaxK = 16;        // query vertices
constexpr uint32_t kMaxM = 120;       // query edges (after dropping repeats)
constexpr uint32_t kNbrBits = 24;     // packed adjacency entry: rel << 24 | neighbour
constexpr uint32_t kNbrMask = (1u << kNbrBits) - 1;
constexpr uint32_t kFull = 0xFFFFFFFFu;

// ------------------------------------------------------------ launches
// Pipeline kernels are launched with programmatic stream serialisation, so
// that the launch of a kernel is prepared while the one before it in the
// stream runs; each kernel first waits for the grids it depends on to
// complete and for their writes to be visible (griddepcontrol.wait; a no-op
// without a preceding dependent grid).  No kernel releases its dependents
// early (griddepcontrol.launch_dependents): blocks scheduled early wait
// holding SM slots that the batches running beside it on other streams
// would use (measured: 21.1 -> 22.3 ms per batch-4m step with the release at
// kernel start, 20.8 ms without it).
__device__ __forceinline__ void gdc_wait() {
#if defined(__CUDA_ARCH__)
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

template <typename... KArgs, typename... Args>
inline void pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ------------------------------------------------------------ errors
void set_error(const std::string &msg);
gs_status fail(gs_status st, const std::string &msg);
gs_status cuda_fail(cudaError_t e, const char *what);
// Every device allocation of the library goes through dev_malloc: plain
// cudaMalloc, except that a test can arm a simulated allocation failure with
// gs_debug_fail_alloc (the armed call then returns cudaErrorMemoryAllocation
// and allocates nothing), so that out-of-memory paths run without exhausting
// the device.
cudaError_t dev_malloc_bytes(void **p, size_t bytes);
void debug_fail_alloc(int64_t after);  // gs_debug_fail_alloc
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
  return dev_malloc_bytes(reinterpret_cast<void **>(p), bytes);
}
#define GS_CUDA(call)                                         \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return ::gs::cuda_fail(e_, #call); \
  } while (0)

// ------------------------------------------------------------ device graph
// Both directions as CSR over packed (relation << 24 | neighbour) entries,
// each row ascending, i.e. sorted by (relation, neighbour).  Signatures:
// for direction d and relation r, plane (d * R + r) holds one 4-bit count per
// vertex (8 vertices per 32-bit word): the number of distinct r-neighbours in
// that direction, saturated at 15.
struct DevGraph {
  uint32_t V, T, R;
  uint64_t E;
  // Adjacency planes: 0 = out, 1 = in, rows of rel << 24 | nbr sorted by
  // (relation, neighbour); 2 = out, 3 = in, rows of the distinct neighbours
  // over all relations, ascending (read by variable edges as relation 0).
  const uint64_t *off[4];   // [plane][V+1]
  const uint32_t *adj[4];   // [plane][row entries]
  const uint8_t *vtype;     // [V]
  const uint32_t *tvid;     // [V] vertex ids grouped by type, ascending within a type
  const uint32_t *toff;     // [T+1] start of each type's run in tvid
  // Signature and neighbour-type planes: dir * R + rel, then 2R + dir for
  // the distinct neighbours over all relations (P = 2R + 2 planes).
  const uint32_t *sigge;    // [(T+1) * P * 16] vertices of type t (t = T: any) with plane count >= c
  const uint32_t *tmask;    // [P][V] OR of 1 << (type mod 32) over v's neighbours in each plane
  const uint32_t *sig_t;    // sig with entry x of each plane belonging to vertex tvid[x]
  const uint32_t *tmask_t;  // tmask likewise
  const uint32_t *sig;      // [P][sig_words]
  uint64_t sig_words;       // ceil(V / 8)
  uint32_t W0;              // bitmap words per candidate set: ceil(V/32)
  uint32_t W1;              // summary words: ceil(W0/32)
  uint32_t nchunks;         // level-2 bits per set: one per 32 summary words, ceil(W1/32)
  uint32_t ipg;             // level-2 words per set = compaction items per set: ceil(nchunks/32)
  uint32_t idbits;          // bits of the largest vertex id (at least 1)
};

}  // namespace gs

struct gs_graph {
  gs::DevGraph d;
  int device;
  int num_sms;
  uint64_t *off_out, *off_in, *off_aout, *off_ain;
  uint32_t *adj_out, *adj_in, *adj_aout, *adj_ain;
  uint8_t *vtype;
  uint32_t *tvid, *toff, *sigge, *tmask, *sig_t, *tmask_t;
  uint32_t *sig;
  uint32_t *type_count;     // host copy [T]
  uint32_t *sigge_host;     // host copy of DevGraph::sigge (admission estimates)
  uint64_t hash;            // content hash (tuning cache key)
  void *cache;              // batches reused by gs_match / gs_match_batch
  void *fallback;           // context of the chunked join
  void *khop;               // buffers of the domain-graph exploration
  uint32_t tuned_group;     // lanes per work item chosen by gs_tune (0 = default)
  uint32_t tuned_rounds;    // refinement rounds chosen by gs_tune (0 = default)
  uint32_t tuned_jgroup;    // lanes per partial row in the join chosen by gs_tune (0 = tuned_group)
};

namespace gs {

void release_cache(gs_graph *g);
// Replace a loaded graph's degree signatures by counts[plane * V + v]
// (saturated at 15; planes as DevGraph::sig) and rebuild the tables derived
// from them (type-ordered planes, signature statistics).  Synchronous.
gs_status graph_set_signatures(gs_graph *g, const uint8_t *counts);
void release_fallback(gs_graph *g);
void release_khop(gs_graph *g);

// ------------------------------------------------------------ primitives
// Exclusive prefix sum of n uint32 counts into out[0..n] (out[n] = total),
// where n is read from device memory (*d_n), in one kernel (single-pass scan
// with decoupled look-back).  max_n bounds n and sizes the launch.  tmp
// holds scan_tmp_words(max_n) uint64 words, zeroed once when allocated and
// used by nothing but scans; scans that share it must run in order (one
// stream).
// scan_error_word() points at a device word that turns non-zero when a
// look-back wait hits its bound on that scratch (the scan then takes that
// tile's prefix by summing its inputs directly, so its result is still
// exact); the word stays set until the host clears it.  scan_set_wait sets
// the bound (polls; 0 = the default, 2^22) and, for tests, makes the first
// tile of every multi-tile scan on the scratch publish nothing, so that every
// later tile's wait runs to the bound.  Both copy from the host on stream s.
uint64_t scan_tmp_words(uint64_t max_n);
void scan_u32(const uint32_t *in, uint64_t *out, const uint64_t *d_n, uint64_t max_n, uint64_t *tmp,
              cudaStream_t s, int num_sms);
inline const uint32_t *scan_error_word(const uint64_t *tmp) { return reinterpret_cast<const uint32_t *>(tmp); }
gs_status scan_set_wait(uint64_t *tmp, uint32_t max_polls, uint32_t withhold_first_tile, cudaStream_t s);
// Same for uint64 inputs.
void scan_u64(const uint64_t *in, uint64_t *out, const uint64_t *d_n, uint64_t max_n, uint64_t *tmp,
              cudaStream_t s, int num_sms);

// Stable LSD radix sort of (key, val) pairs by key bits [0, nbits).  n is read
// from device memory.  Data ping-pongs between (k0, v0) and (k1, v1); the
// return value is 0 if the result ends in (k0, v0), 1 if in (k1, v1).
// tmp must hold radix_tmp_words(max_n) uint64 values, zeroed when allocated
// and not shared with scans run outside the sort.
uint64_t radix_tmp_words(uint64_t max_n);
int radix_sort_pairs(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const uint64_t *d_n, uint64_t max_n,
                     int bit_lo, int nbits, uint64_t *tmp, cudaStream_t s, int num_sms);
int radix_passes(int nbits);

}  // namespace gs
