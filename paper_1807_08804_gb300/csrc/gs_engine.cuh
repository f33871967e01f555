// Engine-internal device structures shared by the kernels and the host
// orchestration.
#pragma once

#include <cooperative_groups.h>

#include "gs_internal.h"

namespace gs {

namespace cg = cooperative_groups;

constexpr uint32_t kUnbound = 0xFFFFFFFFu;
constexpr uint32_t kAny = 0xFFFFFFFFu;
constexpr uint32_t kMaxRounds = 64;
constexpr uint32_t kSmallRows = 2048;    // outputs sorted by one block in shared memory
constexpr uint32_t kTileRows = 1024;     // rows per tile of the large-output merge sort
constexpr uint32_t kBktPerTile = 4;      // sample-sort bucket slots per tile (buckets of 256 entries on average)
constexpr uint64_t kOverCap = 16;        // outputs up to kOverCap * cap rows are sorted on the device

// Per-query status.
enum : uint32_t {
  QS_OK = 0,        // running / finished normally
  QS_EMPTY = 1,     // some candidate set is empty: no embedding
  QS_OVERFLOW = 2,  // a device pool was too small: finish on the fallback path
  QS_INVALID = 3,   // empty slot (padding) or rejected by the host checks
  QS_TOPCAP = 4,    // more embeddings than cap: smallest rows via the fallback path
};

// Pools whose requested sizes the device records (Ctrl::hw), so that the
// host can enlarge a pool that was too small for the next run.
enum : int {
  HW_TLIST = 0, HW_ALIST, HW_FLIST, HW_EC_ITEMS, HW_EC_VALS, HW_LVL_WORDS, HW_ROWS, HW_OUT_ROWS, HW_OUT_WORDS,
  HW_STORE, HW_N
};

// Kernel kinds for statistics.
enum : int {
  KK_PLAN = 0, KK_FILTER, KK_COMPACT, KK_EXPLORE, KK_REFINE, KK_EC_COUNT, KK_EC_WRITE, KK_CLEAR,
  KK_JOIN_COUNT, KK_JOIN_WRITE, KK_SCAN, KK_SORT, KK_GATHER, KK_OTHER, KK_COMPACT_ALL, KK_SORT_LARGE, KK_N
};

// One query as the device sees it.  The host fills the query part (edges
// without repeats, incidence lists, degree needs); the device fills the plan.
struct DQuery {
  uint32_t k, m;
  uint32_t qv_base;                 // slot index of query vertex 0
  uint32_t qe_base;                 // slot index of query edge 0
  uint32_t vtype[kMaxK];            // type or kAny
  uint32_t vbind[kMaxK];            // data id or kUnbound
  uint8_t esrc[kMaxM], edst[kMaxM], erel[kMaxM];  // erel kRelAny8: variable edge
  uint8_t inc_begin[kMaxK + 1];     // incident edges of u: inc_edge[inc_begin[u] .. inc_begin[u+1])
  uint8_t inc_edge[2 * kMaxM];
  uint8_t need_begin[kMaxK + 1];    // degree needs of u: (plane, count) pairs
  uint16_t need_plane[2 * kMaxM];   // sig_plane(dir, rel, R)
  uint8_t need_cnt[2 * kMaxM];
  uint32_t mode;
  uint64_t cap;
  uint32_t proj;                    // projected vertices (bit mask); 0 = whole embeddings
  uint8_t refine_flags;             // kRefineOff, kRefineRev
  uint8_t refine_low;               // refinement skips vertices with at most this many incident edges (0: none)
  uint8_t kp;                       // output columns: the projected vertices pu[0..kp), ascending
  uint8_t pu[kMaxK];                //   (every vertex when proj == 0)
  uint8_t force_root;               // 0xFF, or the first visited vertex (inspection runs)
  uint8_t force_from_src;           // 0xFF, or a fixed edge-table orientation (inspection runs)
  // plan (device)
  uint32_t nvisit;
  uint8_t visit[kMaxK];
  uint8_t parent[kMaxK];            // spanning-tree parent (0xFF at the root)
  uint8_t pedge[kMaxK];             // tree edge to the parent
  uint8_t init_step[kMaxK];         // exploration step after which u has a candidate set
  uint8_t join[kMaxK];              // join order
  uint8_t pos[kMaxK];               // position of u in the join order
  uint8_t opos[kMaxK];              // join-order column of output column i (pos[pu[i]])
  uint8_t rorder[kMaxK];            // reversed refinement: vertex refined at sub-round j
  uint8_t from_src[kMaxM];          // edge-table orientation (1: keyed by esrc)
  uint32_t xinc[2 * kMaxM];         // incident edges packed by the plan (xinc_pack), same order as inc_edge
  uint32_t status;
  // Matching through a compressed graph (Section 3.5): data vertex v may be
  // a candidate of u only if its weighted node wgroup[v] is set in u's
  // weighted-graph candidate bitmap, wmask + u * wstride words (device
  // addresses; wmask = 0: no restriction).
  uint32_t wstride;
  uint64_t wmask, wgroup;
};

// Packed incident edge: bit 0 direction (0: u is the source), bits 1-8
// relation, 9-12 the other endpoint, 13-14 its role when u is explored.
__host__ __device__ __forceinline__ uint32_t xinc_pack(uint32_t dir, uint32_t rel, uint32_t w, uint32_t role) {
  return dir | (rel << 1) | (w << 9) | (role << 13);
}
__host__ __device__ __forceinline__ int xinc_dir(uint32_t x) { return (int)(x & 1u); }
__host__ __device__ __forceinline__ uint32_t xinc_rel(uint32_t x) { return (x >> 1) & 0xFFu; }
__host__ __device__ __forceinline__ uint32_t xinc_w(uint32_t x) { return (x >> 9) & 0xFu; }
__host__ __device__ __forceinline__ uint32_t xinc_role(uint32_t x) { return x >> 13; }

// Variable edges (a relation that is itself a variable, Section 3.2): erel
// kRelAny8 matches a data edge of any relation.  Such an edge reads the
// adjacency planes of distinct neighbours (2 + direction) as relation 0, and
// its signature and neighbour-type planes are 2R + direction.
constexpr uint32_t kRelAny8 = 0xFFu;
// Refinement variants (DQuery::refine_flags).
constexpr uint32_t kRefineOff = 1u, kRefineRev = 2u, kRefineBase = 4u;
__host__ __device__ __forceinline__ int adj_plane(int dir, uint32_t rel) { return rel == kRelAny8 ? dir + 2 : dir; }
__host__ __device__ __forceinline__ uint32_t adj_rel(uint32_t rel) { return rel == kRelAny8 ? 0u : rel; }
__host__ __device__ __forceinline__ uint32_t sig_plane(int dir, uint32_t rel, uint32_t R) {
  return rel == kRelAny8 ? 2 * R + (uint32_t)dir : (uint32_t)dir * R + rel;
}

// Per-query join bookkeeping and results (slot arrays).
struct QState {
  uint64_t count, fp;
  uint64_t cur_row_base, cur_rows, cur_word_base;   // rows of the current level
  uint64_t nxt_rows;                                 // rows produced for the next level
  uint64_t out_row_base, out_rows, out_word_base;   // final rows in the output pool
  uint64_t fin_row_base, fin_word_base;             // sorted rows in query order
  uint64_t lrg_row_base;                             // rows sorted by the merge path
  uint64_t lrg_tile_base;                            // their first tile
  uint64_t sort_rows;                                // rows entering the merge sort (after selection)
  uint64_t nfinal;                                   // rows returned (projected: distinct tuples, at most cap)
  uint64_t inter_words, peak_words;                  // partial-embedding words over the levels before the last
  uint32_t more;                                     // projected: more distinct tuples than cap
  uint32_t bkt_fail;                                 // a bucket of the sample sort overflowed: merge path
};

// BatchOut::nrows top bit: a projected query had more distinct tuples than
// the rows returned.
constexpr uint64_t kRowsMore = 1ull << 63;

// Sort key of the large-output merge sort: the row's output columns packed
// at the graph's id width, the leading ones in hi, the following ones
// (from the first column hi does not hold whole) in lo.
struct SortKey {
  uint64_t hi, lo;
};
__host__ __device__ __forceinline__ bool operator==(const SortKey &a, const SortKey &b) { return a.hi == b.hi && a.lo == b.lo; }
__host__ __device__ __forceinline__ bool operator!=(const SortKey &a, const SortKey &b) { return !(a == b); }
__host__ __device__ __forceinline__ bool operator<(const SortKey &a, const SortKey &b) {
  return a.hi != b.hi ? a.hi < b.hi : a.lo < b.lo;
}

// Top-cap selection of a query with more than cap large rows (radix select
// on the packed sort keys): rows with key <= thresh go into the sort.
struct SelState {
  uint64_t lo, hi;        // smallest and largest key of the query's rows
  uint64_t prefix;        // key bits chosen so far (bits >= mbits)
  uint64_t need;          // rows still to take from the current bucket
  uint64_t thresh;        // the cut, once chosen
  uint64_t kept;          // rows kept (compaction counter)
  uint32_t mbits, shift, width;  // rows in play match prefix at bits >= mbits; digit = bits [shift, shift + width)
  uint32_t state;         // 0: not selected, 1: choosing, 2: cut chosen
};

// Rows of level s kept aside while the allocator lays out level s+1.
struct SrcRows {
  uint64_t row_base, rows, word_base;
};

// What one join level asks of the pools for one query, gathered by a
// grid-wide pass so that the one-block allocator reads it coalesced: rows
// and words of the next level (v[0], v[1]) or of the final output (v[2],
// v[3]); flags 1 = final output, 2 = next level, 4 = sent away by the
// allocator's first pass.
struct LevelSize {
  uint64_t v[4];
  uint32_t flags, pad;
};

// One wave of a batch, as listed in the batch's wave table.
struct WaveDesc {
  uint32_t q0, nq;        // batch query range
  uint32_t qv0, nqv;      // batch query-vertex range
  uint32_t qe0, nqe;      // batch query-edge range
};

// Batch-level results written by the epilogue of each wave.
struct BatchOut {
  uint64_t *count, *fp, *nrows, *word_off;  // [n]
  uint64_t *inter, *peak;                    // [n] partial-embedding words: total and largest level
  uint32_t *status;                          // [n]
  uint32_t *store;                           // rows of every query, query-vertex order
  uint64_t store_cap;                        // words
};

struct Ctrl {
  uint64_t len[10];                 // device-side lengths read by persistent kernels
  uint32_t changed[kMaxRounds];     // refinement: did round t clear any bit
  uint64_t lvl_top, out_top;        // output pool top (words)
  uint64_t out_rows_total;
  uint64_t store_top;               // batch row store top (words)
  uint32_t wave;                    // index of the wave being run
  uint32_t err;
  uint32_t max_nvisit;              // longest visit order in the wave
  uint32_t refine_iters;            // rounds run by the refinement loop
  uint64_t fb_src[3];               // source rows staged by the chunked join
  uint64_t hw[10];                  // sizes the run asked of each pool (see HW_*)
  uint64_t max_large_rows;          // largest output above the one-block sort limit
  uint64_t over_cap;                // large outputs with more rows than cap (selected before sorting)
  uint64_t fin_words;               // words of the rows returned by this wave
  uint64_t bytes[KK_N];             // algorithmic bytes per kernel kind
  uint32_t bkt_fail;                // some query's sample-sort bucket overflowed (merge path runs)
  uint32_t pad_;
  uint64_t nbkt;                    // bucket slots of the sample sort (kBktPerTile per tile)
  uint64_t tlist_top;               // exploration work list: entries claimed this step
};

// Everything a kernel needs, passed by value.  Capacities are fixed when the
// batch is created; the number of live queries of the wave is implicit
// (padding slots are QS_INVALID).
struct Wave {
  DevGraph G;
  DQuery *dq;                       // slot queries [nq + 1]; dq[nq] is a permanent empty slot
  QState *qs;                       // [nq]
  Ctrl *ctrl;
  uint32_t nq, nqv, nqe;            // slot capacities
  uint32_t *qv_q;                   // slot query of each slot query vertex [nqv]
  uint32_t *qe_q;                   // slot query of each slot query edge [nqe]
  // source of the wave descriptors
  const DQuery *all_dq;             // batch queries [n]
  const WaveDesc *waves;
  BatchOut bo;
  // candidate bitmaps
  uint32_t *bm;                     // [nqv][slot_words]
  uint64_t slot_words;
  // compaction
  uint32_t *ccount;                 // candidates per chunk [nqv * nchunks]
  uint64_t *cscan;                  // [nqv * nchunks + 1]
  uint64_t *ascan;                  // [nqv * nchunks + 1] (refinement items)
  // candidate lists
  uint32_t *tlist; uint64_t tlist_cap;   // exploration work list
  uint32_t *alist; uint64_t alist_cap;   // every set before refinement
  uint32_t *tlist_q, *alist_q;           // owner of each entry: query / global query vertex
  uint32_t *fcnt; uint64_t *fscan;       // filter work items per query [nq] and their scan [nq + 1]
  uint64_t *clist;                       // non-empty chunks of a compaction: (gqv << 32) | count index
  uint32_t *flist; uint64_t flist_cap;   // final sets
  uint64_t *flist_off;              // [nqv]
  uint32_t *flist_len;              // [nqv]
  // edge tables
  uint32_t *ec_nkeys;               // [nqe]
  uint64_t *ec_key_base;            // [nqe + 1]
  uint32_t *ec_cnt; uint64_t ec_items_cap;
  uint64_t *ec_off;                 // [ec_items_cap + 1]
  uint32_t *ec_vals; uint64_t ec_vals_cap;
  // join levels
  uint32_t *lvl[2]; uint64_t lvl_words;
  uint32_t *row_cnt; uint64_t row_cap;
  uint64_t *row_scan;               // [row_cap + 1]
  SrcRows *src;                     // [nq]
  LevelSize *lsz;                   // [nq]
  uint32_t *out; uint64_t out_words;  // final rows, join-order columns
  uint32_t *out_q;                  // slot query of each output row
  uint64_t out_rows_cap;
  uint32_t *out_final;              // sorted rows, query-vertex order
  // sort
  SortKey *skey[2];                     // sort keys of the large-output merge sort
  uint32_t *sval[2];                    // row indices of the large-output merge sort
  uint64_t *msplit;                     // merge-path split of each output tile (bucket sort: fill cursors)
  uint32_t merge_only;                  // large outputs: skip the bucket sort, tile sort and merge passes only
  uint32_t *bkt_id;                     // bucket sort: each large entry's bucket (count pass to scatter pass)
  SortKey *bspl_key;                    // bucket sort: splitters of each query's buckets, one slot per tile
  SortKey *bspl_key2;                   //   their second keys
  uint32_t *bspl_row;                   //   and their row indices
  uint32_t *ptcount;                    // projected outputs: distinct tuples starting in each tile
  uint64_t *ptscan;                     //   and their scan [tiles + 1]
  SelState *sel;                        // [nq] top-cap selection
  uint32_t *shist;                      // [nq][256] digit histograms of the selection
  int stats;
  int c0_only;                      // filter: exactly Definition 3.3's set (no neighbour-type test)
};

// ------------------------------------------------------------ launchers
void launch_prologue(const Wave &W, cudaStream_t s, int sms);
void launch_plan(const Wave &W, const uint32_t *type_count, cudaStream_t s, int sms);
void launch_filter(const Wave &W, cudaStream_t s, int sms);
void launch_compact_count(const Wave &W, int mode, uint32_t step, cudaStream_t s, int sms);
void launch_compact_claim(const Wave &W, uint32_t step, cudaStream_t s, int sms);
void launch_compact_write(const Wave &W, int mode, uint32_t step, const uint64_t *scan, uint32_t *dst, uint32_t *owner,
                          uint64_t cap, int hw_slot, cudaStream_t s, int sms);
void launch_explore(const Wave &W, uint32_t step, int group, cudaStream_t s, int sms);
// sub: kAllSub refines every vertex of every query; j < kMaxK refines, in
// queries with kRefineRev, the vertex rorder[j] (other queries at j = 0).
constexpr uint32_t kAllSub = 0xFFFFFFFFu;
void launch_refine(const Wave &W, uint32_t round, uint32_t sub, int group, cudaStream_t s, int sms);
void launch_list_table(const Wave &W, cudaStream_t s, int sms);
void launch_join_plan(const Wave &W, cudaStream_t s, int sms);
void launch_ec_limit(const Wave &W, cudaStream_t s, int sms);
void launch_ec(const Wave &W, bool write, int group, cudaStream_t s, int sms);
void launch_clear(const Wave &W, cudaStream_t s, int sms);
void launch_join0(const Wave &W, cudaStream_t s, int sms);
void launch_join_count(const Wave &W, uint32_t lvl, int group, cudaStream_t s, int sms);
void launch_level_alloc(const Wave &W, uint32_t lvl, cudaStream_t s);
void launch_join_write(const Wave &W, uint32_t lvl, int group, cudaStream_t s, int sms);
void launch_final_bases(const Wave &W, cudaStream_t s);
void launch_small_sort(const Wave &W, cudaStream_t s, int sms);
void launch_sort_keys(const Wave &W, uint32_t *perm, SortKey *keys, cudaStream_t s, int sms);
void launch_select(const Wave &W, const uint32_t *pin, const SortKey *kin, uint32_t *pout, SortKey *kout,
                   cudaStream_t s, int sms);
void launch_bucket_sort(const Wave &W, const uint32_t *pin, const SortKey *kin, uint32_t *px, SortKey *kx,
                        uint32_t *p0, SortKey *k0, uint32_t *p1, SortKey *k1, uint64_t *scan_tmp, cudaStream_t s,
                        int sms);
void launch_tile_sort(const Wave &W, const uint32_t *pin, const SortKey *kin, uint32_t *pout, SortKey *kout,
                      cudaStream_t s, int sms);
void launch_merge_pass(const Wave &W, const uint32_t *pin, const SortKey *kin, uint32_t *pout, SortKey *kout,
                       uint64_t run, cudaStream_t s, int sms);
void launch_gather(const Wave &W, const uint32_t *perm0, const uint32_t *perm1, cudaStream_t s, int sms);
void launch_project(const Wave &W, const uint32_t *perm0, const uint32_t *perm1, const SortKey *key0,
                    const SortKey *key1, uint64_t max_tiles, uint64_t *scan_tmp, cudaStream_t s, int sms);
void launch_epilogue(const Wave &W, cudaStream_t s, int sms);

}  // namespace gs
