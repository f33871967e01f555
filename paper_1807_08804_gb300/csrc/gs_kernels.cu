// The filtering-and-joining kernels (thesis Ch. 3, Algorithm
// "FilteringAndJoining"), each persistent over a device-sized work list so a
// whole batch can be captured once in a CUDA graph:
//   plan        query plan on the device (Section 3.3.2 / 3.5)
//   filter      kernel_check: C0 bitmaps of the first visited vertex
//   compact     kernel_collect: bitmap -> sorted candidate list
//   explore     kernel_explore: prune + expand along the spanning tree
//   refine      refine_node_candidates: prune over every query edge, to a fixpoint
//   ec_*        collect_edge_candidates: count / scan / write
//   join_*      combine_edge_candidates: count / scan / write per level
//   sort/gather lexicographic order of the embeddings, query-vertex columns
#include <mutex>
#include <unordered_map>

#include "gs_engine.cuh"

namespace gs {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint64_t gtid() { return blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; }
__device__ __forceinline__ uint64_t gthreads() { return (uint64_t)gridDim.x * blockDim.x; }

// ------------------------------------------------------------ bitmaps
// A candidate set over V is a three-level bitmap: W0 words of one bit per
// vertex, W1 summary words with one bit per non-zero level-0 word, and ipg
// words with one bit per non-zero group of 32 summary words (a "chunk" of
// 32,768 vertices).  Compaction and clearing visit only non-zero chunks.
__device__ __forceinline__ uint32_t *slot_of(const Wave &W, uint32_t gqv) { return W.bm + (uint64_t)gqv * W.slot_words; }
__device__ __forceinline__ bool bit_test(const uint32_t *slot, uint32_t v) { return (slot[v >> 5] >> (v & 31)) & 1u; }
__device__ __forceinline__ void bit_set(const Wave &W, uint32_t *slot, uint32_t v) {
  uint32_t old = atomicOr(&slot[v >> 5], 1u << (v & 31));
  if (old == 0) {
    uint32_t old1 = atomicOr(&slot[W.G.W0 + (v >> 10)], 1u << ((v >> 5) & 31));
    if (old1 == 0) atomicOr(&slot[W.G.W0 + W.G.W1 + (v >> 20)], 1u << ((v >> 15) & 31));
  }
}
__device__ __forceinline__ void bit_clear(uint32_t *slot, uint32_t v) { atomicAnd(&slot[v >> 5], ~(1u << (v & 31))); }

// Matching through a compressed graph (Section 3.5, Theorem 3.2): v can be
// a match of u only if the weighted node whose mapping list holds v is a
// candidate of u in the weighted graph.
__device__ __forceinline__ bool wmask_ok(const DQuery &Q, uint32_t u, uint32_t v) {
  if (!Q.wmask) return true;
  const uint32_t x = reinterpret_cast<const uint32_t *>(Q.wgroup)[v];
  const uint32_t *m = reinterpret_cast<const uint32_t *>(Q.wmask) + (uint64_t)u * Q.wstride;
  return (m[x >> 5] >> (x & 31)) & 1u;
}

// Candidate test of Definition 3.3 read per direction and relation: binding,
// type, and for every (direction, relation) at least as many distinct data
// neighbours as the query vertex has query neighbours.
__device__ __forceinline__ bool cand_ok(const DevGraph &G, const DQuery &Q, uint32_t u, uint32_t v) {
  uint32_t b = Q.vbind[u];
  if (b != kUnbound && b != v) return false;
  uint32_t t = Q.vtype[u];
  if (t != kAny && G.vtype[v] != t) return false;
  if (!wmask_ok(Q, u, v)) return false;
  for (uint32_t i = Q.need_begin[u]; i < Q.need_begin[u + 1]; ++i) {
    uint32_t w = G.sig[(uint64_t)Q.need_plane[i] * G.sig_words + (v >> 3)];
    if (((w >> ((v & 7) * 4)) & 15u) < Q.need_cnt[i]) return false;
  }
  return true;
}

// ------------------------------------------------------------ group search
// First index in [lo, hi) with a[i] >= key, searched by a tile of G lanes
// (G-ary search, then one probe per lane).
template <int G>
__device__ __forceinline__ uint64_t tile_lower_bound(const cg::thread_block_tile<G> &t, const uint32_t *a, uint64_t lo,
                                                     uint64_t hi, uint32_t key) {
  const uint32_t r = t.thread_rank();
  while (hi - lo > G) {
    uint64_t step = (hi - lo + G - 1) / G;
    uint64_t p = lo + (uint64_t)(r + 1) * step - 1;
    bool less = p < hi && a[p] < key;
    uint32_t c = __popc(t.ballot(less));
    uint64_t nlo = lo + (uint64_t)c * step;
    uint64_t nhi = c < G ? lo + (uint64_t)(c + 1) * step - 1 : hi;
    lo = nlo < hi ? nlo : hi;
    hi = nhi < hi ? nhi : hi;
    if (lo > hi) lo = hi;
  }
  uint64_t i = lo + r;
  bool less = i < hi && a[i] < key;
  return lo + __popc(t.ballot(less));
}

// Relation run of a sorted packed row: entries with (x >> 24) == rel.
template <int G>
__device__ __forceinline__ void rel_range(const cg::thread_block_tile<G> &t, const DevGraph &Gr, int dir, uint32_t v,
                                          uint32_t rel, uint64_t &lo, uint64_t &hi) {
  const uint32_t *a = Gr.adj[dir];
  uint64_t b = Gr.off[dir][v], e = Gr.off[dir][v + 1];
  lo = tile_lower_bound<G>(t, a, b, e, rel << kNbrBits);
  hi = tile_lower_bound<G>(t, a, lo, e, (rel + 1) << kNbrBits);
}

// The same run, with a fast path for a row that fits the tile: one load per
// lane (lane r holds entry base + r in x, all ones past the row) and two
// ballots.  Returns true on the fast path, where the run's entries can be
// taken from the lanes by shuffles instead of reloads.
template <int G>
__device__ __forceinline__ bool rel_run(const cg::thread_block_tile<G> &t, const DevGraph &Gr, int dir, uint32_t v,
                                        uint32_t rel, uint64_t &base, uint64_t &lo, uint64_t &hi, uint32_t &x) {
  const uint32_t *a = Gr.adj[dir];
  const uint64_t b = Gr.off[dir][v], e = Gr.off[dir][v + 1];
  base = b;
  if (e - b <= G) {
    const uint32_t r = t.thread_rank();
    x = r < e - b ? a[b + r] : 0xFFFFFFFFu;
    lo = b + __popc(t.ballot(x < (rel << kNbrBits)));
    hi = b + __popc(t.ballot(x < ((rel + 1) << kNbrBits)));
    return true;
  }
  x = 0xFFFFFFFFu;
  lo = tile_lower_bound<G>(t, a, b, e, rel << kNbrBits);
  hi = tile_lower_bound<G>(t, a, lo, e, (rel + 1) << kNbrBits);
  return false;
}

// Entry j of the run scanned by lane r in the tile: from the lanes on the
// fast path, from memory otherwise (all lanes call it: it may shuffle).
template <int G>
__device__ __forceinline__ uint32_t run_entry(const cg::thread_block_tile<G> &t, const DevGraph &Gr, int dir,
                                              bool fast, uint64_t base, uint32_t x, uint64_t j, uint64_t hi) {
  if (fast) {
    const uint32_t y = t.shfl(x, (unsigned)((j - base) & (G - 1)));
    return j < hi ? y : 0xFFFFFFFFu;
  }
  return j < hi ? Gr.adj[dir][j] : 0xFFFFFFFFu;
}

// Binary search of a sorted uint32 list (all lanes do the same search).
__device__ __forceinline__ int64_t list_find(const uint32_t *a, uint64_t n, uint32_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < n && a[lo] == key) ? (int64_t)lo : -1;
}
__device__ __forceinline__ bool list_has(const uint32_t *a, uint64_t n, uint32_t key) { return list_find(a, n, key) >= 0; }

// Segment of an item: largest s in [0, ns) with base(s) <= item, where
// base(s) = bases[s * stride].
__device__ __forceinline__ uint32_t seg_of(const uint64_t *bases, uint64_t stride, uint32_t ns, uint64_t item) {
  uint32_t lo = 0, hi = ns;  // invariant: answer in [lo, hi)
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (bases[(uint64_t)mid * stride] <= item) lo = mid; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ uint32_t seg_of_rows(const QState *qs, uint32_t nq, uint64_t item) {
  uint32_t lo = 0, hi = nq;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (qs[mid].cur_row_base <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// Tile-cooperative form of the same search: each round the G lanes probe G
// evenly spaced points of [lo, hi) and keep the gap between the last probe
// at or below the item and the first above it, so a search over n segments
// takes log_{G+1}(n) dependent loads instead of log_2(n).  Every lane of the
// tile calls it with the same item and gets the same answer.
template <int G, class Tile, class Base>
__device__ __forceinline__ uint32_t tile_seg(const Tile &tile, uint32_t ns, uint64_t item, Base base) {
  uint32_t lo = 0, hi = ns;  // invariant: answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t step = (hi - lo + G) / (G + 1);
    const uint32_t p = lo + (tile.thread_rank() + 1) * step;
    const bool le = p < hi && base(p) <= item;
    const uint32_t cnt = __popc(tile.ballot(le));  // the probes at or below the item are a prefix
    const uint32_t nlo = lo + cnt * step;
    hi = min(hi, nlo + step);
    lo = nlo;
  }
  return lo;
}

// Algorithmic bytes: each thread accumulates in a register; at the end of
// the kernel one warp-reduced atomic per warp adds them up (statistics runs
// only).  Every lane of the warp must reach flush_bytes.
__device__ __forceinline__ void flush_bytes(const Wave &W, int kind, uint64_t b) {
  if (!W.stats) return;
  for (int o = 16; o; o >>= 1) b += __shfl_down_sync(kFull, b, o);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd((unsigned long long *)&W.ctrl->bytes[kind], (unsigned long long)b);
}

__device__ __forceinline__ void mark(DQuery &Q, uint32_t st) { atomicCAS(&Q.status, QS_OK, st); }

// splitmix64 finaliser (Steele, Lea & Flood 2014); row hash for fingerprints.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// Hash of an embedding in query-vertex order; row holds join-order columns
// 0..s, with column s+1 (query vertex w) = c.
__device__ __forceinline__ uint64_t row_hash(const DQuery &Q, const uint32_t *row, uint32_t w, uint32_t c) {
  uint64_t h = Q.k;
  for (uint32_t u = 0; u < Q.k; ++u) {
    uint32_t x = u == w ? c : row[Q.pos[u]];
    h = mix64(h ^ ((uint64_t)x + (uint64_t)(u + 1) * 0x9E3779B97F4A7C15ull));
  }
  return h;
}

// ============================================================ plan
// Section 3.5 ("Modify the query plan"): start at the bound vertex of largest
// degree; with no bound vertex, Section 3.3.2 ranks by deg(u)/freq(type(u)),
// which this plan refines into the expected size of u's filtered set (type
// frequency times, per degree need, the measured fraction of that type's
// vertices meeting it), so the exploration starts from the fewest
// candidates; then repeatedly explore the already-covered vertex with the
// most uncovered neighbours until every vertex is covered.  The explored vertices
// form the visit order; each newly covered vertex hangs below the vertex that
// covered it (the spanning tree T).
__global__ void k_plan(Wave W, const uint32_t *type_count) {
  gdc_wait();
  const WaveDesc D = W.waves[W.ctrl->wave];
  for (uint64_t qi = gtid(); qi <= W.nq; qi += gthreads()) {
    DQuery &Q = W.dq[qi];
    if (qi >= D.nq) {  // padding and the permanent empty slot
      Q.k = 0; Q.m = 0; Q.status = QS_INVALID; Q.nvisit = 0;
      if (qi < W.nq) {
        QState &S = W.qs[qi];
        S = QState{};
      }
      continue;
    }
    QState &S = W.qs[qi];
    S = QState{};
    Q.qv_base -= D.qv0;
    Q.qe_base -= D.qe0;
    if (Q.status == QS_INVALID) continue;
    Q.status = QS_OK;
    const uint32_t k = Q.k;
    uint32_t nbr[kMaxK];  // neighbour masks
    for (uint32_t u = 0; u < k; ++u) {
      nbr[u] = 0;
      for (uint32_t i = Q.inc_begin[u]; i < Q.inc_begin[u + 1]; ++i) {
        uint32_t e = Q.inc_edge[i];
        nbr[u] |= 1u << (Q.esrc[e] == u ? Q.edst[e] : Q.esrc[e]);
      }
    }
    int root = Q.force_root != 0xFF ? (int)Q.force_root : -1;
    if (root < 0)
      for (uint32_t u = 0; u < k; ++u)
        if (Q.vbind[u] != kUnbound && (root < 0 || __popc(nbr[u]) > __popc(nbr[root]))) root = (int)u;
    if (root < 0) {
      // no bound vertex: the vertex whose filtered candidate set is expected
      // to be smallest (its type's vertex count times, per degree need, the
      // fraction of those vertices that meet it; ties: more neighbours)
      const uint32_t P = 2 * W.G.R + 2;
      float best = 0.f;
      for (uint32_t u = 0; u < k; ++u) {
        const uint32_t t = Q.vtype[u] == kAny ? W.G.T : Q.vtype[u];
        const float f = (float)(t == W.G.T ? W.G.V : type_count[t]);
        float est = f;
        for (uint32_t i = Q.need_begin[u]; i < Q.need_begin[u + 1] && f > 0.f; ++i)
          est *= (float)W.G.sigge[((uint64_t)t * P + Q.need_plane[i]) * 16 + Q.need_cnt[i]] / f;
        if (root < 0 || est < best || (est == best && __popc(nbr[u]) > __popc(nbr[root]))) {
          root = (int)u;
          best = est;
        }
      }
    }
    for (uint32_t u = 0; u < kMaxK; ++u) { Q.parent[u] = 0xFF; Q.pedge[u] = 0xFF; Q.init_step[u] = 0xFF; }
    uint32_t covered = 1u << root, inO = 0, all = (k == 32) ? 0xFFFFFFFFu : ((1u << k) - 1);
    Q.init_step[root] = 0;
    uint32_t nv = 0, cur = (uint32_t)root;
    for (;;) {
      Q.visit[nv] = (uint8_t)cur;
      inO |= 1u << cur;
      uint32_t fresh = nbr[cur] & ~covered;
      for (uint32_t i = Q.inc_begin[cur]; i < Q.inc_begin[cur + 1]; ++i) {
        uint32_t e = Q.inc_edge[i];
        uint32_t w = Q.esrc[e] == cur ? Q.edst[e] : Q.esrc[e];
        if ((fresh >> w) & 1u) {
          if (Q.parent[w] == 0xFF) { Q.parent[w] = (uint8_t)cur; Q.pedge[w] = (uint8_t)e; Q.init_step[w] = (uint8_t)(nv + 1); }
        }
      }
      covered |= fresh;
      nv++;
      if (covered == all) break;
      int best = -1, bestc = -1;
      for (uint32_t u = 0; u < k; ++u) {
        if (!((covered >> u) & 1u) || ((inO >> u) & 1u)) continue;
        int c = __popc(nbr[u] & ~covered);
        if (c > bestc) { bestc = c; best = (int)u; }
      }
      if (best < 0 || bestc <= 0) { Q.status = QS_INVALID; break; }  // disconnected (host rejects these)
      cur = (uint32_t)best;
    }
    Q.nvisit = nv;
    atomicMax(&W.ctrl->max_nvisit, nv);
    // reversed refinement order (only when asked for): vertices by the step
    // that gave them a candidate set, last first (ties: higher index first);
    // u's position is the number of vertices that come before it
    if (Q.refine_flags & kRefineRev)
      for (uint32_t u = 0; u < k; ++u) {
        uint32_t before = 0;
        for (uint32_t w = 0; w < k; ++w)
          before += Q.init_step[w] > Q.init_step[u] || (Q.init_step[w] == Q.init_step[u] && w > u);
        Q.rorder[before] = (uint8_t)u;
      }
    // every incident edge of every query vertex, packed for exploration and
    // refinement: direction, relation, other endpoint and, for a vertex that
    // is explored (leaves of the spanning tree are not), the endpoint's role
    // at that step (0: set not built yet, 1: set built, 2: child initialised
    // now)
    uint8_t step_of[kMaxK];
    for (uint32_t u = 0; u < k; ++u) step_of[u] = 0xFF;
    for (uint32_t s = 0; s < nv; ++s) step_of[Q.visit[s]] = (uint8_t)s;
    for (uint32_t u = 0; u < k; ++u) {
      const uint32_t s = step_of[u];
      for (uint32_t i = Q.inc_begin[u]; i < Q.inc_begin[u + 1]; ++i) {
        const uint32_t e = Q.inc_edge[i];
        const uint32_t dir = Q.esrc[e] == u ? 0u : 1u;
        const uint32_t w = dir == 0 ? Q.edst[e] : Q.esrc[e];
        uint32_t role = 0;
        if (s != 0xFF) {
          role = Q.init_step[w] <= s ? 1u : 0u;
          if (Q.parent[w] == u && Q.init_step[w] == s + 1 && Q.pedge[w] == e) role = 2u;
          // the baseline checks only spanning-tree edges it can follow forwards
          if ((Q.refine_flags & kRefineBase) && (role != 2u || dir != 0u)) role = 3u;
        }
        Q.xinc[i] = xinc_pack(dir, Q.erel[e], w, role);
      }
    }
  }
}

// ============================================================ filter
// kernel_check for the first visited vertex u of each query.  Work items
// (one warp each) per query: a bound u has one (its binding, if it passes the
// test); a typed u has one per 1024 vertices of its type, taken from the
// per-type vertex lists, so the filter reads only vertices that can pass the
// type test, and there the neighbour-type test (masks_ok) is applied as well
// unless the exact Definition 3.3 set is asked for (W.c0_only, inspection);
// an untyped u has one per summary word (1024 vertices), which writes 32
// level-0 words and the summary word outright.
__device__ __forceinline__ uint32_t vertex_filter_items(const DevGraph &G, const DQuery &Q, uint32_t u) {
  if (Q.vbind[u] != kUnbound) return 1;
  if (Q.vtype[u] != kAny) return (G.toff[Q.vtype[u] + 1] - G.toff[Q.vtype[u]] + 1023) / 1024;
  return G.W1;
}
// The vertices whose sets the filter builds: the first visited vertex, and
// for the refinement baseline every spanning-tree child reached against its
// edge's direction (without the incoming graph only a scan finds those).
__device__ __forceinline__ bool filled_by_filter(const DQuery &Q, uint32_t u) {
  if (u == Q.visit[0]) return true;
  if (!(Q.refine_flags & kRefineBase) || Q.parent[u] == 0xFF) return false;
  return Q.esrc[Q.pedge[u]] == u;  // edge u -> parent: the parent's in-edges would be needed
}
__device__ __forceinline__ uint32_t filter_items(const DevGraph &G, const DQuery &Q) {
  if (Q.status != QS_OK || Q.nvisit == 0) return 0;
  uint32_t n = 0;
  for (uint32_t u = 0; u < Q.k; ++u)
    if (filled_by_filter(Q, u)) n += vertex_filter_items(G, Q, u);
  return n;
}

// The typed path tests each vertex of u's type list (type and binding known
// to pass) against the degree signatures and the neighbour-type masks, read
// from the type-ordered planes (contiguous for consecutive list positions).
// The neighbour-type test: for every edge of u to a typed vertex w, the
// vertex's neighbours over the edge's relation and direction include one
// whose type matches w's modulo 32.  Every candidate exploration keeps
// passes it, so applying it to the first visited vertex in the filter
// changes no set after the first exploration step; it only spares the
// exploration the candidates that fail.

// OR `bits` into level-0 word w0, raising the summary bits when the word was empty.
__device__ __forceinline__ void word_or(const Wave &W, uint32_t *slot, uint32_t w0, uint32_t bits) {
  const uint32_t old = atomicOr(&slot[w0], bits);
  if (old == 0) {
    const uint32_t old1 = atomicOr(&slot[W.G.W0 + (w0 >> 5)], 1u << (w0 & 31));
    if (old1 == 0) atomicOr(&slot[W.G.W0 + W.G.W1 + (w0 >> 15)], 1u << ((w0 >> 10) & 31));
  }
}

__global__ void __launch_bounds__(kThreads) k_filter(Wave W) {
  gdc_wait();
  const DevGraph &G = W.G;
  auto warp = cg::tiled_partition<32>(cg::this_thread_block());
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = gthreads() / 32;
  const uint64_t items = W.fscan[W.nq];
  uint64_t acc = 0;
  for (uint64_t it = gtid() / 32; it < items; it += warps) {
    const uint32_t qi = tile_seg<32>(warp, W.nq, it, [&](uint32_t s) { return W.fscan[s]; });
    const DQuery &Q = W.dq[qi];
    if (Q.status != QS_OK) continue;
    uint32_t u = Q.visit[0];
    uint32_t j = (uint32_t)(it - W.fscan[qi]);
    if (Q.refine_flags & kRefineBase) {  // item j of the filled vertices in index order
      for (uint32_t x = 0; x < Q.k; ++x) {
        if (!filled_by_filter(Q, x)) continue;
        const uint32_t n = vertex_filter_items(G, Q, x);
        u = x;
        if (j < n) break;
        j -= n;
      }
    }
    uint32_t *slot = slot_of(W, Q.qv_base + u);
    const uint32_t nneed = Q.need_begin[u + 1] - Q.need_begin[u];
    if (Q.vbind[u] != kUnbound) {
      if (lane == 0 && cand_ok(G, Q, u, Q.vbind[u])) bit_set(W, slot, Q.vbind[u]);
      if (lane == 0) acc += 4 + nneed;
      continue;
    }
    if (Q.vtype[u] != kAny) {
      // 32 rounds of 32 consecutive type-list entries; the ids ascend, so the
      // lanes that share a level-0 word are contiguous: a segmented OR over
      // them leaves one atomic per touched word
      // Four rounds at a time: every test's loads for the four rounds are
      // issued together (the entries' ids, each degree need's signature
      // word, each typed neighbour's mask), then the four segmented ORs.
      const uint32_t t = Q.vtype[u];
      const uint32_t b0 = G.toff[t] + j * 1024, e0 = min(b0 + 1024, G.toff[t + 1]);
      const bool masks = !W.c0_only && !(Q.refine_flags & kRefineBase);
      for (uint32_t x0 = b0; x0 < e0; x0 += 128) {
        uint32_t v[4];
        bool ok[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t x = x0 + 32 * q + lane;
          ok[q] = x < e0;
          v[q] = ok[q] ? G.tvid[x] : 0u;
        }
        for (uint32_t i = Q.need_begin[u]; i < Q.need_begin[u + 1]; ++i) {
          const uint32_t *plane = G.sig_t + (uint64_t)Q.need_plane[i] * G.sig_words;
          const uint32_t c = Q.need_cnt[i];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t x = x0 + 32 * q + lane;
            if (ok[q]) ok[q] = ((plane[x >> 3] >> ((x & 7) * 4)) & 15u) >= c;
          }
        }
        for (uint32_t i = Q.inc_begin[u]; i < Q.inc_begin[u + 1] && masks; ++i) {
          const uint32_t xi = Q.xinc[i];
          const uint32_t tw = Q.vtype[xinc_w(xi)];
          if (tw == kAny) continue;
          const uint32_t *mp = G.tmask_t + (uint64_t)sig_plane(xinc_dir(xi), xinc_rel(xi), G.R) * G.V;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t x = x0 + 32 * q + lane;
            if (ok[q]) ok[q] = (mp[x] >> (tw & 31u)) & 1u;
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t x = x0 + 32 * q + lane;
          const uint32_t w = x < e0 ? v[q] >> 5 : 0xFFFFFFFFu;
          uint32_t bits = ok[q] && wmask_ok(Q, u, v[q]) ? 1u << (v[q] & 31) : 0u;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_down_sync(kFull, bits, o);
            const uint32_t w2 = __shfl_down_sync(kFull, w, o);
            if (lane + o < 32 && w2 == w) bits |= y;
          }
          const uint32_t wp = __shfl_up_sync(kFull, w, 1);
          if ((lane == 0 || wp != w) && w != 0xFFFFFFFFu && bits) word_or(W, slot, w, bits);
        }
      }
      if (lane == 0) acc += (uint64_t)(e0 - b0) * (4 + nneed);
      continue;
    }
    const uint32_t w1 = j;
    const uint32_t w0 = w1 * 32 + lane;
    uint32_t word = 0;
    if (w0 < G.W0) {
      const uint32_t v0 = w0 * 32;
      uint32_t ok = 0xFFFFFFFFu;
      for (uint32_t i = Q.need_begin[u]; i < Q.need_begin[u + 1] && ok; ++i) {
        // eight 4-bit counts per word: even and odd nibbles compared as
        // bytes, then interleaved back into vertex order
        const uint4 s = *reinterpret_cast<const uint4 *>(G.sig + (uint64_t)Q.need_plane[i] * G.sig_words + (uint64_t)w0 * 4);
        uint32_t sw[4] = {s.x, s.y, s.z, s.w};
        const uint32_t cc = Q.need_cnt[i] * 0x01010101u;
        uint32_t m = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t z = __vsetgeu4(sw[q] & 0x0F0F0F0Fu, cc) | (__vsetgeu4((sw[q] >> 4) & 0x0F0F0F0Fu, cc) << 1);
          const uint32_t r = (z & 3u) | ((z >> 6) & 0xCu) | ((z >> 12) & 0x30u) | ((z >> 18) & 0xC0u);
          m |= r << (8 * q);
        }
        ok &= m;
      }
      if (v0 + 32 > G.V) ok &= (G.V - v0 >= 32) ? 0xFFFFFFFFu : ((1u << (G.V - v0)) - 1);
      for (uint32_t m = Q.wmask ? ok : 0u; m; m &= m - 1) {
        const uint32_t b = __ffs(m) - 1;
        if (!wmask_ok(Q, u, v0 + b)) ok &= ~(1u << b);
      }
      word = ok;
      slot[w0] = word;
    }
    uint32_t nz = __ballot_sync(kFull, word != 0);
    if (lane == 0) {
      slot[G.W0 + w1] = nz;
      if (nz) atomicOr(&slot[G.W0 + G.W1 + (w1 >> 10)], 1u << ((w1 >> 5) & 31));
    }
    if (lane == 0) acc += 32ull * 16 * nneed + 32 * 4 + 4;
  }
  flush_bytes(W, KK_FILTER, acc);
}

// ============================================================ compaction
// kernel_collect: the candidate set as a sorted list.  Items are chunks of 32
// summary words (32K vertices) of a selected set; selection mode 0 picks the
// step-th visited vertex of each query, mode 1 every query vertex.
__device__ __forceinline__ bool sel_slot(const Wave &W, int mode, uint32_t step, uint32_t s, uint32_t &gqv) {
  if (mode == 0) {
    const DQuery &Q = W.dq[s];
    if (Q.status != QS_OK || Q.nvisit <= step) return false;
    gqv = Q.qv_base + Q.visit[step];
    return true;
  }
  gqv = s;
  return W.dq[W.qv_q[s]].status == QS_OK;
}

// Items are chunks of 32 summary words (32,768 vertices) of a selected set.
// A chunk whose level-2 bit is clear is skipped after one (cached) word
// load; otherwise the warp loads the chunk's 32 summary words (lane j word
// j) and walks the non-zero ones, lane j taking level-0 word j.  Four items
// per warp iteration keep several summary loads in flight.
constexpr int kCU = 4;

// Compaction items are groups of 32 chunks (one level-2 word) of a set:
// ipg items per set.  A warp reads the group's level-2 word once and visits
// only its non-empty chunks.
__device__ __forceinline__ uint64_t group_items(const Wave &W, int mode) {
  return (uint64_t)(mode == 0 ? W.nq : W.nqv) * W.G.ipg;
}

// Selected set of item `it` and its level-2 word (0 when not selected).
__device__ __forceinline__ uint32_t group_word(const Wave &W, int mode, uint32_t step, uint64_t it, uint32_t &s,
                                               const uint32_t *&slot) {
  const DevGraph &G = W.G;
  s = (uint32_t)(it / G.ipg);
  uint32_t gqv = 0;
  slot = nullptr;
  if (!sel_slot(W, mode, step, s, gqv)) return 0;
  slot = slot_of(W, gqv);
  return slot[G.W0 + G.W1 + (uint32_t)(it % G.ipg)];
}

// Level-0 words of lane `lane`'s level-1 word `sw` in chunk c: eight 16-byte
// loads, issued together, of the quads that hold a set level-1 bit (the
// others read as zero).  Words whose level-1 bit is clear are zeroed, so a
// quad that runs past the last level-0 word counts nothing.
__device__ __forceinline__ void load_l0(const uint32_t *slot, uint32_t c, uint32_t lane, uint32_t sw, uint32_t (&x)[32]) {
  const uint4 *p = reinterpret_cast<const uint4 *>(slot + (uint64_t)(c * 32 + lane) * 32);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    uint4 v = make_uint4(0, 0, 0, 0);
    if ((sw >> (4 * q)) & 0xFu) v = __ldg(p + q);
    x[4 * q] = v.x;
    x[4 * q + 1] = v.y;
    x[4 * q + 2] = v.z;
    x[4 * q + 3] = v.w;
  }
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (!((sw >> i) & 1u)) x[i] = 0;
}

// Level-1 word of lane `lane` in chunk c.
__device__ __forceinline__ uint32_t l1_word(const DevGraph &G, const uint32_t *slot, uint32_t c, uint32_t lane) {
  const uint32_t w1 = c * 32 + lane;
  return w1 < G.W1 ? slot[G.W0 + w1] : 0;
}

// Non-empty chunks of the selected sets as a work list: entry
// (gqv << 32) | (s * nchunks + c) for chunk c of set s (slot gqv).  One warp
// per level-2 word appends its set bits with one atomic; the order of the
// list does not matter (positions come from the scan of the counts).
__global__ void __launch_bounds__(kThreads) k_chunk_list(Wave W, int mode, uint32_t step) {
  gdc_wait();
  const DevGraph &G = W.G;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = gthreads() / 32;
  const uint64_t items = group_items(W, mode);
  if (gtid() == 0) W.ctrl->tlist_top = 0;  // the claim kernel after this one counts from zero
  for (uint64_t it = gtid() / 32; it < items; it += warps) {
    uint32_t s, gqv = 0;
    const uint32_t *slot;
    const uint32_t m = group_word(W, mode, step, it, s, slot);
    // every chunk count of the group starts at zero (the count kernel fills
    // in the listed ones)
    const uint32_t c0 = (uint32_t)(it % G.ipg) * 32 + lane;
    if (c0 < G.nchunks) W.ccount[(uint64_t)s * G.nchunks + c0] = 0;
    if (!m) continue;
    sel_slot(W, mode, step, s, gqv);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd((unsigned long long *)&W.ctrl->len[9], (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, 0);
    if ((m >> lane) & 1u) {
      const uint32_t c = (uint32_t)(it % G.ipg) * 32 + lane;
      W.clist[base + __popc(m & ((1u << lane) - 1))] = ((uint64_t)gqv << 32) | ((uint64_t)s * G.nchunks + c);
    }
  }
}

// Candidates per listed chunk (the list kernel zeroed every count).  Lane j
// owns level-1 word j and counts its level-0 words; the level-1 words of kCU
// chunks are loaded together.
__global__ void __launch_bounds__(kThreads) k_compact_count(Wave W) {
  gdc_wait();
  const DevGraph &G = W.G;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = gthreads() / 32;
  const uint64_t items = W.ctrl->len[9];
  for (uint64_t it0 = (gtid() / 32) * kCU; it0 < items; it0 += warps * kCU) {
    uint64_t e[kCU];
    uint32_t sw[kCU];
#pragma unroll
    for (int u = 0; u < kCU; ++u) {
      e[u] = it0 + u < items ? W.clist[it0 + u] : 0;
      sw[u] = it0 + u < items ? l1_word(G, slot_of(W, (uint32_t)(e[u] >> 32)), (uint32_t)e[u] % G.nchunks, lane) : 0;
    }
#pragma unroll
    for (int u = 0; u < kCU; ++u) {
      if (it0 + u >= items) break;
      const uint32_t ci = (uint32_t)e[u], c = ci % G.nchunks;
      uint32_t cnt = 0;
      if (sw[u]) {
        uint32_t x[32];
        load_l0(slot_of(W, (uint32_t)(e[u] >> 32)), c, lane, sw[u], x);
#pragma unroll
        for (int i = 0; i < 32; ++i) cnt += __popc(x[i]);
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) cnt += __shfl_down_sync(kFull, cnt, o);
      if (lane == 0) W.ccount[ci] = cnt;
    }
  }
}

// The exploration work list of one step in one pass: per listed chunk of a
// query's set, a warp counts the chunk's candidates; the block's warps take
// consecutive chunks of the list and claim places for all of them with one
// atomic, so the list stays grouped by query (the chunk list is in query
// order) and each warp writes its chunk's ids in ascending order with the
// query beside each.  A query whose chunk would pass the list's end is
// marked overflowed, the places of that chunk below the end name it, and
// the size the run asked for is recorded for the pool.
__global__ void __launch_bounds__(kThreads) k_compact_claim(Wave W) {
  gdc_wait();
  __shared__ uint32_t wtot[kThreads / 32];
  __shared__ unsigned long long bbase;
  const DevGraph &G = W.G;
  const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  constexpr uint32_t kWarps = kThreads / 32;
  const uint64_t items = W.ctrl->len[9];
  for (uint64_t it0 = (uint64_t)blockIdx.x * kWarps; it0 < items; it0 += (uint64_t)gridDim.x * kWarps) {  // block-uniform
    const uint64_t it = it0 + wib;
    uint32_t s = 0, c = 0, sw = 0, n = 0;
    const uint32_t *slot = nullptr;
    uint32_t x[32];
    if (it < items) {
      const uint64_t e = W.clist[it];
      const uint32_t ci = (uint32_t)e;
      s = ci / G.nchunks;
      c = ci % G.nchunks;
      slot = slot_of(W, (uint32_t)(e >> 32));
      sw = l1_word(G, slot, c, lane);
      if (sw) {
        load_l0(slot, c, lane, sw, x);
#pragma unroll
        for (int i = 0; i < 32; ++i) n += __popc(x[i]);
      }
    }
    uint32_t incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);  // this warp's chunk
    if (lane == 0) wtot[wib] = total;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long sum = 0;
      for (uint32_t w = 0; w < kWarps; ++w) sum += wtot[w];
      bbase = sum ? atomicAdd((unsigned long long *)&W.ctrl->tlist_top, sum) : 0;
      if (sum) atomicMax((unsigned long long *)&W.ctrl->hw[HW_TLIST], bbase + sum);
    }
    __syncthreads();
    uint64_t base = bbase;
    for (uint32_t w = 0; w < wib; ++w) base += wtot[w];
    __syncthreads();  // wtot and bbase are read before the next round writes them
    if (total == 0) continue;
    if (base + total > W.tlist_cap) {
      if (lane == 0) mark(W.dq[s], QS_OVERFLOW);
      for (uint64_t p = base + lane; p < W.tlist_cap; p += 32) W.tlist_q[p] = s;
      continue;
    }
    if (!sw) continue;
    uint64_t p = base + incl - n;
    const uint32_t id0 = (c * 32 + lane) * 1024;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      uint32_t w = x[i];
      while (w) {
        const int bpos = __ffs(w) - 1;
        w &= w - 1;
        W.tlist_q[p] = s;
        W.tlist[p++] = id0 + i * 32 + bpos;
      }
    }
  }
}

// Writes ids in ascending order at dst[scan[chunk] ...] and, when `owner` is
// given, the set's owner (query for mode 0, global query vertex for mode 1)
// beside each id; marks a query that does not fit dst_cap as overflowed.
// Per listed chunk, lane j writes the ids of level-1 word j after the ids of
// the lanes before it.
__global__ void __launch_bounds__(kThreads) k_compact_write(Wave W, int mode, const uint64_t *scan, uint32_t *dst,
                                                             uint32_t *owner, uint64_t dst_cap, int hw_slot) {
  gdc_wait();
  const DevGraph &G = W.G;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = gthreads() / 32;
  const uint64_t items = W.ctrl->len[9];
  if (gtid() == 0)
    atomicMax((unsigned long long *)&W.ctrl->hw[hw_slot],
              (unsigned long long)scan[(uint64_t)(mode == 0 ? W.nq : W.nqv) * G.nchunks]);
  for (uint64_t it = gtid() / 32; it < items; it += warps) {
    const uint64_t e = W.clist[it];
    const uint32_t ci = (uint32_t)e, s = ci / G.nchunks, c = ci % G.nchunks;
    const uint32_t *slot = slot_of(W, (uint32_t)(e >> 32));
    if (scan[ci + 1] > dst_cap) {
      if (lane == 0) mark(W.dq[mode == 0 ? s : W.qv_q[s]], QS_OVERFLOW);
      // positions of this chunk below the capacity still name their owner,
      // so that every entry a consumer reads below the capacity is defined
      if (owner)
        for (uint64_t p = scan[ci] + lane; p < dst_cap; p += 32) owner[p] = s;
      continue;
    }
    const uint32_t sw = l1_word(G, slot, c, lane);
    uint32_t x[32];
    uint32_t n = 0;
    if (sw) {
      load_l0(slot, c, lane, sw, x);
#pragma unroll
      for (int i = 0; i < 32; ++i) n += __popc(x[i]);
    }
    uint32_t incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (!sw) continue;
    uint64_t p = scan[ci] + incl - n;
    const uint32_t id0 = (c * 32 + lane) * 1024;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      uint32_t w = x[i];
      while (w) {
        const int bpos = __ffs(w) - 1;
        w &= w - 1;
        if (owner) owner[p] = s;
        dst[p++] = id0 + i * 32 + bpos;
      }
    }
  }
}

// ============================================================ explore
// One candidate v (item `it` of the step's list) explored by `tile`'s G lanes.
template <int G>
__device__ __forceinline__ void explore_item(const cg::thread_block_tile<G> &tile, const Wave &W, uint32_t step,
                                             uint64_t it, uint64_t &acc) {
  const DevGraph &Gr = W.G;
  const uint32_t r = tile.thread_rank();
  DQuery &Q = W.dq[W.tlist_q[it]];
  if (Q.status != QS_OK) return;  // no kernel of this step changes a status
  const uint32_t u = Q.visit[step];
  const uint32_t v = W.tlist[it];
  const uint32_t i0 = Q.inc_begin[u], i1 = Q.inc_begin[u + 1];
  uint64_t bytes = 0;
  // every edge to a typed vertex w needs a neighbour of w's type over its
  // relation and direction: the neighbour-type masks of all edges, loaded
  // together, reject most candidates before any row is read (the filter
  // already applied them to the typed, unbound first vertex's candidates)
  bool keep = true;
  const bool masked = step == 0 && Q.vbind[u] == kUnbound && Q.vtype[u] != kAny && !W.c0_only;
  for (uint32_t i = i0; i < i1 && !(Q.refine_flags & kRefineBase) && !masked; ++i) {
    const uint32_t xi = Q.xinc[i];
    const uint32_t t = Q.vtype[xinc_w(xi)];
    if (t == kAny) continue;
    const uint32_t m = Gr.tmask[(uint64_t)sig_plane(xinc_dir(xi), xinc_rel(xi), Gr.R) * Gr.V + v];
    keep = keep && ((m >> (t & 31u)) & 1u);
  }
  bytes += 4ull * (i1 - i0);
  // edges to vertices other than the children initialised by this step
  for (uint32_t i = i0; i < i1 && keep; ++i) {
    const uint32_t xi = Q.xinc[i];
    if (xinc_role(xi) >= 2) continue;  // children below; role 3: not checked (refinement baseline)
    const int dir = adj_plane(xinc_dir(xi), xinc_rel(xi));
    const uint32_t w = xinc_w(xi);
    uint64_t base, lo, hi;
    uint32_t xs;
    const bool fast = rel_run<G>(tile, Gr, dir, v, adj_rel(xinc_rel(xi)), base, lo, hi, xs);
    const bool built = xinc_role(xi) == 1;
    const uint32_t *ws = slot_of(W, Q.qv_base + w);
    bool found = false;
    uint32_t e = run_entry<G>(tile, Gr, dir, fast, base, xs, lo + r, hi);
    uint64_t b = lo;
    for (; b < hi && !found; b += G) {
      const uint64_t j = b + r;
      const uint32_t en = run_entry<G>(tile, Gr, dir, fast, base, xs, j + G, hi);  // the next pass's entry, early
      bool ok = false;
      if (j < hi) {
        const uint32_t x = e & kNbrMask;
        ok = built ? bit_test(ws, x) : cand_ok(Gr, Q, w, x);
      }
      found = tile.any(ok);
      e = en;
    }
    // the run's entries, and per neighbour tested its bitmap word or type byte
    const uint64_t tested = (b < hi ? b : hi) - lo;
    bytes += 16 + 4 * (hi - lo) + tested * (built ? 4 : (Q.vtype[w] != kAny ? 1 : 0));
    if (!found) keep = false;
  }
  // tree edges to the children: test, expand and check existence in one scan
  for (uint32_t i = i0; i < i1 && keep; ++i) {
    const uint32_t xi = Q.xinc[i];
    if (xinc_role(xi) != 2) continue;
    const int dir = adj_plane(xinc_dir(xi), xinc_rel(xi));
    const uint32_t w = xinc_w(xi);
    uint64_t base, lo, hi;
    uint32_t xs;
    const bool fast = rel_run<G>(tile, Gr, dir, v, adj_rel(xinc_rel(xi)), base, lo, hi, xs);
    uint32_t *ws = slot_of(W, Q.qv_base + w);
    uint32_t nset = 0;
    uint32_t e = run_entry<G>(tile, Gr, dir, fast, base, xs, lo + r, hi);
    for (uint64_t b = lo; b < hi; b += G) {
      const uint64_t j = b + r;
      const uint32_t en = run_entry<G>(tile, Gr, dir, fast, base, xs, j + G, hi);  // the next pass's entry, early
      bool ok = false;
      if (j < hi) {
        const uint32_t x = e & kNbrMask;
        ok = cand_ok(Gr, Q, w, x);
        if (ok) bit_set(W, ws, x);
      }
      nset += __popc(tile.ballot(ok));
      e = en;
    }
    // the run's entries, each neighbour's type byte, a bitmap word per bit set
    bytes += 16 + 5 * (hi - lo) - (Q.vtype[w] != kAny ? 0 : hi - lo) + 4ull * nset;
    if (nset == 0) keep = false;
  }
  if (!keep && r == 0) bit_clear(slot_of(W, Q.qv_base + u), v);
  if (r == 0) acc += bytes + 4;
}

// kernel_explore (Algorithm "Candidate nodes initialization"): one tile of G
// lanes per candidate v of the visited vertex u.  v is dropped when some
// query neighbour w of u has no candidate among v's data neighbours over the
// edge's relation and direction (a neighbour whose set is not built yet is
// tested with the candidate test); otherwise v's neighbours that pass the
// candidate test join the sets of u's spanning-tree children.
// The edges to children are scanned once: the candidate test of each
// neighbour both feeds the existence check and sets the child's bit.  They
// are scanned after the other edges, so most dropped candidates expand
// nothing; a candidate dropped by a later child edge may leave extra bits in
// an earlier child's set, which keeps the sets supersets of the exact ones
// (refinement removes them).
// A warp takes 32/G consecutive items; a candidate with a row longer than
// 8G entries in either direction (the thesis gives high-degree vertices a
// whole block) is explored by the whole warp first, so that a hub's long
// relation runs are not walked G entries at a time while the rest of the
// grid waits for them.
template <int G>
__global__ void __launch_bounds__(kThreads, 6) k_explore(Wave W, uint32_t step) {
  gdc_wait();
  const auto warp = cg::tiled_partition<32>(cg::this_thread_block());
  const auto tile = cg::tiled_partition<G>(cg::this_thread_block());
  const DevGraph &Gr = W.G;
  const uint64_t n = W.ctrl->tlist_top;
  const uint64_t items = n < W.tlist_cap ? n : W.tlist_cap;  // entries past the list belong to overflowed queries
  constexpr uint32_t T = 32 / G;
  const uint32_t ti = (threadIdx.x & 31) / G;
  const uint64_t nw = gthreads() / 32;
  uint64_t acc = 0;
  for (uint64_t it0 = (gtid() / 32) * T; it0 < items; it0 += nw * T) {  // uniform in the warp
    const uint64_t it = it0 + ti;
    bool hub = false;
    if (G < 32) {
      if (it < items) {
        const uint32_t v = W.tlist[it];
        const uint64_t lim = 8 * G;
        hub = Gr.off[0][v + 1] - Gr.off[0][v] > lim || Gr.off[1][v + 1] - Gr.off[1][v] > lim;
      }
      uint32_t hm = warp.ballot(hub && tile.thread_rank() == 0);
      while (hm) {
        const uint32_t src = __ffs(hm) - 1;
        hm &= hm - 1;
        explore_item<32>(warp, W, step, warp.shfl(it, src), acc);
      }
    }
    if (it < items && !hub) explore_item<G>(tile, W, step, it, acc);
  }
  flush_bytes(W, KK_EXPLORE, acc);
}

// ============================================================ refine
// refine_node_candidates, one round: every live candidate v of every query
// vertex u keeps its place only if, for every query edge at u, some data
// neighbour of v over that relation and direction is a live candidate of the
// other endpoint.  Rounds repeat until one clears nothing (the fixpoint).
// Variants per query: no refinement; one vertex per launch in reversed order
// (launch `sub` refines rorder[sub]); low-connectivity vertices (at most
// refine_low incident edges) neither refined nor used to refine.
template <int G>
__global__ void __launch_bounds__(kThreads, 6) k_refine(Wave W, uint32_t round, uint32_t sub) {
  gdc_wait();
  if (round > 0 && W.ctrl->changed[round - 1] == 0) return;
  auto tile = cg::tiled_partition<G>(cg::this_thread_block());
  const DevGraph &Gr = W.G;
  const uint32_t r = tile.thread_rank();
  const uint64_t ntile = gthreads() / G;
  const uint64_t items = W.ascan[(uint64_t)W.nqv * Gr.nchunks];
  bool changed = false;
  uint64_t acc = 0;
  for (uint64_t it = gtid() / G; it < items; it += ntile) {
    if (it >= W.alist_cap) break;  // entries past the list belong to overflowed queries
    const uint32_t gqv = W.alist_q[it];
    DQuery &Q = W.dq[W.qv_q[gqv]];
    if (Q.status != QS_OK) continue;
    const uint32_t u = gqv - Q.qv_base;
    if (Q.refine_flags | Q.refine_low | sub) {  // a variant, or a sub-round of the reversed order
      if (Q.refine_flags & kRefineOff) continue;
      const bool mine = (Q.refine_flags & kRefineRev) ? (sub < Q.k && Q.rorder[sub] == u) : (sub == kAllSub || sub == 0);
      if (!mine || (uint32_t)(Q.inc_begin[u + 1] - Q.inc_begin[u]) <= Q.refine_low) continue;
    }
    const uint32_t v = W.alist[it];
    uint32_t *us = slot_of(W, gqv);
    if (!bit_test(us, v)) continue;
    uint64_t bytes = 0;
    for (uint32_t i = Q.inc_begin[u]; i < Q.inc_begin[u + 1]; ++i) {
      const uint32_t xi = Q.xinc[i];
      const uint32_t w = xinc_w(xi);
      if (Q.refine_low && (uint32_t)(Q.inc_begin[w + 1] - Q.inc_begin[w]) <= Q.refine_low) continue;
      const int dir = adj_plane(xinc_dir(xi), xinc_rel(xi));
      uint64_t base, lo, hi;
      uint32_t xs;
      const bool fast = rel_run<G>(tile, Gr, dir, v, adj_rel(xinc_rel(xi)), base, lo, hi, xs);
      const uint32_t *ws = slot_of(W, Q.qv_base + w);
      bool found = false;
      for (uint64_t b = lo; b < hi && !found; b += G) {
        const uint64_t j = b + r;
        const uint32_t e = run_entry<G>(tile, Gr, dir, fast, base, xs, j, hi);
        found = tile.any(j < hi && bit_test(ws, e & kNbrMask));
      }
      bytes += 16 + 4 * (hi - lo);
      if (!found) {
        if (r == 0) bit_clear(us, v);
        changed = true;
        break;
      }
    }
    if (r == 0) acc += bytes + 4;
  }
  if (changed && tile.thread_rank() == 0) W.ctrl->changed[round] = 1;
  flush_bytes(W, KK_REFINE, acc);
}

// Final candidate lists: offsets and lengths per query vertex; a query with
// an empty set has no embedding.
__global__ void k_list_table(Wave W) {
  gdc_wait();
  const uint32_t ipg = W.G.nchunks;
  for (uint64_t g = gtid(); g < W.nqv; g += gthreads()) {
    uint64_t b = W.cscan[g * ipg], e = W.cscan[(g + 1) * ipg];
    W.flist_off[g] = b;
    W.flist_len[g] = (uint32_t)(e - b);
    DQuery &Q = W.dq[W.qv_q[g]];
    if (e == b) mark(Q, QS_EMPTY);
  }
}

// ============================================================ join plan
// Join order (Section 3.3.4, combine_edge_candidates): begin with the vertex
// of fewest candidates, then repeatedly take the vertex with the most edges
// into the joined part (ties: fewer candidates, then lower index).  Each
// query edge is oriented from its earlier-joined endpoint, whose candidates
// key its candidate-edge table.
__global__ void k_join_plan(Wave W) {
  gdc_wait();
  for (uint64_t qi = gtid(); qi < W.nq; qi += gthreads()) {
    DQuery &Q = W.dq[qi];
    const bool ok = Q.status == QS_OK;
    const uint32_t k = Q.k;
    if (ok) {
      uint32_t size[kMaxK];
      for (uint32_t u = 0; u < k; ++u) size[u] = W.flist_len[Q.qv_base + u];
      uint32_t joined = 0;
      for (uint32_t s = 0; s < k; ++s) {
        int best = -1, bl = -1;
        for (uint32_t u = 0; u < k; ++u) {
          if ((joined >> u) & 1u) continue;
          int links = 0;
          for (uint32_t i = Q.inc_begin[u]; i < Q.inc_begin[u + 1]; ++i) {
            uint32_t e = Q.inc_edge[i];
            uint32_t w = Q.esrc[e] == u ? Q.edst[e] : Q.esrc[e];
            links += (joined >> w) & 1u;
          }
          if (s > 0 && links == 0) continue;
          if (best < 0 || links > bl || (links == bl && size[u] < size[best])) { best = (int)u; bl = links; }
        }
        Q.join[s] = (uint8_t)best;
        Q.pos[best] = (uint8_t)s;
        joined |= 1u << best;
      }
    }
    for (uint32_t i = 0; i < Q.kp; ++i) Q.opos[i] = Q.pos[Q.pu[i]];
    for (uint32_t e = 0; e < Q.m; ++e) {
      uint32_t n = 0;
      if (ok) {
        Q.from_src[e] = Q.force_from_src != 0xFF ? Q.force_from_src : (Q.pos[Q.esrc[e]] < Q.pos[Q.edst[e]] ? 1 : 0);
        n = W.flist_len[Q.qv_base + (Q.from_src[e] ? Q.esrc[e] : Q.edst[e])];
      }
      W.ec_nkeys[Q.qe_base + e] = n;
    }
  }
}

// ============================================================ edge tables
// collect_edge_candidates with the two-step output scheme: for query edge e
// keyed by endpoint x (candidates in ascending order), the list of key c
// holds c's data neighbours over e's relation and direction that are
// candidates of the other endpoint y, ascending.
template <int G, bool WRITE>
__global__ void __launch_bounds__(kThreads) k_ec(Wave W) {
  gdc_wait();
  auto tile = cg::tiled_partition<G>(cg::this_thread_block());
  const DevGraph &Gr = W.G;
  const uint32_t r = tile.thread_rank();
  const uint64_t ntile = gthreads() / G;
  const uint64_t items = W.ctrl->len[5];  // clamped to the table capacity by k_ec_limit
  uint64_t acc = 0;
  if (WRITE && gtid() == 0) atomicMax((unsigned long long *)&W.ctrl->hw[HW_EC_VALS], (unsigned long long)W.ec_off[items]);
  for (uint64_t it = gtid() / G; it < items; it += ntile) {
    const uint32_t ge = tile_seg<G>(tile, W.nqe, it, [&](uint32_t s) { return W.ec_key_base[s]; });
    DQuery &Q = W.dq[W.qe_q[ge]];
    if (Q.status != QS_OK) {
      if (!WRITE && r == 0) W.ec_cnt[it] = 0;
      continue;
    }
    const uint32_t e = ge - Q.qe_base;
    const uint32_t x = Q.from_src[e] ? Q.esrc[e] : Q.edst[e];
    const uint32_t y = Q.from_src[e] ? Q.edst[e] : Q.esrc[e];
    const int dir = adj_plane(Q.from_src[e] ? 0 : 1, Q.erel[e]);
    const uint32_t key = W.flist[W.flist_off[Q.qv_base + x] + (it - W.ec_key_base[ge])];
    uint64_t lo, hi;
    rel_range<G>(tile, Gr, dir, key, adj_rel(Q.erel[e]), lo, hi);
    const uint32_t *ys = slot_of(W, Q.qv_base + y);
    if (!WRITE) {
      uint32_t cnt = 0;
      for (uint64_t b = lo; b < hi; b += G) {
        uint64_t j = b + r;
        cnt += __popc(tile.ballot(j < hi && bit_test(ys, Gr.adj[dir][j] & kNbrMask)));
      }
      if (r == 0) {
        W.ec_cnt[it] = cnt;
        acc += 16 + 4 * (hi - lo) + 4 * (uint64_t)((hi - lo + 31) / 32) + 4;
      }
    } else {
      uint64_t p = W.ec_off[it];
      if (W.ec_off[it + 1] > W.ec_vals_cap) {
        if (r == 0) mark(Q, QS_OVERFLOW);
        continue;
      }
      for (uint64_t b = lo; b < hi; b += G) {
        uint64_t j = b + r;
        uint32_t xv = j < hi ? (Gr.adj[dir][j] & kNbrMask) : 0;
        bool ok = j < hi && bit_test(ys, xv);
        uint32_t m = tile.ballot(ok);
        if (ok) W.ec_vals[p + __popc(m & ((1u << r) - 1))] = xv;
        p += __popc(m);
      }
      if (r == 0) acc += 16 + 4 * (hi - lo) + 4 * (W.ec_off[it + 1] - W.ec_off[it]) + 8;
    }
  }
  flush_bytes(W, WRITE ? KK_EC_WRITE : KK_EC_COUNT, acc);
}

// Restore every touched bitmap word to zero (only chunks flagged at level 2
// and words flagged at level 1 are visited), so the slots are clean for the
// next run.
__global__ void __launch_bounds__(kThreads) k_clear(Wave W) {
  gdc_wait();
  const DevGraph &G = W.G;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = gthreads() / 32;
  const uint64_t items = (uint64_t)W.nqv * G.ipg;
  for (uint64_t it = gtid() / 32; it < items; it += warps) {
    const uint32_t gqv = (uint32_t)(it / G.ipg), grp = (uint32_t)(it % G.ipg);
    uint32_t *slot = slot_of(W, gqv);
    uint32_t m2 = slot[G.W0 + G.W1 + grp];
    while (m2) {
      const uint32_t c = grp * 32 + (__ffs(m2) - 1);
      m2 &= m2 - 1;
      const uint32_t w1 = c * 32 + lane;
      const uint32_t sw = w1 < G.W1 ? slot[G.W0 + w1] : 0;
      uint32_t m = __ballot_sync(kFull, sw != 0);
      while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        const uint32_t swj = __shfl_sync(kFull, sw, j);
        if ((swj >> lane) & 1u) slot[(c * 32 + j) * 32 + lane] = 0;
      }
      if (sw) slot[G.W0 + w1] = 0;
    }
    __syncwarp();
    if (lane == 0) slot[G.W0 + G.W1 + grp] = 0;
  }
}

// Queries whose edge-table keys would pass the capacity are sent to the
// fallback path; the item count is clamped so no kernel reads past it.
__global__ void k_ec_limit(Wave W) {
  gdc_wait();
  const uint64_t total = W.ec_key_base[W.nqe];
  for (uint64_t ge = gtid(); ge < W.nqe; ge += gthreads())
    if (W.ec_key_base[ge + 1] > W.ec_items_cap && W.ec_key_base[ge + 1] > W.ec_key_base[ge])
      mark(W.dq[W.qe_q[ge]], QS_OVERFLOW);
  if (gtid() == 0) {
    W.ctrl->len[5] = total < W.ec_items_cap ? total : W.ec_items_cap;
    atomicMax((unsigned long long *)&W.ctrl->hw[HW_EC_ITEMS], (unsigned long long)total);
  }
}

// ============================================================ wave I/O
// Prologue: copy the wave's queries into the slots and reset the control
// block.  The wave index advances in the epilogue, so replaying the same
// captured graph runs the waves in order.
__global__ void k_prologue(Wave W) {
  gdc_wait();
  const WaveDesc D = W.waves[W.ctrl->wave];
  const uint64_t words = sizeof(DQuery) / 4;
  const uint32_t *src = reinterpret_cast<const uint32_t *>(W.all_dq + D.q0);
  uint32_t *dst = reinterpret_cast<uint32_t *>(W.dq);
  for (uint64_t i = gtid(); i < (uint64_t)D.nq * words; i += gthreads()) dst[i] = src[i];
  for (uint64_t g = gtid(); g < W.nqv; g += gthreads()) W.qv_q[g] = W.nq;  // owners come from k_owners
  for (uint64_t g = gtid(); g < W.nqe; g += gthreads()) {
    W.qe_q[g] = W.nq;
    W.ec_nkeys[g] = 0;
  }
  if (gtid() == 0) {
    for (int i = 0; i < 8; ++i)
      if (i >= 3) W.ctrl->len[i] = 0;
    for (uint32_t i = 0; i < kMaxRounds; ++i) W.ctrl->changed[i] = 0;
    W.ctrl->lvl_top = 0;
    W.ctrl->out_top = 0;
    W.ctrl->out_rows_total = 0;
    W.ctrl->max_nvisit = 0;
  }
}

// Owner tables of the wave's query vertices and edges (after the plan has
// rebased each slot's vertex and edge ranges).
__global__ void k_owners(Wave W) {
  gdc_wait();
  for (uint64_t qi = gtid(); qi < W.nq; qi += gthreads()) {
    const DQuery &Q = W.dq[qi];
    W.fcnt[qi] = filter_items(W.G, Q);
    if (Q.status == QS_INVALID && Q.k == 0) continue;
    for (uint32_t u = 0; u < Q.k; ++u) W.qv_q[Q.qv_base + u] = (uint32_t)qi;
    for (uint32_t e = 0; e < Q.m; ++e) W.qe_q[Q.qe_base + e] = (uint32_t)qi;
  }
}

// ============================================================ join
// Level 0: the candidates of join[0] are the first partial embeddings.
__global__ void k_join0_rows(Wave W) {
  gdc_wait();
  for (uint64_t qi = gtid(); qi < W.nq; qi += gthreads()) {
    const DQuery &Q = W.dq[qi];
    QState &S = W.qs[qi];
    S.nxt_rows = Q.status == QS_OK ? W.flist_len[Q.qv_base + Q.join[0]] : 0;
    if (Q.status == QS_OK && Q.k == 1) S.count = S.nxt_rows;
    S.inter_words = 0;
    S.peak_words = 0;
  }
}

// Layout of level `lvl` (rows of width lvl+1), one block over the queries in
// order.  A non-final level goes to level buffer (lvl & 1); a final level
// goes to the output pool when rows are wanted and count <= cap.  Pass 0
// marks queries that do not fit; pass 1 lays out the rest (which then fit).
__device__ __forceinline__ void level_sizes(const Wave &W, uint32_t qi, uint32_t lvl, bool pass0, uint64_t v[4],
                                            bool &to_out, bool &mid) {
  v[0] = v[1] = v[2] = v[3] = 0;
  to_out = mid = false;
  if (qi >= W.nq) return;
  DQuery &Q = W.dq[qi];
  const QState &S = W.qs[qi];
  if (Q.status != QS_OK || Q.k <= lvl) return;
  if (Q.k == lvl + 1) {
    if (Q.mode == GS_COUNT_ONLY || Q.cap == 0) return;
    // More rows than cap are still written (and the smallest cap kept after
    // the sort) while they stay within kOverCap * cap; beyond, the chunked
    // path keeps a running top-cap instead.
    if (S.count > Q.cap && S.count > kOverCap * Q.cap) {
      if (pass0) mark(Q, QS_TOPCAP);
      return;
    }
    to_out = true;
    v[2] = S.nxt_rows;
    v[3] = S.nxt_rows * Q.k;
  } else {
    mid = true;
    v[0] = S.nxt_rows;
    v[1] = S.nxt_rows * (lvl + 1);
  }
}

// Every query's sizes for level lvl, one thread per query; after a count
// pass also the rows produced per query (from the scan of the per-row
// counts), and the current level kept aside as the source of the write pass.
__global__ void k_level_sizes(Wave W, uint32_t lvl) {
  gdc_wait();
  for (uint64_t qi = gtid(); qi < W.nq; qi += gthreads()) {
    if (lvl > 0) {
      QState &S = W.qs[qi];
      S.nxt_rows = S.cur_rows ? W.row_scan[S.cur_row_base + S.cur_rows] - W.row_scan[S.cur_row_base] : 0;
      W.src[qi] = SrcRows{S.cur_row_base, S.cur_rows, S.cur_word_base};
    }
    LevelSize z;
    bool to_out, mid;
    level_sizes(W, (uint32_t)qi, lvl, true, z.v, to_out, mid);
    z.flags = (to_out ? 1u : 0u) | (mid ? 2u : 0u);
    z.pad = 0;
    W.lsz[qi] = z;
  }
  if (gtid() == 0 && lvl > 0) W.ctrl->len[4] = W.ctrl->len[3];
}

// The row allocator of a join level (one block): an exclusive scan of the
// sizes over the queries places every query's rows.  A first pass sends away
// (QS_OVERFLOW) each query that would pass a pool's end and assigns the
// places as if none did; only when some query was sent away does a second
// pass assign the places of the others again.
__global__ void __launch_bounds__(1024) k_level_alloc(Wave W, uint32_t lvl) {
  gdc_wait();
  __shared__ uint64_t sm[4][32];
  __shared__ uint64_t carry[4];
  __shared__ int any_over;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) any_over = 0;
  for (int pass = 0; pass < 2; ++pass) {
    __syncthreads();
    if (pass == 1 && !any_over) break;  // block-uniform: the first pass's places stand
    if (threadIdx.x == 0) {
      carry[0] = 0; carry[1] = 0;
      carry[2] = W.ctrl->out_rows_total; carry[3] = W.ctrl->out_top;
    }
    __syncthreads();
    for (uint32_t base = 0; base < W.nq; base += blockDim.x) {
      const uint32_t qi = base + threadIdx.x;
      uint64_t v[4] = {0, 0, 0, 0}, ex[4];
      uint32_t flags = 0;
      if (qi < W.nq) {
        const LevelSize &z = W.lsz[qi];
        flags = z.flags;
        if (!(flags & 4u))
          for (int a = 0; a < 4; ++a) v[a] = z.v[a];
      }
      const bool to_out = flags & 1u, mid = flags & 2u;
      for (int a = 0; a < 4; ++a) {
        uint64_t x = v[a];
        for (int o = 1; o < 32; o <<= 1) {
          uint64_t y = __shfl_up_sync(kFull, x, o);
          if (lane >= o) x += y;
        }
        if (lane == 31) sm[a][warp] = x;
        ex[a] = x - v[a];
      }
      __syncthreads();
      if (warp < 4) {
        uint64_t x = sm[warp][lane];
        for (int o = 1; o < 32; o <<= 1) {
          uint64_t y = __shfl_up_sync(kFull, x, o);
          if (lane >= o) x += y;
        }
        sm[warp][lane] = x;
      }
      __syncthreads();
      uint64_t pos[4];
      for (int a = 0; a < 4; ++a) pos[a] = carry[a] + ex[a] + (warp ? sm[a][warp - 1] : 0);
      if (qi < W.nq) {
        if (pass == 0) {
          const bool over = (mid && (pos[0] + v[0] > W.row_cap || pos[1] + v[1] > W.lvl_words)) ||
                            (to_out && (pos[2] + v[2] > W.out_rows_cap || pos[3] + v[3] > W.out_words));
          if (over) {
            mark(W.dq[qi], QS_OVERFLOW);
            W.lsz[qi].flags = flags | 4u;
            any_over = 1;
          }
          QState &S = W.qs[qi];  // the places if no query is sent away
          S.cur_row_base = pos[0];
          S.cur_word_base = pos[1];
          S.cur_rows = over ? 0 : v[0];
          if (to_out && !over) {
            S.out_row_base = pos[2];
            S.out_word_base = pos[3];
            S.out_rows = v[2];
          }
        } else {
          QState &S = W.qs[qi];
          S.cur_row_base = pos[0];
          S.cur_word_base = pos[1];
          S.cur_rows = v[0];
          if (mid && !(flags & 4u)) {
            S.inter_words += v[1];
            S.peak_words = max(S.peak_words, v[1]);
          }
          if (to_out && !(flags & 4u)) {
            S.out_row_base = pos[2];
            S.out_word_base = pos[3];
            S.out_rows = v[2];
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0)
        for (int a = 0; a < 4; ++a) carry[a] += sm[a][31];
      __syncthreads();
    }
    if (pass == 0 && threadIdx.x == 0) {  // what this level asked for before any query was sent away
      atomicMax((unsigned long long *)&W.ctrl->hw[HW_ROWS], (unsigned long long)carry[0]);
      atomicMax((unsigned long long *)&W.ctrl->hw[HW_LVL_WORDS], (unsigned long long)carry[1]);
      atomicMax((unsigned long long *)&W.ctrl->hw[HW_OUT_ROWS], (unsigned long long)carry[2]);
      atomicMax((unsigned long long *)&W.ctrl->hw[HW_OUT_WORDS], (unsigned long long)carry[3]);
    }
    __syncthreads();
  }
  if (!any_over)  // block-uniform; the second pass counted them otherwise
    for (uint32_t qi = threadIdx.x; qi < W.nq; qi += blockDim.x) {
      const LevelSize &z = W.lsz[qi];
      if (!(z.flags & 2u)) continue;
      QState &S = W.qs[qi];
      S.inter_words += z.v[1];
      S.peak_words = max(S.peak_words, z.v[1]);
    }
  if (threadIdx.x == 0) {
    W.ctrl->len[3] = carry[0];
    W.ctrl->out_rows_total = carry[2];
    W.ctrl->out_top = carry[3];
  }
}

// Level-0 rows (final rows when k == 1), one block per query.
__global__ void k_join0_write(Wave W) {
  gdc_wait();
  for (uint64_t qi = blockIdx.x; qi < W.nq; qi += gridDim.x) {
    const DQuery &Q = W.dq[qi];
    QState &S = W.qs[qi];
    if (Q.status != QS_OK) continue;
    const uint32_t j0 = Q.join[0];
    const uint64_t n = W.flist_len[Q.qv_base + j0];
    const uint32_t *lst = W.flist + W.flist_off[Q.qv_base + j0];
    const bool final = Q.k == 1;
    uint64_t fp = 0;
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t v = lst[i];
      if (final) {
        fp += mix64((uint64_t)1 ^ ((uint64_t)v + 0x9E3779B97F4A7C15ull));
        if (S.out_rows) {
          W.out[S.out_word_base + i] = v;
          W.out_q[S.out_row_base + i] = (uint32_t)qi;
        }
      } else {
        W.lvl[0][S.cur_word_base + i] = v;
      }
    }
    if (final) {
      for (int o = 16; o; o >>= 1) fp += __shfl_down_sync(kFull, fp, o);
      if ((threadIdx.x & 31) == 0 && fp) atomicAdd((unsigned long long *)&S.fp, (unsigned long long)fp);
    }
  }
}

// Candidates for the next vertex w = join[s+1] of one partial row: the
// candidate-edge table of every query edge between w and the joined part is
// looked up by the joined endpoint's id; the shortest list drives and the
// others are probed (sorted-list intersection); ids already in the row are
// skipped (injectivity).
struct JoinCtx {
  uint32_t w, nedge, drive;
  const uint32_t *lst[kMaxK];
  uint32_t len[kMaxK];
};

__device__ __forceinline__ bool join_setup(const Wave &W, const DQuery &Q, uint32_t s, const uint32_t *row, JoinCtx &c) {
  c.w = Q.join[s + 1];
  c.nedge = 0;
  c.drive = 0;
  uint64_t best = ~0ull;
  for (uint32_t i = Q.inc_begin[c.w]; i < Q.inc_begin[c.w + 1]; ++i) {
    const uint32_t e = Q.inc_edge[i];
    const uint32_t x = Q.esrc[e] == c.w ? Q.edst[e] : Q.esrc[e];
    if (Q.pos[x] > s) continue;
    const uint32_t gx = Q.qv_base + x;
    const int64_t t = list_find(W.flist + W.flist_off[gx], W.flist_len[gx], row[Q.pos[x]]);
    if (t < 0) return false;
    const uint64_t item = W.ec_key_base[Q.qe_base + e] + (uint64_t)t;
    const uint64_t b = W.ec_off[item], en = W.ec_off[item + 1];
    c.lst[c.nedge] = W.ec_vals + b;
    c.len[c.nedge] = (uint32_t)(en - b);
    if (en - b < best) { best = en - b; c.drive = c.nedge; }
    c.nedge++;
  }
  return c.nedge > 0;
}

__device__ __forceinline__ bool join_ok(const JoinCtx &c, const uint32_t *row, uint32_t s, uint32_t cand) {
  for (uint32_t i = 0; i <= s; ++i)
    if (row[i] == cand) return false;
  for (uint32_t j = 0; j < c.nedge; ++j)
    if (j != c.drive && !list_has(c.lst[j], c.len[j], cand)) return false;
  return true;
}

__device__ __forceinline__ uint32_t seg_of_src(const SrcRows *src, uint32_t nq, uint64_t item) {
  uint32_t lo = 0, hi = nq;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (src[mid].row_base <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// Count pass of level s -> s+1; a query whose last vertex is w also adds its
// embeddings and their hashes to its count and fingerprint here.
template <int G>
__global__ void __launch_bounds__(kThreads) k_join_count(Wave W, uint32_t s) {
  gdc_wait();
  auto tile = cg::tiled_partition<G>(cg::this_thread_block());
  const uint32_t r = tile.thread_rank();
  const uint64_t ntile = gthreads() / G;
  const uint64_t items = W.ctrl->len[3];
  const uint32_t *lvl = W.lvl[s & 1];
  uint64_t acc = 0;
  uint32_t run_q = 0xFFFFFFFFu;
  uint64_t run_cnt = 0, run_fp = 0;
  auto flush_run = [&]() {
    if (run_q == 0xFFFFFFFFu) return;
    QState &R = W.qs[run_q];
    if (run_cnt) atomicAdd((unsigned long long *)&R.count, (unsigned long long)run_cnt);
    if (run_fp) atomicAdd((unsigned long long *)&R.fp, (unsigned long long)run_fp);
    run_cnt = run_fp = 0;
  };
  for (uint64_t it = gtid() / G; it < items; it += ntile) {
    const uint32_t qi = tile_seg<G>(tile, W.nq, it, [&](uint32_t s) { return W.qs[s].cur_row_base; });
    const DQuery &Q = W.dq[qi];
    QState &S = W.qs[qi];
    uint32_t cnt = 0;
    uint64_t fp = 0, bytes = 0;
    const bool live = Q.status == QS_OK && it < S.cur_row_base + S.cur_rows;
    if (live) {
      const uint32_t *row = lvl + S.cur_word_base + (it - S.cur_row_base) * (s + 1);
      JoinCtx c;
      if (join_setup(W, Q, s, row, c)) {
        const bool final = Q.k == s + 2;
        const uint32_t *d = c.lst[c.drive];
        for (uint32_t j = r; j < c.len[c.drive]; j += G) {
          const uint32_t cand = d[j];
          if (join_ok(c, row, s, cand)) {
            cnt++;
            if (final) fp += row_hash(Q, row, c.w, cand);
          }
        }
        bytes = 4ull * (s + 1) + 4ull * c.len[c.drive] + 24ull * c.nedge;
      }
    }
    for (int o = G / 2; o; o >>= 1) {
      cnt += tile.shfl_down(cnt, o);
      fp += tile.shfl_down(fp, o);
    }
    if (r == 0) {
      W.row_cnt[it] = cnt;
      if (live && Q.k == s + 2 && (cnt || fp)) {
        // a query's final embeddings are summed in registers while the
        // tile's items stay in that query, then added with one atomic pair
        if (run_q != qi) {
          flush_run();
          run_q = qi;
        }
        run_cnt += cnt;
        run_fp += fp;
      }
      acc += bytes;
    }
  }
  if (r == 0) flush_run();
  flush_bytes(W, KK_JOIN_COUNT, acc);
}

// Write pass of level s -> s+1 into the layout made by k_level_alloc.
template <int G>
__global__ void __launch_bounds__(kThreads) k_join_write(Wave W, uint32_t s) {
  gdc_wait();
  auto tile = cg::tiled_partition<G>(cg::this_thread_block());
  const uint32_t r = tile.thread_rank();
  const uint64_t ntile = gthreads() / G;
  const uint64_t items = W.ctrl->len[4];
  const uint32_t *lvl = W.lvl[s & 1];
  uint32_t *nxt = W.lvl[(s + 1) & 1];
  uint64_t acc = 0;
  for (uint64_t it = gtid() / G; it < items; it += ntile) {
    const uint32_t qi = tile_seg<G>(tile, W.nq, it, [&](uint32_t s) { return W.src[s].row_base; });
    const DQuery &Q = W.dq[qi];
    const QState &S = W.qs[qi];
    const SrcRows R = W.src[qi];
    if (Q.status != QS_OK || it >= R.row_base + R.rows) continue;
    const bool final = Q.k == s + 2;
    const uint32_t width = s + 2;
    uint32_t *dst;
    uint64_t rbase;
    if (final) {
      if (S.out_rows == 0) continue;
      dst = W.out + S.out_word_base;
      rbase = S.out_row_base;
    } else {
      dst = nxt + S.cur_word_base;
      rbase = 0;
    }
    const uint32_t *row = lvl + R.word_base + (it - R.row_base) * (s + 1);
    uint64_t p = W.row_scan[it] - W.row_scan[R.row_base];
    JoinCtx c;
    if (!join_setup(W, Q, s, row, c)) continue;
    const uint32_t *d = c.lst[c.drive];
    uint64_t written = 0;
    for (uint32_t b = 0; b < c.len[c.drive]; b += G) {
      const uint32_t j = b + r;
      const uint32_t cand = j < c.len[c.drive] ? d[j] : 0;
      const bool ok = j < c.len[c.drive] && join_ok(c, row, s, cand);
      const uint32_t m = tile.ballot(ok);
      if (ok) {
        const uint64_t at = p + __popc(m & ((1u << r) - 1));
        uint32_t *o = dst + at * width;
        for (uint32_t i = 0; i <= s; ++i) o[i] = row[i];
        o[s + 1] = cand;
        if (final && W.out_q) W.out_q[rbase + at] = qi;
      }
      p += __popc(m);
      written += __popc(m);
    }
    if (r == 0) acc += 4ull * written * width + 4ull * (s + 1) + 4ull * c.len[c.drive] + 24ull * c.nedge;
  }
  flush_bytes(W, KK_JOIN_WRITE, acc);
}

// Query-order layout of the sorted rows, and of the rows of queries whose
// output is too large for the one-block sort (sorted by the merge path).
__device__ __forceinline__ bool small_output(const DQuery &, const QState &S) { return S.out_rows <= kSmallRows; }

__global__ void __launch_bounds__(1024) k_final_bases(Wave W) {
  gdc_wait();
  __shared__ uint64_t sm[4][32];
  __shared__ uint64_t carry[4];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 4) carry[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    W.ctrl->max_large_rows = 0;
    W.ctrl->over_cap = 0;
  }
  __syncthreads();
  for (uint32_t base = 0; base < W.nq; base += blockDim.x) {
    const uint32_t qi = base + threadIdx.x;
    uint64_t v[4] = {0, 0, 0, 0}, ex[4];
    if (qi < W.nq && W.dq[qi].status == QS_OK) {
      const uint64_t keep = min(W.qs[qi].out_rows, W.dq[qi].cap);  // rows returned (at most)
      v[0] = keep;
      v[1] = keep * W.dq[qi].kp;
      v[2] = small_output(W.dq[qi], W.qs[qi]) ? 0 : W.qs[qi].out_rows;
      v[3] = (v[2] + kTileRows - 1) / kTileRows;
      if (v[2]) atomicMax((unsigned long long *)&W.ctrl->max_large_rows, (unsigned long long)v[2]);
    }
    if (qi < W.nq) {
      W.qs[qi].sort_rows = v[2];
      W.qs[qi].nfinal = v[0];  // projected queries replace it once duplicates are dropped
      W.qs[qi].more = 0;
      // a projected output is never cut before sorting: the cap-th distinct
      // tuple can lie past the cap-th row
      const bool over = v[2] > W.dq[qi].cap && !W.dq[qi].proj;
      W.sel[qi] = SelState{~0ull, 0, 0, W.dq[qi].cap, ~0ull, 0, 0, 0, 0, over ? 1u : 0u};
      if (over) atomicAdd((unsigned long long *)&W.ctrl->over_cap, 1ull);
    }
    for (int a = 0; a < 4; ++a) {
      uint64_t x = v[a];
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) sm[a][warp] = x;
      ex[a] = x - v[a];
    }
    __syncthreads();
    if (warp < 4) {
      uint64_t x = sm[warp][lane];
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      sm[warp][lane] = x;
    }
    __syncthreads();
    if (qi < W.nq) {
      W.qs[qi].fin_row_base = carry[0] + ex[0] + (warp ? sm[0][warp - 1] : 0);
      W.qs[qi].fin_word_base = carry[1] + ex[1] + (warp ? sm[1][warp - 1] : 0);
      W.qs[qi].lrg_row_base = carry[2] + ex[2] + (warp ? sm[2][warp - 1] : 0);
      W.qs[qi].lrg_tile_base = carry[3] + ex[3] + (warp ? sm[3][warp - 1] : 0);
    }
    __syncthreads();
    if (threadIdx.x < 4) carry[threadIdx.x] += sm[threadIdx.x][31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    W.ctrl->len[6] = carry[2];
    W.ctrl->len[7] = carry[3];
    W.ctrl->fin_words = carry[1];
  }
}

// ============================================================ sort + gather
// Large outputs (more than the one-block limit) are sorted as a merge sort
// of (key, row index) pairs.  The key packs the row's output columns in
// query-vertex order at the graph's id width into two words: the first
// holds the leading columns (the first column in the top bits; the column
// that does not fit whole contributes its top bits), the second the columns
// from that one on.  Key order is row order on those bits, and only equal
// keys compare full rows (never when the two words hold every column).
// Each block first sorts one tile of kTileRows rows of one query in shared
// memory (bitonic network); merge passes then double the sorted runs within
// each query, one partition kernel placing every output tile's split and one
// merge kernel per pass moving contiguous slices.
__device__ __forceinline__ uint32_t seg_of_large(const QState *qs, uint32_t nq, uint64_t item, bool tiles) {
  uint32_t lo = 0, hi = nq;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if ((tiles ? qs[mid].lrg_tile_base : qs[mid].lrg_row_base) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// Key of a row whose column of query vertex u is x[pos(u)].
template <class Col>
__device__ __forceinline__ uint64_t pack_key(uint32_t k, uint32_t b, Col col) {
  uint64_t key = 0;
  uint32_t used = 0;
  for (uint32_t u = 0; u < k && used < 64; ++u) {
    const uint64_t c = col(u);
    if (used + b <= 64) {
      key |= c << (64 - used - b);
      used += b;
    } else {
      key |= c >> (b - (64 - used));
      used = 64;
    }
  }
  return key;
}

// Output columns the two sort-key words hold whole: rows with equal keys
// agree on them.
__device__ __forceinline__ uint32_t key_cols(const Wave &W) { return 2 * (64 / W.G.idbits); }

// Row r of the output pool (query qi) compared on its output columns (the
// projected vertices, or every vertex) in query-vertex order.  Callers
// compare rows only when their sort keys are equal, so the columns the keys
// hold whole are skipped.
__device__ __forceinline__ bool out_row_le(const Wave &W, const DQuery &Q, const QState &S, uint32_t a, uint32_t b) {
  const uint32_t *x = W.out + S.out_word_base + (uint64_t)(a - S.out_row_base) * Q.k;
  const uint32_t *y = W.out + S.out_word_base + (uint64_t)(b - S.out_row_base) * Q.k;
  for (uint32_t i = key_cols(W); i < Q.kp; ++i) {
    const uint32_t c = Q.opos[i];
    const uint32_t xa = x[c], yb = y[c];
    if (xa != yb) return xa < yb;
  }
  return true;
}

// Do rows a and b of the output pool, with equal sort keys, agree on every
// output column?
__device__ __forceinline__ bool out_row_eq(const Wave &W, const DQuery &Q, const QState &S, uint32_t a, uint32_t b) {
  const uint32_t *x = W.out + S.out_word_base + (uint64_t)(a - S.out_row_base) * Q.k;
  const uint32_t *y = W.out + S.out_word_base + (uint64_t)(b - S.out_row_base) * Q.k;
  for (uint32_t i = key_cols(W); i < Q.kp; ++i)
    if (x[Q.opos[i]] != y[Q.opos[i]]) return false;
  return true;
}

// (ka, a) <= (kb, b): keys first, the rows on equal keys.
// Do the two key words hold every output column whole?
__device__ __forceinline__ bool keys_exact(const Wave &W, const DQuery &Q) { return Q.kp <= 2 * (64 / W.G.idbits); }

__device__ __forceinline__ bool kr_le(const Wave &W, const DQuery &Q, const QState &S, SortKey ka, uint32_t ra,
                                      SortKey kb, uint32_t rb) {
  if (ka != kb) return ka < kb;
  return keys_exact(W, Q) || out_row_le(W, Q, S, ra, rb);
}

// The sort key of a row whose output column c is col(c).
template <class Col>
__device__ __forceinline__ SortKey sort_key(uint32_t kp, uint32_t b, Col col) {
  const uint32_t f = 64 / b;
  SortKey k;
  k.hi = pack_key(kp, b, col);
  k.lo = kp > f ? pack_key(kp - f, b, [&](uint32_t c) { return col(f + c); }) : 0;
  return k;
}

// Exclusive scan of v[0..n) in shared memory by one block of 256 threads,
// each taking n / 256 consecutive entries (n a multiple of 256 up to 2048);
// returns the total.
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t *v, uint32_t n) {
  __shared__ uint32_t wsum[8];
  __shared__ uint32_t total;
  const uint32_t per = n / 256, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *mine = v + threadIdx.x * per;
  uint32_t sum = 0;
  for (uint32_t j = 0; j < per; ++j) sum += mine[j];
  uint32_t x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int w = 0; w < 8; ++w) {
      const uint32_t t = wsum[w];
      wsum[w] = acc;
      acc += t;
    }
    total = acc;
  }
  __syncthreads();
  uint32_t run = wsum[warp] + x - sum;
  for (uint32_t j = 0; j < per; ++j) {
    const uint32_t t = mine[j];
    mine[j] = run;
    run += t;
  }
  const uint32_t tot = total;
  __syncthreads();
  return tot;
}

// One block sorts one query's rows: the two-word packed keys of the rows
// (see the large-output sort below) and row indices in shared memory,
// bitonic network, full rows compared on equal keys only; then the first `cap` rows
// are written in query-vertex column order.  A projected query keeps only
// the first row of each run of equal projected tuples (its rank among the
// runs from a block scan) and writes the first `cap` of them.
__global__ void __launch_bounds__(256) k_small_sort(Wave W) {
  gdc_wait();
  __shared__ uint64_t key[kSmallRows];
  __shared__ uint64_t key2[kSmallRows];  // the columns from the first one key does not hold whole
  __shared__ uint32_t idx[kSmallRows];
  const uint32_t b = W.G.idbits;
  const uint32_t f = 64 / b;  // output columns held whole by one key word
  for (uint32_t qi = blockIdx.x; qi < W.nq; qi += gridDim.x) {
    const DQuery &Q = W.dq[qi];
    const QState &S = W.qs[qi];
    const uint32_t n = (uint32_t)S.out_rows, k = Q.k;
    if (Q.status != QS_OK || n == 0 || !small_output(Q, S)) continue;
    const uint32_t *rows = W.out + S.out_word_base;
    const uint32_t r0 = (uint32_t)S.out_row_base;
    uint32_t np2 = 1;
    while (np2 < n) np2 <<= 1;
    const uint32_t kp = Q.kp;
    const bool exact = kp <= 2 * f;  // the two key words decide every comparison
    for (uint32_t i = threadIdx.x; i < np2; i += blockDim.x) {
      idx[i] = i;
      if (i < n) {
        const uint32_t *x = rows + (uint64_t)i * k;
        key[i] = pack_key(kp, b, [&](uint32_t c) { return x[Q.opos[c]]; });
        key2[i] = kp > f ? pack_key(kp - f, b, [&](uint32_t c) { return x[Q.opos[f + c]]; }) : 0;
      }
    }
    __syncthreads();
    auto less = [&](uint32_t a, uint32_t c) {
      if (a >= n) return false;
      if (c >= n) return true;
      if (key[a] != key[c]) return key[a] < key[c];
      if (key2[a] != key2[c]) return key2[a] < key2[c];
      return !exact && !out_row_le(W, Q, S, r0 + c, r0 + a);
    };
    for (uint32_t size = 2; size <= np2; size <<= 1)
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t x = threadIdx.x; x < np2 / 2; x += blockDim.x) {
          const uint32_t i = 2 * x - (x & (stride - 1)), p = i + stride;
          const bool up = (i & size) == 0;
          const uint32_t a = idx[i], c = idx[p];
          if (up ? less(c, a) : less(a, c)) { idx[i] = c; idx[p] = a; }
        }
        __syncthreads();
      }
    uint32_t *dst = W.out_final + S.fin_word_base;
    if (!Q.proj) {
      const uint32_t keep = (uint32_t)min((uint64_t)n, Q.cap);
      for (uint32_t t = threadIdx.x; t < keep * k; t += blockDim.x) {
        const uint32_t i = t / k, u = t % k;
        dst[t] = rows[(uint64_t)idx[i] * k + Q.pos[u]];
      }
      __syncthreads();
      continue;
    }
    // run starts marked in bit 31 of idx (entries are below kSmallRows; a
    // neighbour's read masks the bit, so marking in place is safe); then the
    // keys are done with and their space holds the ranks
    constexpr uint32_t kMark = 0x80000000u;
    const uint32_t nr = (np2 + 255) / 256 * 256;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t a = idx[i] & ~kMark, p = i ? idx[i - 1] & ~kMark : 0;
      if (i == 0 || key[a] != key[p] || key2[a] != key2[p] || (!exact && !out_row_eq(W, Q, S, r0 + a, r0 + p)))
        idx[i] = a | kMark;
    }
    __syncthreads();
    uint32_t *rnk = reinterpret_cast<uint32_t *>(key);
    for (uint32_t i = threadIdx.x; i < nr; i += blockDim.x) rnk[i] = i < n ? idx[i] >> 31 : 0;
    __syncthreads();
    const uint32_t d = block_scan_excl(rnk, nr);  // distinct tuples
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t r = rnk[i];
      if (!(idx[i] & kMark) || r >= Q.cap) continue;  // not a run start, or past cap
      const uint32_t *x = rows + (uint64_t)(idx[i] & ~kMark) * k;
      for (uint32_t c = 0; c < kp; ++c) dst[(uint64_t)r * kp + c] = x[Q.opos[c]];
    }
    if (threadIdx.x == 0) {
      W.qs[qi].nfinal = min((uint64_t)d, Q.cap);
      W.qs[qi].more = d > Q.cap;
    }
    __syncthreads();
  }
}

// Sort keys of every large row, in query order (row i of a query at
// lrg_row_base + i); for a query to be cut at cap, the smallest and largest
// key (one atomic per warp when the warp's rows share a query).
// A warp whose 32 rows belong to one query first copies their words into
// shared memory with coalesced loads (rows are contiguous there), then each
// lane builds its row's key from shared memory.
__global__ void __launch_bounds__(256) k_sort_keys(Wave W, uint32_t *perm, SortKey *keys) {
  gdc_wait();
  __shared__ uint32_t stage[256 / 32][32 * kMaxK];
  const uint64_t n = W.ctrl->len[6];
  const uint32_t b = W.G.idbits, lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint64_t acc = 0;
  for (uint64_t base = gtid() - lane; base < n; base += gthreads()) {
    const uint64_t i = base + lane;
    uint32_t qi = 0xFFFFFFFFu;
    uint64_t key = 0;
    if (i < n) {
      qi = seg_of_large(W.qs, W.nq, i, false);
      acc += 4ull * W.dq[qi].k + 20;  // the row read, its key and index written
    }
    const uint32_t q0 = __shfl_sync(kFull, qi, 0);
    if (__all_sync(kFull, i >= n || qi == q0)) {  // warp-uniform
      const DQuery &Q = W.dq[q0];
      const QState &S = W.qs[q0];
      const uint64_t local0 = base - S.lrg_row_base;
      const uint32_t rows = (uint32_t)(n - base < 32 ? n - base : 32), words = rows * Q.k;
      const uint32_t *src = W.out + S.out_word_base + local0 * Q.k;
      for (uint32_t w = lane; w < words; w += 32) stage[wib][w] = src[w];
      __syncwarp();
      if (i < n) {
        const uint32_t *x = stage[wib] + lane * Q.k;
        const SortKey k2 = sort_key(Q.kp, b, [&](uint32_t c) { return x[Q.opos[c]]; });
        key = k2.hi;  // the selection works on the leading word
        keys[i] = k2;
        perm[i] = (uint32_t)(S.out_row_base + local0 + lane);
      }
      __syncwarp();
    } else if (i < n) {
      const DQuery &Q = W.dq[qi];
      const QState &S = W.qs[qi];
      const uint64_t local = i - S.lrg_row_base;
      const uint32_t *x = W.out + S.out_word_base + local * Q.k;
      const SortKey k2 = sort_key(Q.kp, b, [&](uint32_t c) { return x[Q.opos[c]]; });
      key = k2.hi;
      keys[i] = k2;
      perm[i] = (uint32_t)(S.out_row_base + local);
    }
    const bool sel = i < n && W.sel[qi].state == 1;
    if (__all_sync(kFull, sel && qi == q0)) {
      uint64_t lo = key, hi = key;
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(kFull, lo, o));
        hi = max(hi, __shfl_xor_sync(kFull, hi, o));
      }
      if (lane == 0) {
        atomicMin((unsigned long long *)&W.sel[q0].lo, (unsigned long long)lo);
        atomicMax((unsigned long long *)&W.sel[q0].hi, (unsigned long long)hi);
      }
    } else if (sel) {
      atomicMin((unsigned long long *)&W.sel[qi].lo, (unsigned long long)key);
      atomicMax((unsigned long long *)&W.sel[qi].hi, (unsigned long long)key);
    }
  }
  flush_bytes(W, KK_SORT_LARGE, acc);
}

// Top-cap selection (radix select on the keys, most significant digit
// first).  The smallest cap rows of a query are among its rows with key <=
// K, K the cap-th smallest key; each round histograms one 8-bit digit of the
// keys still in play and keeps the bucket that holds K.  The first digit
// starts at the highest bit where the query's keys differ; selection stops
// when the chosen bucket exceeds what is still needed by at most cap / 8,
// when the key bits run out, or after kSelRounds rounds, and the cut is then
// every key up to the end of the bucket.  The cut keeps at least cap rows,
// and every row with key K, so sorting the kept rows gives the same first
// cap rows as sorting all of them.
constexpr int kSelRounds = 3;

__device__ __forceinline__ void sel_finish(SelState &s) {
  s.thresh = s.prefix | (s.shift ? ((1ull << s.shift) - 1) : 0);
  s.state = 2;
}

__global__ void k_sel_start(Wave W) {
  gdc_wait();
  for (uint64_t qi = gtid(); qi < W.nq; qi += gthreads()) {
    SelState &s = W.sel[qi];
    if (s.state != 1) continue;
    const uint64_t x = s.lo ^ s.hi;
    if (x == 0) {  // all keys equal: no cut
      s.thresh = ~0ull;
      s.state = 2;
      continue;
    }
    const uint32_t hb = 63 - __clzll((long long)x);
    s.mbits = hb + 1;
    s.prefix = hb == 63 ? 0 : s.lo & ~((2ull << hb) - 1);
    s.width = min(8u, hb + 1);
    s.shift = hb + 1 - s.width;
  }
}

__device__ __forceinline__ bool sel_in_play(const SelState &s, uint64_t key) {
  return s.mbits >= 64 || (key >> s.mbits) == (s.prefix >> s.mbits);
}

// Digit histogram of the keys in play; a block's rows are nearly always
// one query's, so counts gather in shared memory for the block's first
// query and go to global memory directly for any other.
__global__ void __launch_bounds__(256) k_sel_hist(Wave W, const SortKey *keys) {
  gdc_wait();
  __shared__ uint32_t h[256];
  const uint64_t n = W.ctrl->len[6];
  const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint64_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t q0 = b0 < n ? seg_of_large(W.qs, W.nq, b0, false) : 0;
  uint64_t acc = 0;
  for (uint64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const uint32_t qi = seg_of_large(W.qs, W.nq, i, false);
    const SelState &s = W.sel[qi];
    if (s.state != 1) continue;
    const uint64_t key = keys[i].hi;
    acc += 8;
    if (!sel_in_play(s, key)) continue;
    const uint32_t d = (uint32_t)(key >> s.shift) & ((1u << s.width) - 1);
    if (qi == q0) atomicAdd(&h[d], 1u);
    else atomicAdd(&W.shist[(uint64_t)qi * 256 + d], 1u);
  }
  __syncthreads();
  if (b0 < n && W.sel[q0].state == 1 && h[threadIdx.x])
    atomicAdd(&W.shist[(uint64_t)q0 * 256 + threadIdx.x], h[threadIdx.x]);
  flush_bytes(W, KK_SORT_LARGE, acc);
}

// Choose the bucket holding the need-th key; one warp per query.
__global__ void k_sel_pick(Wave W, int last) {
  gdc_wait();
  const uint32_t lane = threadIdx.x & 31;
  for (uint64_t qi = gtid() / 32; qi < W.nq; qi += gthreads() / 32) {
    SelState &s = W.sel[qi];
    if (s.state != 1) continue;  // warp-uniform
    uint32_t *hq = W.shist + qi * 256;
    uint32_t c[8];
    uint64_t sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c[j] = hq[lane * 8 + j];
      sum += c[j];
    }
    uint64_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    // the lane whose 8 digits hold the need-th key
    const uint64_t need = s.need;
    const uint32_t mine = __ballot_sync(kFull, incl >= need && incl - sum < need);
    if (!mine) {  // fewer rows in play than needed (cannot happen): keep every row
      if (lane == 0) {
        s.thresh = ~0ull;
        s.state = 2;
      }
      continue;
    }
    const int owner = __ffs(mine) - 1;
    uint32_t v = 0;
    uint64_t below = 0, bucket = 0;
    if (lane == owner) {
      uint64_t run = incl - sum;
      for (int j = 0; j < 8; ++j) {
        if (run + c[j] >= need) { v = lane * 8 + j; below = run; bucket = c[j]; break; }
        run += c[j];
      }
    }
    v = __shfl_sync(kFull, v, owner);
    below = __shfl_sync(kFull, below, owner);
    bucket = __shfl_sync(kFull, bucket, owner);
#pragma unroll
    for (int j = 0; j < 8; ++j) hq[lane * 8 + j] = 0;
    if (lane == 0) {
      s.need = need - below;
      s.prefix |= (uint64_t)v << s.shift;
      s.mbits = s.shift;
      if (s.shift == 0 || bucket - s.need <= W.dq[qi].cap / 8 || last) {
        sel_finish(s);
      } else {
        s.width = min(8u, s.shift);
        s.shift -= s.width;
      }
    }
  }
}

// Rows of a cut query with key <= thresh, packed at the front of its range
// (order does not matter: the sort follows); other rows are copied as they
// are.  One atomic per warp and query.
__global__ void k_sel_compact(Wave W, const uint32_t *pin, const SortKey *kin, uint32_t *pout, SortKey *kout) {
  gdc_wait();
  const uint64_t n = W.ctrl->len[6];
  const uint32_t lane = threadIdx.x & 31;
  uint64_t acc = 0;
  for (uint64_t base = gtid() - lane; base < n; base += gthreads()) {
    const uint64_t i = base + lane;
    uint32_t qi = 0xFFFFFFFFu;
    bool cut = false, keep = false;
    SortKey key{0, 0};
    if (i < n) {
      qi = seg_of_large(W.qs, W.nq, i, false);
      key = kin[i];
      cut = W.sel[qi].state == 2;
      keep = !cut || key.hi <= W.sel[qi].thresh;
      acc += 16 + (keep ? 24 : 0);  // key read; a kept row's index read, key and index written
      if (!cut) {
        pout[i] = pin[i];
        kout[i] = key;
      }
    }
    const uint32_t peers = __match_any_sync(kFull, cut && keep ? qi : 0xFFFFFFFFu);
    if (cut && keep) {
      const int leader = __ffs(peers) - 1;
      unsigned long long pos = 0;
      if (lane == leader) pos = atomicAdd((unsigned long long *)&W.sel[qi].kept, (unsigned long long)__popc(peers));
      pos = __shfl_sync(peers, pos, leader) + __popc(peers & ((1u << lane) - 1));
      const uint64_t at = W.qs[qi].lrg_row_base + pos;
      pout[at] = pin[i];
      kout[at] = key;
    }
  }
  flush_bytes(W, KK_SORT_LARGE, acc);
}

// Rows entering the sort and the tile layout after the cut.
__global__ void __launch_bounds__(1024) k_sort_bases(Wave W) {
  gdc_wait();
  __shared__ uint64_t sm[32];
  __shared__ uint64_t carry;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < W.nq; base += blockDim.x) {
    const uint32_t qi = base + threadIdx.x;
    uint64_t tiles = 0;
    if (qi < W.nq) {
      QState &S = W.qs[qi];
      if (W.sel[qi].state == 2) S.sort_rows = W.sel[qi].kept;
      tiles = (S.sort_rows + kTileRows - 1) / kTileRows;
    }
    uint64_t x = tiles;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = sm[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(kFull, w, o);
        if (lane >= o) w += y;
      }
      sm[lane] = w;
    }
    __syncthreads();
    if (qi < W.nq) W.qs[qi].lrg_tile_base = carry + x - tiles + (warp ? sm[warp - 1] : 0);
    __syncthreads();
    if (threadIdx.x == 0) carry += sm[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) W.ctrl->len[7] = carry;
}

// Tile sort (queries the bucket sort left): keys (and row indices) in
// shared memory, bitonic network; rows are read from the output pool only to
// order equal keys.
__global__ void __launch_bounds__(256) k_tile_sort(Wave W, const uint32_t *pin, const SortKey *kin, uint32_t *pout,
                                                   SortKey *kout) {
  gdc_wait();
  __shared__ SortKey key[kTileRows];
  __shared__ uint32_t row[kTileRows];
  __shared__ uint32_t idx[kTileRows];
  if (!W.ctrl->bkt_fail) return;  // every query was sorted by buckets
  const uint64_t ntiles = W.ctrl->len[7];
  uint64_t acc = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t qi = seg_of_large(W.qs, W.nq, t, true);
    const DQuery &Q = W.dq[qi];
    const QState &S = W.qs[qi];
    if (!S.bkt_fail) continue;  // block-uniform: sorted by buckets
    const uint64_t first = (t - S.lrg_tile_base) * kTileRows, at = S.lrg_row_base + first;
    const uint32_t n = (uint32_t)min((uint64_t)kTileRows, S.sort_rows - first);
    if (threadIdx.x == 0) acc += 40ull * n;  // keys and indices read and written
    uint32_t np2 = 1;
    while (np2 < n) np2 <<= 1;
    for (uint32_t i = threadIdx.x; i < np2; i += blockDim.x) {
      idx[i] = i;
      if (i < n) {
        key[i] = kin[at + i];
        row[i] = pin[at + i];
      }
    }
    __syncthreads();
    // a < c in (key, row) order; positions past n sort last
    auto less = [&](uint32_t a, uint32_t c) {
      if (a >= n) return false;
      if (c >= n) return true;
      if (key[a] != key[c]) return key[a] < key[c];
      return !keys_exact(W, Q) && !out_row_le(W, Q, S, row[c], row[a]);
    };
    for (uint32_t size = 2; size <= np2; size <<= 1)
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t x = threadIdx.x; x < np2 / 2; x += blockDim.x) {
          // x-th compare-exchange pair of this stage: (i, i + stride)
          const uint32_t i = 2 * x - (x & (stride - 1));
          const uint32_t p = i + stride;
          const bool up = (i & size) == 0;
          const uint32_t a = idx[i], c = idx[p];
          if (up ? less(c, a) : less(a, c)) { idx[i] = c; idx[p] = a; }
        }
        __syncthreads();
      }
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      pout[at + i] = row[idx[i]];
      kout[at + i] = key[idx[i]];
    }
    __syncthreads();
  }
  flush_bytes(W, KK_SORT_LARGE, acc);
}

// Where output tile t of a merge pass with runs of `run` rows sits: its
// query, the start of its pair of runs and their lengths (nb = 0: a lone
// run).  Only the smallest cap rows of a query are returned, so only the
// first cap entries of a run are kept (va, vb: the valid prefixes; out: the
// valid length of the merged run).  A query whose rows already form one run
// (n <= run) is finished and takes no part in the pass.
struct MergeTile {
  uint32_t qi;
  bool active;
  uint64_t base, first, a0, na, nb, va, vb, out;
};
__device__ __forceinline__ MergeTile merge_tile(const Wave &W, uint64_t t, uint64_t run) {
  MergeTile m;
  m.qi = seg_of_large(W.qs, W.nq, t, true);
  const QState &S = W.qs[m.qi];
  // a projected output keeps every row: duplicates go only after sorting
  const uint64_t n = S.sort_rows, cap = W.dq[m.qi].proj ? ~0ull : W.dq[m.qi].cap;
  m.base = S.lrg_row_base;
  m.first = (t - S.lrg_tile_base) * kTileRows;
  m.a0 = (m.first / (2 * run)) * 2 * run;
  m.na = min(run, n - m.a0);
  m.nb = n - m.a0 > run ? min(run, n - m.a0 - run) : 0;
  m.va = min(m.na, cap);
  m.vb = min(m.nb, cap);
  m.out = min(m.va + m.vb, cap);
  m.active = S.bkt_fail && n > run && m.first - m.a0 < m.out;  // only queries the bucket sort left
  return m;
}

// Merge-path split at diagonal o of runs A (va valid) and B (vb valid): how
// many of the first o outputs come from A (stable: A wins ties).
__device__ __forceinline__ uint64_t merge_split_at(const Wave &W, const DQuery &Q, const QState &S, const uint32_t *perm,
                                                   const SortKey *key, uint64_t A, uint64_t B, uint64_t va,
                                                   uint64_t vb, uint64_t o) {
  uint64_t lo = o > vb ? o - vb : 0, hi = min(o, va);
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1, j = o - 1 - mid;
    if (kr_le(W, Q, S, key[A + mid], perm[A + mid], key[B + j], perm[B + j])) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Split of every active output tile at its first output.  One thread per tile.
__global__ void k_merge_split(Wave W, const uint32_t *perm, const SortKey *key, uint64_t run) {
  gdc_wait();
  if (!W.ctrl->bkt_fail) return;
  const uint64_t ntiles = W.ctrl->len[7];
  for (uint64_t t = gtid(); t < ntiles; t += gthreads()) {
    const MergeTile m = merge_tile(W, t, run);
    if (!m.active) continue;
    const uint64_t o = m.first - m.a0;
    if (m.nb == 0) {
      W.msplit[t] = o;
      continue;
    }
    const uint64_t A = m.base + m.a0;
    W.msplit[t] = merge_split_at(W, W.dq[m.qi], W.qs[m.qi], perm, key, A, A + m.na, m.va, m.vb, o);
  }
}

// One merge pass: runs of `run` (>= kTileRows) rows become runs of 2*run.
// One block per active output tile: the tile's slices of both runs (bounded
// by the splits at its first and last output) are staged in shared memory
// with their keys; each thread places four outputs after a short search in
// the slices.
__global__ void __launch_bounds__(256) k_merge_tiles(Wave W, const uint32_t *pin, const SortKey *kin, uint32_t *pout,
                                                     SortKey *kout, uint64_t run) {
  gdc_wait();
  __shared__ SortKey sk[kTileRows];
  __shared__ uint32_t si[kTileRows];
  __shared__ uint64_t s_end;
  if (!W.ctrl->bkt_fail) return;
  const uint64_t ntiles = W.ctrl->len[7];
  uint64_t acc = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const MergeTile m = merge_tile(W, t, run);
    if (!m.active) continue;  // block-uniform
    const uint64_t o0 = m.first - m.a0, o1 = min(o0 + kTileRows, m.out);
    if (threadIdx.x == 0) acc += 40 * (o1 - o0);  // keys and indices read and written
    if (m.nb == 0) {
      for (uint64_t i = m.base + m.first + threadIdx.x; i < m.base + m.a0 + o1; i += blockDim.x) {
        pout[i] = pin[i];
        kout[i] = kin[i];
      }
      continue;
    }
    const DQuery &Q = W.dq[m.qi];
    const QState &S = W.qs[m.qi];
    const uint64_t A0 = m.base + m.a0, B0 = A0 + m.na;
    // the end split: the next tile's start, the end of both runs, or (a run
    // cut at cap inside this tile) a search at the cut
    if (threadIdx.x == 0) {
      if (o1 < m.out) s_end = W.msplit[t + 1];
      else if (m.out == m.va + m.vb) s_end = m.va;
      else s_end = merge_split_at(W, Q, S, pin, kin, A0, B0, m.va, m.vb, o1);
    }
    __syncthreads();
    const uint64_t ab = W.msplit[t], bb = o0 - ab;
    const uint64_t ae = s_end, be = o1 - ae;
    const uint32_t la = (uint32_t)(ae - ab), lb = (uint32_t)(be - bb), total = la + lb;
    const uint64_t A = A0 + ab, B = B0 + bb;
    for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
      const uint64_t src = i < la ? A + i : B + (i - la);
      sk[i] = kin[src];
      si[i] = pin[src];
    }
    __syncthreads();
    for (uint32_t p0 = threadIdx.x * 4; p0 < total; p0 += blockDim.x * 4) {
      uint32_t lo = p0 > lb ? p0 - lb : 0, hi = min(p0, la);
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1, j = la + p0 - 1 - mid;
        if (kr_le(W, Q, S, sk[mid], si[mid], sk[j], si[j])) lo = mid + 1; else hi = mid;
      }
      uint32_t ia = lo, ib = p0 - lo;
      for (uint32_t p = p0; p < min(p0 + 4, total); ++p) {
        bool take_a;
        if (ib >= lb) take_a = true;
        else if (ia >= la) take_a = false;
        else take_a = kr_le(W, Q, S, sk[ia], si[ia], sk[la + ib], si[la + ib]);
        const uint32_t src = take_a ? ia++ : la + ib++;
        pout[m.base + m.first + p] = si[src];
        kout[m.base + m.first + p] = sk[src];
      }
    }
    __syncthreads();
  }
  flush_bytes(W, KK_SORT_LARGE, acc);
}

// Merge passes a query of n large rows takes: its runs double from
// kTileRows until one run holds every row; the tile sort writes buffer 0 and
// pass p writes buffer (p + 1) & 1, so the query ends in buffer passes & 1.
__device__ __forceinline__ uint32_t merge_passes(uint64_t n) {
  uint32_t p = 0;
  for (uint64_t run = kTileRows; run < n; run *= 2) ++p;
  return p;
}

// ------------------------------------------------------------ sample sort
// The large outputs are sorted by a sample sort.  A query of n entries gets
// nb = ceil(n / kBktAvg) buckets (kBktPerTile slots per tile of the query), bounded
// by nb - 1 splitters taken at even ranks from a sorted stratified sample of
// its entries; each entry goes to its bucket (count, scan, scatter), and one
// block sorts each bucket in shared memory.  Entries are ordered by (key,
// then, when the key does not hold the whole row, a second key of the next
// output columns and the columns after those, then the entry's row index):
// a total order, so only the sample decides bucket sizes.  The second keys
// are built from the rows when entries are staged in shared memory, so that
// the comparisons of rows with equal first keys stay on chip (rows of more
// than twice the first key's columns still compare their last columns in
// the output pool).  A query with a bucket above kBktCap entries (a sample
// far off the data) is sorted by the tile sort and merge passes instead,
// from the input its entries still hold there (every query is, when the
// batch is set to the merge path only).
constexpr uint32_t kBktAvg = kTileRows / kBktPerTile;  // entries per bucket, on average
constexpr uint32_t kBktSmall = 512;        // buckets up to this size: small blocks, many per SM
constexpr uint32_t kBktMid = 1024;         //   up to this size: small blocks, two pairs per thread
constexpr uint32_t kBktCap = 4096;         // entries one block sorts in shared memory
constexpr uint32_t kBktOversample = 4;     // sample entries per bucket
constexpr uint32_t kBktSampleMax = 4096;   // sample entries per query
constexpr uint32_t kBktSmemSpl = 4096;     // splitters' leading key words staged in shared memory for the search

// Three-way comparison of output rows a and b, equal on their first `from`
// output columns, on the columns after those.
__device__ __forceinline__ int out_row_cmp_from(const Wave &W, const DQuery &Q, const QState &S, uint32_t a,
                                                uint32_t b, uint32_t from) {
  const uint32_t *x = W.out + S.out_word_base + (uint64_t)(a - S.out_row_base) * Q.k;
  const uint32_t *y = W.out + S.out_word_base + (uint64_t)(b - S.out_row_base) * Q.k;
  for (uint32_t i = from; i < Q.kp; ++i) {
    const uint32_t c = Q.opos[i];
    const uint32_t xa = x[c], yb = y[c];
    if (xa != yb) return xa < yb ? -1 : 1;
  }
  return 0;
}

// Second key of output row r: its output columns from key_cols(W) on,
// packed as the first key packs the leading ones.
__device__ __forceinline__ SortKey row_key2(const Wave &W, const DQuery &Q, const QState &S, uint32_t r) {
  const uint32_t *x = W.out + S.out_word_base + (uint64_t)(r - S.out_row_base) * Q.k;
  const uint32_t kc = key_cols(W);
  return sort_key(Q.kp - kc, W.G.idbits, [&](uint32_t c) { return x[Q.opos[kc + c]]; });
}

// The sample sort's total order on entries (first key ka, second key ka2,
// row index ra); exact: the first key holds every output column (second
// keys unused).
__device__ __forceinline__ bool ent_lt(const Wave &W, const DQuery &Q, const QState &S, bool exact, SortKey ka,
                                       SortKey ka2, uint32_t ra, SortKey kb, SortKey kb2, uint32_t rb) {
  if (ka != kb) return ka < kb;
  if (ra == rb) return false;
  if (!exact) {
    if (ka2 != kb2) return ka2 < kb2;
    if (Q.kp > 2 * key_cols(W)) {
      const int c = out_row_cmp_from(W, Q, S, ra, rb, 2 * key_cols(W));
      if (c) return c < 0;
    }
  }
  return ra < rb;
}

// Entries staged in shared memory as arrays: first key words, second key
// words (queries whose first key does not hold the whole row) and row
// indices.  Padding entries past the live ones hold all-ones keys and the
// row index kPadRow, so they sort last.
constexpr uint32_t kPadRow = 0xFFFFFFFFu;
struct SmemEnts {
  uint64_t *hi, *lo, *hi2, *lo2;
  uint32_t *row;
};

template <bool EXACT>
__device__ __forceinline__ bool sm_less(const Wave &W, const DQuery &Q, const QState &S, const SmemEnts &e, uint32_t a,
                                        uint32_t b) {
  const uint64_t ah = e.hi[a], bh = e.hi[b];
  if (ah != bh) return ah < bh;
  const uint64_t al = e.lo[a], bl = e.lo[b];
  if (al != bl) return al < bl;
  const uint32_t ra = e.row[a], rb = e.row[b];
  if (!EXACT && ra != rb && ra != kPadRow && rb != kPadRow) {
    const uint64_t ah2 = e.hi2[a], bh2 = e.hi2[b];
    if (ah2 != bh2) return ah2 < bh2;
    const uint64_t al2 = e.lo2[a], bl2 = e.lo2[b];
    if (al2 != bl2) return al2 < bl2;
    if (Q.kp > 2 * key_cols(W)) {
      const int c = out_row_cmp_from(W, Q, S, ra, rb, 2 * key_cols(W));
      if (c) return c < 0;
    }
  }
  return ra < rb;
}

// Bitonic network over the np2 staged entries (a power of two), exchanging
// the entries themselves, so that every stage reads consecutive words.
// Thread t takes the pairs t, t + blockDim.x, ...: a warp's pairs cover
// whole 64-entry groups, so a stage of stride at most 32 exchanges only
// inside the warp's own groups, and two such stages in a row need only a
// warp barrier.
template <bool EXACT>
__device__ __forceinline__ void block_sort_ents(const Wave &W, const DQuery &Q, const QState &S, const SmemEnts &e,
                                                uint32_t np2) {
  for (uint32_t size = 2; size <= np2; size <<= 1)
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t x = threadIdx.x; x < np2 / 2; x += blockDim.x) {
        const uint32_t i = 2 * x - (x & (stride - 1));
        const uint32_t p = i + stride;
        const bool up = (i & size) == 0;
        if (up ? sm_less<EXACT>(W, Q, S, e, p, i) : sm_less<EXACT>(W, Q, S, e, i, p)) {
          uint64_t t = e.hi[i]; e.hi[i] = e.hi[p]; e.hi[p] = t;
          t = e.lo[i]; e.lo[i] = e.lo[p]; e.lo[p] = t;
          if (!EXACT) {
            t = e.hi2[i]; e.hi2[i] = e.hi2[p]; e.hi2[p] = t;
            t = e.lo2[i]; e.lo2[i] = e.lo2[p]; e.lo2[p] = t;
          }
          const uint32_t r = e.row[i]; e.row[i] = e.row[p]; e.row[p] = r;
        }
      }
      const uint32_t next = stride > 1 ? stride >> 1 : size;  // the next stage's stride
      if (stride <= 32 && next <= 32 && size < np2) __syncwarp();
      else __syncthreads();
    }
}

__device__ __forceinline__ void block_sort_ents(const Wave &W, const DQuery &Q, const QState &S, const SmemEnts &e,
                                                uint32_t np2, bool exact) {
  if (exact) block_sort_ents<true>(W, Q, S, e, np2);
  else block_sort_ents<false>(W, Q, S, e, np2);
}

// Entry j of the staged arrays: live (key k, row r, second key of r unless
// exact) or padding.
__device__ __forceinline__ void stage_ent(const Wave &W, const DQuery &Q, const QState &S, const SmemEnts &e, uint32_t j,
                                          bool live, bool exact, SortKey k, uint32_t r) {
  if (!live) {
    e.hi[j] = e.lo[j] = e.hi2[j] = e.lo2[j] = ~0ull;
    e.row[j] = kPadRow;
    return;
  }
  e.hi[j] = k.hi;
  e.lo[j] = k.lo;
  e.row[j] = r;
  if (!exact) {
    const SortKey k2 = row_key2(W, Q, S, r);
    e.hi2[j] = k2.hi;
    e.lo2[j] = k2.lo;
  }
}

__device__ __forceinline__ SmemEnts carve_ents(uint8_t *base, uint32_t cap) {
  SmemEnts e;
  e.hi = reinterpret_cast<uint64_t *>(base);
  e.lo = e.hi + cap;
  e.hi2 = e.lo + cap;
  e.lo2 = e.hi2 + cap;
  e.row = reinterpret_cast<uint32_t *>(e.lo2 + cap);
  return e;
}
constexpr size_t kEntBytes = 4 * sizeof(uint64_t) + sizeof(uint32_t);

__device__ __forceinline__ uint64_t bkt_count_of(uint64_t n) { return (n + kBktAvg - 1) / kBktAvg; }
__device__ __forceinline__ uint64_t bkt_base(const QState &S) { return kBktPerTile * S.lrg_tile_base; }

// Splitters: one block per query of more than one bucket samples
// m = min(4 nb, 4096, n) entries, one at a hashed position in each of m
// equal strata, sorts them, and keeps the entries at ranks b m / nb
// (b = 1 .. nb - 1) with their second keys.  Also clears every query's
// overflow flag and sets the number of bucket slots (kBktPerTile per tile).
__global__ void __launch_bounds__(1024) k_bkt_split(Wave W, const uint32_t *pin, const SortKey *kin) {
  gdc_wait();
  extern __shared__ __align__(16) uint8_t bkt_smem[];
  const SmemEnts e = carve_ents(bkt_smem, kBktSampleMax);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    W.ctrl->bkt_fail = W.merge_only;
    W.ctrl->nbkt = kBktPerTile * W.ctrl->len[7];
  }
  uint64_t acc = 0;
  for (uint32_t qi = blockIdx.x; qi < W.nq; qi += gridDim.x) {
    QState &S = W.qs[qi];
    if (threadIdx.x == 0) S.bkt_fail = W.merge_only;
    const uint64_t n = S.sort_rows, nb = bkt_count_of(n);
    if (nb <= 1 || W.merge_only) continue;  // block-uniform
    const DQuery &Q = W.dq[qi];
    const bool exact = keys_exact(W, Q);
    uint64_t mm = nb * kBktOversample;
    if (mm > kBktSampleMax) mm = kBktSampleMax;
    if (mm > n) mm = n;
    const uint32_t m = (uint32_t)mm;
    uint32_t np2 = 1;
    while (np2 < m) np2 <<= 1;
    for (uint32_t j = threadIdx.x; j < np2; j += blockDim.x) {
      SortKey k{0, 0};
      uint32_t r = 0;
      if (j < m) {
        const uint64_t lo = (uint64_t)j * n / m, hi = (uint64_t)(j + 1) * n / m;
        const uint64_t p = lo + (hi > lo ? mix64(((uint64_t)qi << 32) ^ j) % (hi - lo) : 0);
        k = kin[S.lrg_row_base + p];
        r = pin[S.lrg_row_base + p];
      }
      stage_ent(W, Q, S, e, j, j < m, exact, k, r);
    }
    __syncthreads();
    block_sort_ents(W, Q, S, e, np2, exact);
    for (uint64_t b = 1 + threadIdx.x; b < nb; b += blockDim.x) {
      const uint32_t j = (uint32_t)(b * m / nb);
      W.bspl_key[bkt_base(S) + b - 1] = SortKey{e.hi[j], e.lo[j]};
      W.bspl_key2[bkt_base(S) + b - 1] = exact ? SortKey{0, 0} : SortKey{e.hi2[j], e.lo2[j]};
      W.bspl_row[bkt_base(S) + b - 1] = e.row[j];
    }
    if (threadIdx.x == 0) acc += 20ull * m + 36ull * (nb - 1);  // samples read, splitters written
    __syncthreads();
  }
  flush_bytes(W, KK_SORT_LARGE, acc);
}

// Bucket of each entry (count pass: found by a search of the query's
// splitters, kept in bkt_id and counted into ptcount; scatter pass: each
// entry to its bucket's next free place, from the cursors k_bkt_bases set in
// msplit, into pout / kout).  Each block takes a
// contiguous range of tiles, so consecutive tiles are mostly one query's and
// the leading words of its splitters' keys are staged in shared memory once
// (the rest of a splitter is read only when the leading words are equal).  An entry's
// second key is built only when its first key equals a splitter's.
__global__ void __launch_bounds__(256) k_bkt_place(Wave W, const uint32_t *pin, const SortKey *kin, uint32_t *pout,
                                                   SortKey *kout, int scatter) {
  gdc_wait();
  __shared__ uint64_t ssh[kBktSmemSpl];
  if (W.merge_only) return;
  const uint64_t nt = W.ctrl->len[7];
  const uint64_t per = (nt + gridDim.x - 1) / gridDim.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * per, t1 = t0 + per < nt ? t0 + per : nt;
  uint32_t qi = t0 < t1 ? seg_of_large(W.qs, W.nq, t0, true) : 0;
  uint32_t staged_q = 0xFFFFFFFFu;
  uint64_t acc = 0;
  for (uint64_t t = t0; t < t1; ++t) {  // block-uniform
    while (qi + 1 < W.nq && W.qs[qi + 1].lrg_tile_base <= t) ++qi;
    QState &S = W.qs[qi];
    const DQuery &Q = W.dq[qi];
    const bool exact = keys_exact(W, Q);
    const uint64_t nb = bkt_count_of(S.sort_rows), sb = bkt_base(S);
    const bool staged = !scatter && nb > 1 && nb - 1 <= kBktSmemSpl;
    if (staged && staged_q != qi) {
      __syncthreads();  // every search in the previous query's splitters is done
      for (uint32_t j = threadIdx.x; j < nb - 1; j += blockDim.x) ssh[j] = W.bspl_key[sb + j].hi;
      __syncthreads();
      staged_q = qi;
    }
    const uint64_t first = (t - S.lrg_tile_base) * kTileRows;
    const uint32_t cnt = (uint32_t)(S.sort_rows - first < kTileRows ? S.sort_rows - first : kTileRows);
    for (uint32_t e = threadIdx.x; e < cnt; e += blockDim.x) {
      const uint64_t i = S.lrg_row_base + first + e;
      const SortKey key = kin[i];
      const uint32_t row = pin[i];
      if (scatter) {
        const uint64_t pos = atomicAdd((unsigned long long *)&W.msplit[sb + W.bkt_id[i]], 1ull);
        pout[pos] = row;
        kout[pos] = key;
        acc += 44;  // key, index and bucket read; key and index written
        continue;
      }
      SortKey key2{0, 0};
      bool have2 = exact;
      uint32_t b = 0;
      if (nb > 1) {  // splitters below the entry
        uint32_t lo = 0, hi = (uint32_t)(nb - 1);
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          bool lt;
          const uint64_t sh = staged ? ssh[mid] : W.bspl_key[sb + mid].hi;
          const SortKey s1 = sh != key.hi ? SortKey{sh, 0} : W.bspl_key[sb + mid];
          if (sh != key.hi) {
            lt = sh < key.hi;
          } else if (s1 != key) {
            lt = s1 < key;
          } else {
            if (!have2) {
              key2 = row_key2(W, Q, S, row);
              have2 = true;
            }
            lt = ent_lt(W, Q, S, exact, s1, W.bspl_key2[sb + mid], W.bspl_row[sb + mid], key, key2, row);
          }
          if (lt) lo = mid + 1; else hi = mid;
        }
        b = lo;
      }
      W.bkt_id[i] = b;
      atomicAdd(&W.ptcount[sb + b], 1u);
      acc += 24;  // key and index read, bucket written
    }
  }
  flush_bytes(W, KK_SORT_LARGE, acc);
}

// Each bucket slot's first place (from the scan of the counts) as its fill
// cursor for the scatter pass; a bucket above kBktCap entries sends its
// query to the merge path.
__global__ void k_bkt_bases(Wave W) {
  gdc_wait();
  const uint64_t nt = W.ctrl->nbkt;
  for (uint64_t t = gtid(); t < nt; t += gthreads()) {
    const uint32_t qi = seg_of_large(W.qs, W.nq, t / kBktPerTile, true);
    QState &S = W.qs[qi];
    W.msplit[t] = S.lrg_row_base + (W.ptscan[t] - W.ptscan[bkt_base(S)]);
    if (W.ptcount[t] > kBktCap) {
      S.bkt_fail = 1;
      W.ctrl->bkt_fail = 1;
    }
  }
}

// One block per bucket of (LO, CAP] entries: the entries, with their second
// keys when the first does not hold the whole row, sorted in shared memory
// and written, in place, to the buffer the query's sorted rows are read from
// (the one the merge passes would have ended in).  Bucket slots are per
// tile: the bucket of slot t belongs to the query holding tile t / kBktPerTile.
template <uint32_t LO, uint32_t CAP>
__global__ void k_bkt_sort(Wave W, const uint32_t *px, const SortKey *kx, uint32_t *p0, SortKey *k0, uint32_t *p1,
                           SortKey *k1) {
  gdc_wait();
  extern __shared__ __align__(16) uint8_t bkt_smem[];
  const SmemEnts e = carve_ents(bkt_smem, CAP);
  const uint64_t nt = W.ctrl->nbkt;
  uint64_t acc = 0;
  for (uint64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const uint32_t n = W.ptcount[t];
    if (n <= LO || n > CAP) continue;  // block-uniform: another tier's, empty, or overflowed
    const uint32_t qi = seg_of_large(W.qs, W.nq, t / kBktPerTile, true);
    const QState &S = W.qs[qi];
    if (S.bkt_fail) continue;
    const DQuery &Q = W.dq[qi];
    const bool exact = keys_exact(W, Q);
    const uint64_t at = S.lrg_row_base + (W.ptscan[t] - W.ptscan[bkt_base(S)]);
    uint32_t np2 = 1;
    while (np2 < n) np2 <<= 1;
    for (uint32_t j = threadIdx.x; j < np2; j += blockDim.x)
      stage_ent(W, Q, S, e, j, j < n, exact, j < n ? kx[at + j] : SortKey{0, 0}, j < n ? px[at + j] : 0);
    __syncthreads();
    block_sort_ents(W, Q, S, e, np2, exact);
    const bool odd = merge_passes(S.sort_rows) & 1;
    uint32_t *po = odd ? p1 : p0;
    SortKey *ko = odd ? k1 : k0;
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
      po[at + j] = e.row[j];
      ko[at + j] = SortKey{e.hi[j], e.lo[j]};
    }
    if (threadIdx.x == 0) acc += (exact ? 40ull : 40ull + 4ull * Q.kp) * n;  // keys and indices (and rows) read, written
    __syncthreads();
  }
  flush_bytes(W, KK_SORT_LARGE, acc);
}

// Sorted large rows in query-vertex column order, laid out query by query:
// the first cap rows of each query, from the buffer its last pass wrote.
__global__ void k_gather(Wave W, const uint32_t *perm0, const uint32_t *perm1) {
  gdc_wait();
  const uint64_t n = W.ctrl->len[6];
  uint64_t acc = 0;
  for (uint64_t i = gtid(); i < n; i += gthreads()) {
    const uint32_t qi = seg_of_large(W.qs, W.nq, i, false);
    const DQuery &Q = W.dq[qi];
    const QState &S = W.qs[qi];
    if (Q.proj || i - S.lrg_row_base >= Q.cap) continue;  // projected: k_proj_write; past the rows returned
    acc += 4 + 8ull * Q.k;  // index, the row read and written
    const uint32_t row = ((merge_passes(S.sort_rows) & 1) ? perm1 : perm0)[i];
    const uint32_t *src = W.out + S.out_word_base + (uint64_t)(row - S.out_row_base) * Q.k;
    uint32_t *dst = W.out_final + S.fin_word_base + (uint64_t)(i - S.lrg_row_base) * Q.k;
    for (uint32_t u = 0; u < Q.k; ++u) dst[u] = src[Q.pos[u]];
  }
  flush_bytes(W, KK_GATHER, acc);
}

// Projected large outputs: after the merge sort, rows with equal projected
// tuples sit next to each other, and a row starts a new tuple when it
// differs from the row before it.  Per tile of kTileRows sorted rows, one
// kernel counts the starts; a scan of the counts gives each tile's first
// rank; a second kernel writes every start whose rank is below cap.
__device__ __forceinline__ bool proj_start(const Wave &W, const DQuery &Q, const QState &S, const uint32_t *perm,
                                           const SortKey *key, uint64_t i) {
  if (i == 0) return true;
  const uint64_t a = S.lrg_row_base + i;
  return key[a] != key[a - 1] || (!keys_exact(W, Q) && !out_row_eq(W, Q, S, perm[a], perm[a - 1]));
}

__global__ void __launch_bounds__(256) k_proj_count(Wave W, const uint32_t *perm0, const uint32_t *perm1,
                                                    const SortKey *key0, const SortKey *key1) {
  gdc_wait();
  __shared__ uint32_t wsum[8];
  const uint64_t ntiles = W.ctrl->len[7];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t qi = seg_of_large(W.qs, W.nq, t, true);
    const DQuery &Q = W.dq[qi];
    const QState &S = W.qs[qi];
    uint32_t c = 0;
    if (Q.proj) {  // block-uniform
      const bool odd = merge_passes(S.sort_rows) & 1;
      const uint64_t first = (t - S.lrg_tile_base) * kTileRows;
      const uint64_t n = min((uint64_t)kTileRows, S.sort_rows - first);
      for (uint64_t i = threadIdx.x; i < n; i += blockDim.x)
        c += proj_start(W, Q, S, odd ? perm1 : perm0, odd ? key1 : key0, first + i);
    }
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < 8; ++w) tot += wsum[w];
      W.ptcount[t] = tot;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_proj_write(Wave W, const uint32_t *perm0, const uint32_t *perm1,
                                                    const SortKey *key0, const SortKey *key1) {
  gdc_wait();
  __shared__ uint32_t rk[kTileRows];
  const uint64_t ntiles = W.ctrl->len[7];
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t qi = seg_of_large(W.qs, W.nq, t, true);
    const DQuery &Q = W.dq[qi];
    const QState &S = W.qs[qi];
    if (!Q.proj) continue;  // block-uniform
    const bool odd = merge_passes(S.sort_rows) & 1;
    const uint32_t *perm = odd ? perm1 : perm0;
    const SortKey *key = odd ? key1 : key0;
    const uint64_t first = (t - S.lrg_tile_base) * kTileRows;
    const uint32_t n = (uint32_t)min((uint64_t)kTileRows, S.sort_rows - first);
    for (uint32_t i = threadIdx.x; i < kTileRows; i += blockDim.x) rk[i] = i < n && proj_start(W, Q, S, perm, key, first + i);
    __syncthreads();
    const uint32_t here = block_scan_excl(rk, kTileRows);
    const uint64_t q0 = W.ptscan[S.lrg_tile_base], base = W.ptscan[t] - q0;
    uint32_t *dst = W.out_final + S.fin_word_base;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t r = rk[i];
      if ((i + 1 < n ? rk[i + 1] : here) == r || base + r >= Q.cap) continue;  // not a start, or past cap
      const uint32_t *x = W.out + S.out_word_base + (uint64_t)(perm[S.lrg_row_base + first + i] - S.out_row_base) * Q.k;
      for (uint32_t c = 0; c < Q.kp; ++c) dst[(base + r) * Q.kp + c] = x[Q.opos[c]];
    }
    if (threadIdx.x == 0 && t == S.lrg_tile_base) {
      const uint64_t tiles = (S.sort_rows + kTileRows - 1) / kTileRows;
      const uint64_t d = W.ptscan[S.lrg_tile_base + tiles] - q0;
      W.qs[qi].nfinal = min(d, Q.cap);
      W.qs[qi].more = d > Q.cap;
    }
    __syncthreads();
  }
}

// Epilogue: per-query results and rows of this wave into the batch store.
__global__ void k_epilogue_copy(Wave W) {
  gdc_wait();
  const WaveDesc D = W.waves[W.ctrl->wave];
  const uint64_t top = W.ctrl->store_top, words = W.ctrl->fin_words;
  const bool fits = top + words <= W.bo.store_cap;
  for (uint64_t qi = gtid(); qi < D.nq; qi += gthreads()) {
    const uint64_t b = D.q0 + qi;
    const DQuery &Q = W.dq[qi];
    const QState &S = W.qs[qi];
    uint32_t st = Q.status;
    if (st == QS_OK && S.out_rows && !fits) st = QS_OVERFLOW;
    W.bo.count[b] = S.count;
    W.bo.fp[b] = S.fp;
    W.bo.status[b] = st;
    W.bo.nrows[b] = st == QS_OK ? (S.nfinal | (S.more ? kRowsMore : 0)) : 0;
    W.bo.word_off[b] = top + S.fin_word_base;
    W.bo.inter[b] = S.inter_words;
    W.bo.peak[b] = S.peak_words;
  }
  if (fits)
    for (uint64_t i = gtid(); i < words; i += gthreads()) W.bo.store[top + i] = W.out_final[i];
}

__global__ void k_epilogue_advance(Wave W) {
  gdc_wait();
  const uint64_t top = W.ctrl->store_top, words = W.ctrl->fin_words;
  if (top + words > W.ctrl->hw[HW_STORE]) W.ctrl->hw[HW_STORE] = top + words;
  if (top + words <= W.bo.store_cap) W.ctrl->store_top = top + words;
  W.ctrl->wave += 1;
}

inline unsigned grid_for(int sms, int per_sm) { return (unsigned)(sms * per_sm); }

// Resident blocks per SM of a kernel (from its registers and shared memory),
// capped at 8; queried once per kernel.  Persistent grid-stride kernels are
// launched with exactly this many blocks per SM, so that no block waits for a
// second wave behind the others.
int resident_per_sm(const void *fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void *, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(fn);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  n = n > 8 ? 8 : n;
  cache.emplace(fn, n);
  return n;
}
template <class... P>
unsigned persistent_grid(void (*fn)(P...), int sms, int threads = kThreads, size_t smem = 0) {
  return (unsigned)(sms * resident_per_sm((const void *)fn, threads, smem));
}
// Blocks for a fixed number of warp-sized items, at most the persistent grid.
template <class... P>
unsigned grid_items(void (*fn)(P...), uint64_t warp_items, int sms) {
  uint64_t b = (warp_items + kThreads / 32 - 1) / (kThreads / 32);
  if (b == 0) b = 1;
  const uint64_t cap = persistent_grid(fn, sms);
  return (unsigned)(b < cap ? b : cap);
}
inline unsigned blocks_for(uint64_t n, unsigned per) {
  uint64_t b = (n + per - 1) / per;
  return (unsigned)(b ? b : 1);
}

}  // namespace

// ------------------------------------------------------------ launchers
void launch_prologue(const Wave &W, cudaStream_t s, int sms) {
  pdl(k_prologue, grid_for(sms, 2), kThreads, 0, s, W);
}
void launch_plan(const Wave &W, const uint32_t *type_count, cudaStream_t s, int sms) {
  pdl(k_plan, blocks_for(W.nq + 1, 128), 128, 0, s, W, type_count);
  pdl(k_owners, blocks_for(W.nq, 128), 128, 0, s, W);
}
void launch_filter(const Wave &W, cudaStream_t s, int sms) {
  pdl(k_filter, grid_items(k_filter, (uint64_t)W.nq * W.G.W1, sms), kThreads, 0, s, W);
}
void launch_compact_count(const Wave &W, int mode, uint32_t step, cudaStream_t s, int sms) {
  const uint64_t sets = mode == 0 ? W.nq : W.nqv;
  cudaMemsetAsync(&W.ctrl->len[9], 0, sizeof(uint64_t), s);
  pdl(k_chunk_list, grid_items(k_chunk_list, sets * W.G.ipg, sms), kThreads, 0, s, W, mode, step);
  pdl(k_compact_count, persistent_grid(k_compact_count, sms), kThreads, 0, s, W);
}
void launch_compact_claim(const Wave &W, uint32_t step, cudaStream_t s, int sms) {
  cudaMemsetAsync(&W.ctrl->len[9], 0, sizeof(uint64_t), s);
  pdl(k_chunk_list, grid_items(k_chunk_list, (uint64_t)W.nq * W.G.ipg, sms), kThreads, 0, s, W, 0, step);
  pdl(k_compact_claim, persistent_grid(k_compact_claim, sms), kThreads, 0, s, W);
}
void launch_compact_write(const Wave &W, int mode, uint32_t step, const uint64_t *scan, uint32_t *dst, uint32_t *owner,
                          uint64_t cap, int hw_slot, cudaStream_t s, int sms) {
  pdl(k_compact_write, persistent_grid(k_compact_write, sms), kThreads, 0, s, W, mode, scan, dst, owner, cap, hw_slot);
}
void launch_explore(const Wave &W, uint32_t step, int group, cudaStream_t s, int sms) {
  switch (group) {
    case 4: pdl(k_explore<4>, persistent_grid(k_explore<4>, sms), kThreads, 0, s, W, step); break;
    case 8: pdl(k_explore<8>, persistent_grid(k_explore<8>, sms), kThreads, 0, s, W, step); break;
    case 16: pdl(k_explore<16>, persistent_grid(k_explore<16>, sms), kThreads, 0, s, W, step); break;
    default: pdl(k_explore<32>, persistent_grid(k_explore<32>, sms), kThreads, 0, s, W, step); break;
  }
}
void launch_refine(const Wave &W, uint32_t round, uint32_t sub, int group, cudaStream_t s, int sms) {
  switch (group) {
    case 4: pdl(k_refine<4>, persistent_grid(k_refine<4>, sms), kThreads, 0, s, W, round, sub); break;
    case 8: pdl(k_refine<8>, persistent_grid(k_refine<8>, sms), kThreads, 0, s, W, round, sub); break;
    case 16: pdl(k_refine<16>, persistent_grid(k_refine<16>, sms), kThreads, 0, s, W, round, sub); break;
    default: pdl(k_refine<32>, persistent_grid(k_refine<32>, sms), kThreads, 0, s, W, round, sub); break;
  }
}
void launch_list_table(const Wave &W, cudaStream_t s, int sms) {
  pdl(k_list_table, blocks_for(W.nqv, kThreads), kThreads, 0, s, W);
}
void launch_join_plan(const Wave &W, cudaStream_t s, int sms) { pdl(k_join_plan, blocks_for(W.nq, 64), 64, 0, s, W); }
void launch_ec_limit(const Wave &W, cudaStream_t s, int sms) {
  pdl(k_ec_limit, blocks_for(W.nqe, kThreads), kThreads, 0, s, W);
}
void launch_ec(const Wave &W, bool write, int group, cudaStream_t s, int sms) {
  switch (group) {
    case 4: if (write) pdl(k_ec<4, true>, persistent_grid(k_ec<4, true>, sms), kThreads, 0, s, W); else pdl(k_ec<4, false>, persistent_grid(k_ec<4, false>, sms), kThreads, 0, s, W); break;
    case 8: if (write) pdl(k_ec<8, true>, persistent_grid(k_ec<8, true>, sms), kThreads, 0, s, W); else pdl(k_ec<8, false>, persistent_grid(k_ec<8, false>, sms), kThreads, 0, s, W); break;
    case 16: if (write) pdl(k_ec<16, true>, persistent_grid(k_ec<16, true>, sms), kThreads, 0, s, W); else pdl(k_ec<16, false>, persistent_grid(k_ec<16, false>, sms), kThreads, 0, s, W); break;
    default: if (write) pdl(k_ec<32, true>, persistent_grid(k_ec<32, true>, sms), kThreads, 0, s, W); else pdl(k_ec<32, false>, persistent_grid(k_ec<32, false>, sms), kThreads, 0, s, W); break;
  }
}
void launch_clear(const Wave &W, cudaStream_t s, int sms) {
  pdl(k_clear, grid_items(k_clear, (uint64_t)W.nqv * W.G.ipg, sms), kThreads, 0, s, W);
}
void launch_join0(const Wave &W, cudaStream_t s, int sms) {
  pdl(k_join0_rows, blocks_for(W.nq, 256), 256, 0, s, W);
  pdl(k_level_sizes, blocks_for(W.nq, kThreads), kThreads, 0, s, W, 0);
  pdl(k_level_alloc, 1, 1024, 0, s, W, 0);
  pdl(k_join0_write, persistent_grid(k_join0_write, sms), kThreads, 0, s, W);
}
void launch_join_count(const Wave &W, uint32_t lvl, int group, cudaStream_t s, int sms) {
  switch (group) {
    case 4: pdl(k_join_count<4>, persistent_grid(k_join_count<4>, sms), kThreads, 0, s, W, lvl); break;
    case 8: pdl(k_join_count<8>, persistent_grid(k_join_count<8>, sms), kThreads, 0, s, W, lvl); break;
    case 16: pdl(k_join_count<16>, persistent_grid(k_join_count<16>, sms), kThreads, 0, s, W, lvl); break;
    default: pdl(k_join_count<32>, persistent_grid(k_join_count<32>, sms), kThreads, 0, s, W, lvl); break;
  }
}
void launch_level_alloc(const Wave &W, uint32_t lvl, cudaStream_t s) {
  pdl(k_level_sizes, blocks_for(W.nq, kThreads), kThreads, 0, s, W, lvl);
  pdl(k_level_alloc, 1, 1024, 0, s, W, lvl);
}
void launch_join_write(const Wave &W, uint32_t lvl, int group, cudaStream_t s, int sms) {
  switch (group) {
    case 4: pdl(k_join_write<4>, persistent_grid(k_join_write<4>, sms), kThreads, 0, s, W, lvl); break;
    case 8: pdl(k_join_write<8>, persistent_grid(k_join_write<8>, sms), kThreads, 0, s, W, lvl); break;
    case 16: pdl(k_join_write<16>, persistent_grid(k_join_write<16>, sms), kThreads, 0, s, W, lvl); break;
    default: pdl(k_join_write<32>, persistent_grid(k_join_write<32>, sms), kThreads, 0, s, W, lvl); break;
  }
}
void launch_final_bases(const Wave &W, cudaStream_t s) { pdl(k_final_bases, 1, 1024, 0, s, W); }
void launch_small_sort(const Wave &W, cudaStream_t s, int sms) {
  const unsigned cap = persistent_grid(k_small_sort, sms, 256);
  pdl(k_small_sort, W.nq < cap ? (W.nq ? W.nq : 1) : cap, 256, 0, s, W);
}
void launch_sort_keys(const Wave &W, uint32_t *perm, SortKey *keys, cudaStream_t s, int sms) {
  pdl(k_sort_keys, persistent_grid(k_sort_keys, sms), kThreads, 0, s, W, perm, keys);
}
void launch_select(const Wave &W, const uint32_t *pin, const SortKey *kin, uint32_t *pout, SortKey *kout,
                   cudaStream_t s, int sms) {
  pdl(k_sel_start, blocks_for(W.nq, 256), 256, 0, s, W);
  for (int r = 0; r < kSelRounds; ++r) {
    pdl(k_sel_hist, persistent_grid(k_sel_hist, sms, 256), 256, 0, s, W, kin);
    pdl(k_sel_pick, blocks_for((uint64_t)W.nq * 32, 256), 256, 0, s, W, r == kSelRounds - 1);
  }
  pdl(k_sel_compact, persistent_grid(k_sel_compact, sms), kThreads, 0, s, W, pin, kin, pout, kout);
  pdl(k_sort_bases, 1, 1024, 0, s, W);
}
void launch_bucket_sort(const Wave &W, const uint32_t *pin, const SortKey *kin, uint32_t *px, SortKey *kx,
                        uint32_t *p0, SortKey *k0, uint32_t *p1, SortKey *k1, uint64_t *scan_tmp, cudaStream_t s,
                        int sms) {
  constexpr size_t split_smem = (size_t)kBktSampleMax * kEntBytes;
  constexpr size_t small_smem = (size_t)kBktSmall * kEntBytes;
  constexpr size_t mid_smem = (size_t)kBktMid * kEntBytes;
  constexpr size_t big_smem = (size_t)kBktCap * kEntBytes;
  static const bool attrs = [] {
    cudaFuncSetAttribute(k_bkt_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_smem);
    cudaFuncSetAttribute(k_bkt_sort<kBktMid, kBktCap>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem);
    return true;
  }();
  (void)attrs;
  const uint64_t slots = kBktPerTile * (W.out_rows_cap / kTileRows + W.nq + 1);
  cudaMemsetAsync(W.ptcount, 0, 4 * slots, s);
  pdl(k_bkt_split, std::max(1u, std::min<unsigned>(W.nq, (unsigned)sms * 2)), 1024, split_smem, s, W, pin, kin);
  const unsigned place = persistent_grid(k_bkt_place, sms);
  pdl(k_bkt_place, place, kThreads, 0, s, W, pin, kin, px, kx, 0);
  scan_u32(W.ptcount, W.ptscan, &W.ctrl->nbkt, slots, scan_tmp, s, sms);
  pdl(k_bkt_bases, persistent_grid(k_bkt_bases, sms), kThreads, 0, s, W);
  pdl(k_bkt_place, place, kThreads, 0, s, W, pin, kin, px, kx, 1);
  pdl(k_bkt_sort<0, kBktSmall>, persistent_grid(k_bkt_sort<0, kBktSmall>, sms, 256, small_smem), 256, small_smem, s, 
      W, px, kx, p0, k0, p1, k1);
  pdl(k_bkt_sort<kBktSmall, kBktMid>, persistent_grid(k_bkt_sort<kBktSmall, kBktMid>, sms, 256, mid_smem), 256, mid_smem, s, W, px, kx, p0, k0, p1, k1);
  pdl(k_bkt_sort<kBktMid, kBktCap>, persistent_grid(k_bkt_sort<kBktMid, kBktCap>, sms, 1024, big_smem), 1024, big_smem, s, W, px, kx, p0, k0, p1, k1);
}
void launch_tile_sort(const Wave &W, const uint32_t *pin, const SortKey *kin, uint32_t *pout, SortKey *kout,
                      cudaStream_t s, int sms) {
  pdl(k_tile_sort, persistent_grid(k_tile_sort, sms, 256), 256, 0, s, W, pin, kin, pout, kout);
}
void launch_merge_pass(const Wave &W, const uint32_t *pin, const SortKey *kin, uint32_t *pout, SortKey *kout,
                       uint64_t run, cudaStream_t s, int sms) {
  pdl(k_merge_split, persistent_grid(k_merge_split, sms), kThreads, 0, s, W, pin, kin, run);
  pdl(k_merge_tiles, persistent_grid(k_merge_tiles, sms, 256), 256, 0, s, W, pin, kin, pout, kout, run);
}
void launch_gather(const Wave &W, const uint32_t *perm0, const uint32_t *perm1, cudaStream_t s, int sms) {
  pdl(k_gather, persistent_grid(k_gather, sms), kThreads, 0, s, W, perm0, perm1);
}

void launch_project(const Wave &W, const uint32_t *perm0, const uint32_t *perm1, const SortKey *key0,
                    const SortKey *key1, uint64_t max_tiles, uint64_t *scan_tmp, cudaStream_t s, int sms) {
  const unsigned grid = (unsigned)std::min<uint64_t>(std::max<uint64_t>(max_tiles, 1), (uint64_t)sms * 8);
  pdl(k_proj_count, grid, 256, 0, s, W, perm0, perm1, key0, key1);
  scan_u32(W.ptcount, W.ptscan, &W.ctrl->len[7], max_tiles, scan_tmp, s, sms);
  pdl(k_proj_write, grid, 256, 0, s, W, perm0, perm1, key0, key1);
}
void launch_epilogue(const Wave &W, cudaStream_t s, int sms) {
  pdl(k_epilogue_copy, persistent_grid(k_epilogue_copy, sms), kThreads, 0, s, W);
  pdl(k_epilogue_advance, 1, 1, 0, s, W);
}

}  // namespace gs
