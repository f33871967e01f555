/*
 * CPU oracle for exact labeled subgraph matching (thesis Ch. 3, "GpSense").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  It shares no code, header
 * or table with the CUDA engine; the two meet only at the seeded inputs.
 *
 * Plain, slow and meant to be checked by eye against the definitions:
 *   - Definition 3.2 (subgraph isomorphism: an injective map f with every
 *     query edge mapped onto a data edge), applied to directed graphs whose
 *     edges carry relation labels (Section 3.2, "Commonsense Graph
 *     Transformation": concepts become vertex ids, relations edge labels),
 *     with bound ("concept") and variable query vertices (Section 3.2: a
 *     concept node maps to exactly one data node) and vertex types standing
 *     in for Definition 3.1's node labels;
 *   - Definition 3.3 (candidate: same label, degree(u) <= degree(v)), read
 *     per (direction, relation) pair over distinct neighbours;
 *   - the pruning rule of Algorithm "Candidate nodes initialization"
 *     (drop a candidate that has no candidate neighbour for some query
 *     neighbour) repeated "until no more can be pruned" (Section 3.3.3,
 *     "Candidate Nodes Refinement");
 *   - the candidate-edge tables of Section 3.3.4 ("Joining Phase");
 *   - projection (Section 3.5, "Modify the query plan": only the matches of
 *     a subset of the query vertices are wanted): the rows returned are the
 *     distinct tuples (f(u)) over the projected vertices u, ascending, while
 *     the count and fingerprint still cover every embedding;
 *   - variable edges (Section 3.2: a relation may itself be a variable):
 *     a query edge with relation ORC_ANY maps onto a data edge of any
 *     relation.  An embedding is still a map of vertices, so two data edges
 *     of different relations between the same pair count once.
 *
 * Every function keeps its own data structures: per-vertex adjacency built
 * from a sorted, de-duplicated triple array, and binary search in that array
 * for edge tests.
 *
 * Parity pins live in tests/test_oracle_pins.py (brute force over all
 * injective maps, closed-form counts, homomorphism projections, planted
 * mistakes).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define ORC_UNBOUND 0xFFFFFFFFu
#define ORC_ANY 0xFFFFFFFFu

typedef struct { uint32_t src, rel, dst; } orc_triple;

typedef struct {
  uint32_t V, T, R;
  uint64_t E;               /* distinct triples */
  orc_triple *by_src;       /* sorted by (src, rel, dst), de-duplicated */
  orc_triple *by_dst;       /* same triples sorted by (dst, rel, src) */
  uint64_t *src_begin;      /* [V+1] ranges into by_src */
  uint64_t *dst_begin;      /* [V+1] ranges into by_dst */
  uint32_t *vtype;          /* [V] */
} orc_graph;

static int cmp_src(const void *a, const void *b) {
  const orc_triple *x = (const orc_triple *)a, *y = (const orc_triple *)b;
  if (x->src != y->src) return x->src < y->src ? -1 : 1;
  if (x->rel != y->rel) return x->rel < y->rel ? -1 : 1;
  if (x->dst != y->dst) return x->dst < y->dst ? -1 : 1;
  return 0;
}
static int cmp_dst(const void *a, const void *b) {
  const orc_triple *x = (const orc_triple *)a, *y = (const orc_triple *)b;
  if (x->dst != y->dst) return x->dst < y->dst ? -1 : 1;
  if (x->rel != y->rel) return x->rel < y->rel ? -1 : 1;
  if (x->src != y->src) return x->src < y->src ? -1 : 1;
  return 0;
}

/* Build the oracle's graph from an out-CSR (any order, duplicates allowed).
 * Parallel (src, rel, dst) triples collapse into one: an embedding is a map
 * of vertices, so repeated triples never change the set of embeddings. */
orc_graph *orc_graph_build(uint32_t V, uint64_t E, const uint64_t *row_off, const uint32_t *col,
                           const uint32_t *rel, const uint32_t *vtype, uint32_t T, uint32_t R) {
  orc_graph *g = (orc_graph *)calloc(1, sizeof(orc_graph));
  g->V = V; g->T = T; g->R = R;
  g->by_src = (orc_triple *)malloc(sizeof(orc_triple) * (E ? E : 1));
  uint64_t n = 0;
  for (uint32_t s = 0; s < V; ++s)
    for (uint64_t e = row_off[s]; e < row_off[s + 1]; ++e) {
      g->by_src[n].src = s; g->by_src[n].rel = rel[e]; g->by_src[n].dst = col[e]; n++;
    }
  qsort(g->by_src, n, sizeof(orc_triple), cmp_src);
  uint64_t w = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (w == 0 || cmp_src(&g->by_src[i], &g->by_src[w - 1]) != 0) g->by_src[w++] = g->by_src[i];
  g->E = w;
  g->by_dst = (orc_triple *)malloc(sizeof(orc_triple) * (w ? w : 1));
  memcpy(g->by_dst, g->by_src, sizeof(orc_triple) * w);
  qsort(g->by_dst, w, sizeof(orc_triple), cmp_dst);
  g->src_begin = (uint64_t *)calloc(V + 1, sizeof(uint64_t));
  g->dst_begin = (uint64_t *)calloc(V + 1, sizeof(uint64_t));
  for (uint64_t i = 0; i < w; ++i) { g->src_begin[g->by_src[i].src + 1]++; g->dst_begin[g->by_dst[i].dst + 1]++; }
  for (uint32_t v = 0; v < V; ++v) { g->src_begin[v + 1] += g->src_begin[v]; g->dst_begin[v + 1] += g->dst_begin[v]; }
  g->vtype = (uint32_t *)malloc(sizeof(uint32_t) * (V ? V : 1));
  memcpy(g->vtype, vtype, sizeof(uint32_t) * V);
  return g;
}

void orc_graph_free(orc_graph *g) {
  if (!g) return;
  free(g->by_src); free(g->by_dst); free(g->src_begin); free(g->dst_begin); free(g->vtype); free(g);
}

uint64_t orc_graph_num_edges(const orc_graph *g) { return g->E; }

/* Is (a, r, b) a data edge?  Binary search in the (src, rel, dst) order;
 * r = ORC_ANY: is there a data edge a -> b of any relation (scan of a's
 * out-edges). */
static int orc_has_edge(const orc_graph *g, uint32_t a, uint32_t r, uint32_t b) {
  if (r == ORC_ANY) {
    for (uint64_t i = g->src_begin[a]; i < g->src_begin[a + 1]; ++i)
      if (g->by_src[i].dst == b) return 1;
    return 0;
  }
  orc_triple key = {a, r, b};
  uint64_t lo = g->src_begin[a], hi = g->src_begin[a + 1];
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    int c = cmp_src(&g->by_src[mid], &key);
    if (c == 0) return 1;
    if (c < 0) lo = mid + 1; else hi = mid;
  }
  return 0;
}

/* The neighbour of v held by entry t of its out-edges (dir 0) or in-edges
 * (dir 1), and that entry's relation. */
static uint32_t orc_nbr(const orc_graph *g, int dir, uint64_t t) { return dir == 0 ? g->by_src[t].dst : g->by_dst[t].src; }
static uint32_t orc_rel(const orc_graph *g, int dir, uint64_t t) { return dir == 0 ? g->by_src[t].rel : g->by_dst[t].rel; }
static uint64_t orc_begin(const orc_graph *g, int dir, uint32_t v) { return dir == 0 ? g->src_begin[v] : g->dst_begin[v]; }

/* Does entry t of v's edges in direction dir match relation r, and (for
 * r = ORC_ANY) is it the first of v's edges to its neighbour?  Walking v's
 * edges and keeping the entries for which this holds visits each neighbour
 * over r exactly once. */
static int orc_first_nbr(const orc_graph *g, int dir, uint32_t v, uint64_t t, uint32_t r) {
  if (r != ORC_ANY) return orc_rel(g, dir, t) == r;
  for (uint64_t i = orc_begin(g, dir, v); i < t; ++i)
    if (orc_nbr(g, dir, i) == orc_nbr(g, dir, t)) return 0;
  return 1;
}

/* Number of distinct out-neighbours of v over relation r (dir 0) or of
 * distinct in-neighbours (dir 1); r = ORC_ANY counts distinct neighbours
 * over all relations. */
static uint64_t orc_degree(const orc_graph *g, uint32_t v, int dir, uint32_t r) {
  uint64_t c = 0;
  if (r == ORC_ANY) {
    for (uint64_t t = orc_begin(g, dir, v); t < orc_begin(g, dir, v + 1); ++t) c += orc_first_nbr(g, dir, v, t, r);
    return c;
  }
  if (dir == 0) { for (uint64_t i = g->src_begin[v]; i < g->src_begin[v + 1]; ++i) c += g->by_src[i].rel == r; }
  else { for (uint64_t i = g->dst_begin[v]; i < g->dst_begin[v + 1]; ++i) c += g->by_dst[i].rel == r; }
  return c;
}

/* ---------------------------------------------------------------- query */
typedef struct {
  uint32_t k, m;
  const uint32_t *vtype, *vbind;
  uint32_t esrc[512], edst[512], erel[512];  /* de-duplicated edges */
} orc_query;

/* Copy a query, dropping repeated (src, dst, rel) edges.  Returns -1 for a
 * query the definition does not cover: k = 0, an endpoint out of range, a
 * self-loop, too many edges. */
static int orc_query_make(orc_query *q, uint32_t k, uint32_t m, const uint32_t *vtype, const uint32_t *vbind,
                          const uint32_t *esrc, const uint32_t *edst, const uint32_t *erel) {
  if (k == 0 || k > 32) return -1;
  q->k = k; q->vtype = vtype; q->vbind = vbind; q->m = 0;
  for (uint32_t e = 0; e < m; ++e) {
    if (esrc[e] >= k || edst[e] >= k || esrc[e] == edst[e]) return -1;
    int dup = 0;
    for (uint32_t j = 0; j < q->m; ++j)
      if (q->esrc[j] == esrc[e] && q->edst[j] == edst[e] && q->erel[j] == erel[e]) dup = 1;
    if (dup) continue;
    if (q->m >= 512) return -1;
    q->esrc[q->m] = esrc[e]; q->edst[q->m] = edst[e]; q->erel[q->m] = erel[e]; q->m++;
  }
  return 0;
}

/* Unary part of the match definition: binding and type. */
static int orc_unary_ok(const orc_graph *g, const orc_query *q, uint32_t u, uint32_t v) {
  if (q->vbind[u] != ORC_UNBOUND && q->vbind[u] != v) return 0;
  if (q->vtype[u] != ORC_ANY && g->vtype[v] != q->vtype[u]) return 0;
  return 1;
}

/* ----------------------------------------------------------- fingerprint */
/* splitmix64 finaliser (Steele, Lea & Flood 2014): the output function of
 * the splitmix64 generator, whose n-th output from seed s is
 * orc_mix64(s + n * 0x9E3779B97F4A7C15).  Exported so that the tests can pin
 * it to that generator's published outputs. */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
/* Hash of one embedding written in query-vertex order.  The fingerprint of a
 * result is the sum (mod 2^64) of this over every embedding: independent of
 * order, so truncated or chunked outputs can still be checked in full. */
uint64_t orc_row_hash(uint32_t k, const uint32_t *row) {
  uint64_t h = k;
  for (uint32_t i = 0; i < k; ++i) h = orc_mix64(h ^ ((uint64_t)row[i] + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull));
  return h;
}

/* Fingerprint of n rows of width k (row-major): the sum of their hashes. */
uint64_t orc_fingerprint(uint32_t k, const uint32_t *rows, uint64_t n) {
  uint64_t acc = 0;
  for (uint64_t i = 0; i < n; ++i) acc += orc_row_hash(k, rows + i * k);
  return acc;
}

/* --------------------------------------------------------- row collection */
typedef struct {
  uint32_t k;
  uint32_t w, proj[32];  /* stored row: f(proj[0]), ..., f(proj[w-1]) */
  uint64_t cap;          /* keep the cap lexicographically smallest distinct rows */
  uint64_t n, room;
  uint32_t *rows;
  uint64_t count, fp;
  int more;              /* more than cap distinct rows were seen */
} orc_sink;

static __thread uint32_t g_sort_k;
static int cmp_row(const void *a, const void *b) {
  const uint32_t *x = (const uint32_t *)a, *y = (const uint32_t *)b;
  for (uint32_t i = 0; i < g_sort_k; ++i) if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}
/* Sort the stored rows, drop repeats (only projected rows can repeat) and
 * keep the first cap. */
static void orc_sink_trim(orc_sink *s) {
  g_sort_k = s->w;
  qsort(s->rows, s->n, sizeof(uint32_t) * s->w, cmp_row);
  uint64_t d = 0;
  for (uint64_t i = 0; i < s->n; ++i)
    if (d == 0 || cmp_row(s->rows + (d - 1) * s->w, s->rows + i * s->w) != 0) {
      if (d != i) memcpy(s->rows + d * s->w, s->rows + i * s->w, sizeof(uint32_t) * s->w);
      d++;
    }
  s->n = d;
  if (s->n > s->cap) { s->n = s->cap; s->more = 1; }
}
static void orc_sink_put(orc_sink *s, const uint32_t *row) {
  s->count++;
  s->fp += orc_row_hash(s->k, row);
  if (s->cap == 0) return;
  if (s->n == s->room) orc_sink_trim(s);
  for (uint32_t i = 0; i < s->w; ++i) s->rows[s->n * s->w + i] = row[s->proj[i]];
  s->n++;
}

/* --------------------------------------------------------- backtracking */
typedef struct {
  const orc_graph *g;
  const orc_query *q;
  uint32_t order[32];
  uint32_t f[32];
  uint8_t *used;            /* [V] */
  orc_sink *sink;
  uint64_t nodes;
  double deadline;
  int timed_out;
} orc_bt;

static double orc_now(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

/* Does candidate v for query vertex i keep every query edge between i and
 * the already matched vertices order[0..depth) ? */
static int orc_edges_ok(orc_bt *b, uint32_t depth, uint32_t i, uint32_t v) {
  const orc_query *q = b->q;
  for (uint32_t e = 0; e < q->m; ++e) {
    uint32_t s = q->esrc[e], d = q->edst[e];
    if (s != i && d != i) continue;
    uint32_t other = s == i ? d : s;
    int matched = 0;
    for (uint32_t t = 0; t < depth; ++t) if (b->order[t] == other) matched = 1;
    if (!matched) continue;
    uint32_t a = s == i ? v : b->f[s], c = d == i ? v : b->f[d];
    if (!orc_has_edge(b->g, a, q->erel[e], c)) return 0;
  }
  return 1;
}

void orc_extend(orc_bt *b, uint32_t depth);

static void orc_try(orc_bt *b, uint32_t depth, uint32_t i, uint32_t v) {
  if (b->used[v]) return;
  if (!orc_unary_ok(b->g, b->q, i, v)) return;
  if (!orc_edges_ok(b, depth, i, v)) return;
  b->f[i] = v; b->used[v] = 1;
  orc_extend(b, depth + 1);
  b->used[v] = 0;
}

void orc_extend(orc_bt *b, uint32_t depth) {
  if (b->timed_out) return;
  if ((++b->nodes & 0xFFFF) == 0 && b->deadline > 0 && orc_now() > b->deadline) { b->timed_out = 1; return; }
  const orc_query *q = b->q;
  if (depth == q->k) { orc_sink_put(b->sink, b->f); return; }
  uint32_t i = b->order[depth];
  /* Iterate the data neighbours of one matched query neighbour when there is
   * one (first such edge in edge order), else every data vertex. */
  for (uint32_t e = 0; e < q->m; ++e) {
    uint32_t s = q->esrc[e], d = q->edst[e];
    if (s != i && d != i) continue;
    uint32_t other = s == i ? d : s;
    int matched = 0;
    for (uint32_t t = 0; t < depth; ++t) if (b->order[t] == other) matched = 1;
    if (!matched) continue;
    /* edge other -> i: out-neighbours of f(other) over relation r (dir 0);
     * edge i -> other: its in-neighbours (dir 1); each neighbour once */
    const orc_graph *g = b->g;
    const int dir = d == i ? 0 : 1;
    const uint32_t x = b->f[other];
    for (uint64_t t = orc_begin(g, dir, x); t < orc_begin(g, dir, x + 1); ++t)
      if (orc_first_nbr(g, dir, x, t, q->erel[e])) orc_try(b, depth, i, orc_nbr(g, dir, t));
    return;
  }
  for (uint32_t v = 0; v < b->g->V; ++v) orc_try(b, depth, i, v);
}

/*
 * orc_match_proj: every embedding of the query (Definition 3.2 read for
 * directed, relation-labelled graphs with bound and typed vertices).
 * Outputs: *count = number of embeddings; *fp = fingerprint (sum of
 * orc_row_hash over the embeddings); rows_out = the lexicographically
 * smallest min(D, cap) of the D distinct tuples (f(u)) over the query
 * vertices u in `project` (a bit mask, ascending u; 0 = every vertex, when
 * the tuples are the embeddings themselves), row-major [nrows][w];
 * *truncated = D > cap.  time_limit_s > 0 stops the search after that long
 * (returns 2).  Returns 0 on success, 1 for an invalid query, 2 on
 * time-out.
 *
 * Matching order: a bound vertex first (lowest index), else vertex 0; then
 * repeatedly the unmatched vertex with the most edges to matched vertices
 * (lowest index on ties).  The order only changes the running time.
 */
int orc_match_proj(const orc_graph *g, uint32_t k, uint32_t m, const uint32_t *vtype, const uint32_t *vbind,
                   const uint32_t *esrc, const uint32_t *edst, const uint32_t *erel, uint32_t project, uint64_t cap,
                   uint64_t *count, uint64_t *fp, uint32_t *rows_out, uint64_t *nrows, uint32_t *truncated,
                   double time_limit_s) {
  orc_query q;
  if (orc_query_make(&q, k, m, vtype, vbind, esrc, edst, erel) != 0) return 1;
  if (k < 32 && (project >> k) != 0) return 1;
  for (uint32_t u = 0; u < k; ++u) {
    if (vbind[u] != ORC_UNBOUND && vbind[u] >= g->V) return 1;
    if (vtype[u] != ORC_ANY && vtype[u] >= g->T) return 1;
  }
  for (uint32_t e = 0; e < q.m; ++e) if (q.erel[e] >= g->R && q.erel[e] != ORC_ANY) return 1;
  orc_bt b;
  memset(&b, 0, sizeof b);
  b.g = g; b.q = &q;
  uint8_t in_order[32] = {0};
  uint32_t first = 0;
  for (uint32_t u = 0; u < k; ++u) if (vbind[u] != ORC_UNBOUND) { first = u; break; }
  b.order[0] = first; in_order[first] = 1;
  for (uint32_t t = 1; t < k; ++t) {
    uint32_t best = k; int best_links = -1;
    for (uint32_t u = 0; u < k; ++u) {
      if (in_order[u]) continue;
      int links = 0;
      for (uint32_t e = 0; e < q.m; ++e)
        if ((q.esrc[e] == u && in_order[q.edst[e]]) || (q.edst[e] == u && in_order[q.esrc[e]])) links++;
      if (links > best_links) { best_links = links; best = u; }
    }
    b.order[t] = best; in_order[best] = 1;
  }
  orc_sink sink;
  memset(&sink, 0, sizeof sink);
  sink.k = k; sink.cap = cap;
  for (uint32_t u = 0; u < k; ++u)
    if (project == 0 || ((project >> u) & 1u)) sink.proj[sink.w++] = u;
  sink.room = cap == 0 ? 0 : (cap < (1u << 20) ? 2 * cap : cap + (1u << 20));
  sink.rows = cap ? (uint32_t *)malloc(sizeof(uint32_t) * sink.w * sink.room) : NULL;
  b.sink = &sink;
  b.used = (uint8_t *)calloc(g->V ? g->V : 1, 1);
  b.deadline = time_limit_s > 0 ? orc_now() + time_limit_s : 0;
  orc_extend(&b, 0);
  free(b.used);
  if (cap) orc_sink_trim(&sink);
  *count = sink.count; *fp = sink.fp; *nrows = sink.n;
  if (truncated) *truncated = cap ? (uint32_t)sink.more : (sink.count > 0);
  if (cap && rows_out) memcpy(rows_out, sink.rows, sizeof(uint32_t) * sink.w * sink.n);
  free(sink.rows);
  return b.timed_out ? 2 : 0;
}

/* orc_match_proj over every query vertex: rows are the embeddings. */
int orc_match(const orc_graph *g, uint32_t k, uint32_t m, const uint32_t *vtype, const uint32_t *vbind,
              const uint32_t *esrc, const uint32_t *edst, const uint32_t *erel, uint64_t cap,
              uint64_t *count, uint64_t *fp, uint32_t *rows_out, uint64_t *nrows, double time_limit_s) {
  return orc_match_proj(g, k, m, vtype, vbind, esrc, edst, erel, 0, cap, count, fp, rows_out, nrows, NULL,
                        time_limit_s);
}

/*
 * orc_match_many: orc_match over n queries (flat arrays with per-query
 * offsets), counts and fingerprints only, spread over `threads` OpenMP
 * threads (0 = all).  status[i] as orc_match.  Returns the thread count used.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
int orc_match_many(const orc_graph *g, uint32_t n, const uint32_t *qk, const uint32_t *qm,
                   const uint64_t *voff, const uint64_t *eoff, const uint32_t *vtype, const uint32_t *vbind,
                   const uint32_t *esrc, const uint32_t *edst, const uint32_t *erel, int threads,
                   double time_limit_s, uint64_t *count, uint64_t *fp, int *status) {
  int used = 1;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
      uint64_t nr;
      status[i] = orc_match(g, qk[i], qm[i], vtype + voff[i], vbind + voff[i], esrc + eoff[i], edst + eoff[i],
                            erel + eoff[i], 0, &count[i], &fp[i], NULL, &nr, time_limit_s);
    }
  }
#else
  (void)threads;
  for (uint32_t i = 0; i < n; ++i) {
    uint64_t nr;
    status[i] = orc_match(g, qk[i], qm[i], vtype + voff[i], vbind + voff[i], esrc + eoff[i], edst + eoff[i],
                          erel + eoff[i], 0, &count[i], &fp[i], NULL, &nr, time_limit_s);
  }
#endif
  return used;
}

/*
 * orc_brute: the same outputs as orc_match by trying every injective map
 * [0,k) -> V in lexicographic order and keeping those that satisfy the
 * definition.  Exponential; for tiny graphs only.
 */
int orc_brute(const orc_graph *g, uint32_t k, uint32_t m, const uint32_t *vtype, const uint32_t *vbind,
              const uint32_t *esrc, const uint32_t *edst, const uint32_t *erel, uint64_t cap,
              uint64_t *count, uint64_t *fp, uint32_t *rows_out, uint64_t *nrows) {
  orc_query q;
  if (orc_query_make(&q, k, m, vtype, vbind, esrc, edst, erel) != 0) return 1;
  if (g->V < k) { *count = 0; *fp = 0; *nrows = 0; return 0; }
  uint32_t f[32];
  for (uint32_t i = 0; i < k; ++i) f[i] = 0;
  uint64_t c = 0, h = 0, nr = 0;
  for (;;) {
    int ok = 1;
    for (uint32_t i = 0; i < k && ok; ++i)
      for (uint32_t j = i + 1; j < k && ok; ++j) if (f[i] == f[j]) ok = 0;
    for (uint32_t i = 0; i < k && ok; ++i) if (!orc_unary_ok(g, &q, i, f[i])) ok = 0;
    for (uint32_t e = 0; e < q.m && ok; ++e) if (!orc_has_edge(g, f[q.esrc[e]], q.erel[e], f[q.edst[e]])) ok = 0;
    if (ok) {
      c++; h += orc_row_hash(k, f);
      if (nr < cap && rows_out) { memcpy(rows_out + nr * k, f, sizeof(uint32_t) * k); nr++; }
    }
    /* next map in lexicographic order */
    int32_t i = (int32_t)k - 1;
    while (i >= 0 && f[i] == g->V - 1) { f[i] = 0; --i; }
    if (i < 0) break;
    f[i]++;
  }
  *count = c; *fp = h; *nrows = nr;
  return 0;
}

/*
 * orc_candidates: C0(u) for every query vertex, as a [k][V] byte matrix
 * (1 = candidate).  v is a candidate of u when the binding and the type
 * allow it and, for every direction and relation, v has at least as many
 * distinct neighbours as u has query neighbours (Definition 3.3's degree
 * test, read per direction and relation; the variable relation ORC_ANY is
 * one more relation whose neighbours are all of v's distinct neighbours in
 * that direction, needed by u's variable edges only).  signature = 0 leaves
 * the degree test out (binding and type only).
 */
int orc_candidates(const orc_graph *g, uint32_t k, uint32_t m, const uint32_t *vtype, const uint32_t *vbind,
                   const uint32_t *esrc, const uint32_t *edst, const uint32_t *erel, int signature,
                   uint8_t *out) {
  orc_query q;
  if (orc_query_make(&q, k, m, vtype, vbind, esrc, edst, erel) != 0) return 1;
  for (uint32_t u = 0; u < k; ++u)
    for (uint32_t v = 0; v < g->V; ++v) {
      int ok = orc_unary_ok(g, &q, u, v);
      if (ok && signature) {
        for (uint32_t e = 0; e < q.m && ok; ++e) {
          int dir;
          if (q.esrc[e] == u) dir = 0; else if (q.edst[e] == u) dir = 1; else continue;
          uint64_t need = 0;
          for (uint32_t f = 0; f < q.m; ++f)
            if (q.erel[f] == q.erel[e] && ((dir == 0 && q.esrc[f] == u) || (dir == 1 && q.edst[f] == u))) need++;
          if (orc_degree(g, v, dir, q.erel[e]) < need) ok = 0;
        }
      }
      out[(uint64_t)u * g->V + v] = (uint8_t)ok;
    }
  return 0;
}

/*
 * orc_refine: the refinement of Section 3.3.3 run until nothing changes.
 * For every query edge (a -> b, r): a candidate x of a stays only if some
 * candidate y of b has (x, r, y) in E, and a candidate y of b stays only if
 * some candidate x of a has (x, r, y) in E (r = ORC_ANY: an edge of any
 * relation).  sets is [k][V] bytes, updated in place.  Returns the number of
 * passes over the edges.
 */
int orc_refine(const orc_graph *g, uint32_t k, uint32_t m, const uint32_t *vtype, const uint32_t *vbind,
               const uint32_t *esrc, const uint32_t *edst, const uint32_t *erel, uint8_t *sets) {
  orc_query q;
  if (orc_query_make(&q, k, m, vtype, vbind, esrc, edst, erel) != 0) return -1;
  int passes = 0, changed = 1;
  while (changed) {
    changed = 0; passes++;
    for (uint32_t e = 0; e < q.m; ++e) {
      uint32_t a = q.esrc[e], b = q.edst[e], r = q.erel[e];
      uint8_t *sa = sets + (uint64_t)a * g->V, *sb = sets + (uint64_t)b * g->V;
      for (uint32_t x = 0; x < g->V; ++x) {
        if (!sa[x]) continue;
        int found = 0;
        for (uint64_t t = g->src_begin[x]; t < g->src_begin[x + 1] && !found; ++t)
          if ((r == ORC_ANY || g->by_src[t].rel == r) && sb[g->by_src[t].dst]) found = 1;
        if (!found) { sa[x] = 0; changed = 1; }
      }
      for (uint32_t y = 0; y < g->V; ++y) {
        if (!sb[y]) continue;
        int found = 0;
        for (uint64_t t = g->dst_begin[y]; t < g->dst_begin[y + 1] && !found; ++t)
          if ((r == ORC_ANY || g->by_dst[t].rel == r) && sa[g->by_dst[t].src]) found = 1;
        if (!found) { sb[y] = 0; changed = 1; }
      }
    }
  }
  return passes;
}

/*
 * orc_edge_table: the candidate edges of query edge e (Section 3.3.4).
 * from_src = 1: keys are the candidates x of esrc[e] in ascending order and
 * the list of key x holds every y with (x, r, y) in E and y a candidate of
 * edst[e]; from_src = 0: keys are the candidates y of edst[e] and each list
 * holds every x with (x, r, y) in E and x a candidate of esrc[e].
 * Lists ascend and hold each vertex once (r = ORC_ANY: edges of any
 * relation).  Outputs keys[nkeys], off[nkeys+1], vals[off[nkeys]]; with
 * vals == NULL only *nkeys and *nvals are written.  e indexes the query's
 * edges as given (before de-duplication).
 */
int orc_edge_table(const orc_graph *g, uint32_t k, uint32_t m, const uint32_t *esrc, const uint32_t *edst,
                   const uint32_t *erel, const uint8_t *sets, uint32_t e, int from_src, uint32_t *keys,
                   uint64_t *off, uint32_t *vals, uint64_t *nkeys, uint64_t *nvals) {
  if (e >= m || esrc[e] >= k || edst[e] >= k) return 1;
  uint32_t a = esrc[e], b = edst[e], r = erel[e];
  uint32_t x = from_src ? a : b, y = from_src ? b : a;
  const uint8_t *sx = sets + (uint64_t)x * g->V, *sy = sets + (uint64_t)y * g->V;
  uint64_t nk = 0, nv = 0;
  for (uint32_t v = 0; v < g->V; ++v) {
    if (!sx[v]) continue;
    if (vals) { keys[nk] = v; off[nk] = nv; }
    nk++;
    const int dir = from_src ? 0 : 1;
    const uint64_t first = nv;
    for (uint64_t t = orc_begin(g, dir, v); t < orc_begin(g, dir, v + 1); ++t)
      if (orc_first_nbr(g, dir, v, t, r) && sy[orc_nbr(g, dir, t)]) { if (vals) vals[nv] = orc_nbr(g, dir, t); nv++; }
    /* a relation's entries ascend by neighbour; over all relations they do
     * not, so sort the list (insertion sort) */
    if (vals && r == ORC_ANY)
      for (uint64_t i = first + 1; i < nv; ++i)
        for (uint64_t j = i; j > first && vals[j - 1] > vals[j]; --j) { uint32_t t = vals[j]; vals[j] = vals[j - 1]; vals[j - 1] = t; }
  }
  if (vals) off[nk] = nv;
  *nkeys = nk; *nvals = nv;
  return 0;
}

/*
 * orc_verify: check rows [n][k] edge by edge against the definition.
 * Returns the index of the first row that is not an embedding, or -1.
 */
int64_t orc_verify(const orc_graph *g, uint32_t k, uint32_t m, const uint32_t *vtype, const uint32_t *vbind,
                   const uint32_t *esrc, const uint32_t *edst, const uint32_t *erel, const uint32_t *rows,
                   uint64_t n) {
  orc_query q;
  if (orc_query_make(&q, k, m, vtype, vbind, esrc, edst, erel) != 0) return 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint32_t *f = rows + i * k;
    for (uint32_t a = 0; a < k; ++a) {
      if (f[a] >= g->V || !orc_unary_ok(g, &q, a, f[a])) return (int64_t)i;
      for (uint32_t b = a + 1; b < k; ++b) if (f[a] == f[b]) return (int64_t)i;
    }
    for (uint32_t e = 0; e < q.m; ++e)
      if (!orc_has_edge(g, f[q.esrc[e]], q.erel[e], f[q.edst[e]])) return (int64_t)i;
  }
  return -1;
}

/*
 * orc_khop: domain-graph exploration (Ch. 5, "Domain-specific knowledge
 * graph generation": the knowledge graph explored a few levels out from
 * chosen seed concepts).  level_out[v] = the number of hops of a shortest path
 * from any seed to v, when that is at most `levels`, else 255.  A hop
 * follows a data edge forwards (dirs bit 0) or backwards (dirs bit 1) whose
 * relation r has bit r set in relmask (8 words, 256 relations).  Plain
 * breadth-first search with a queue.  counts[l] = vertices at level l
 * (levels + 1 entries).  Returns 1 for a seed out of range, else 0.
 */
int orc_khop(const orc_graph *g, const uint32_t *seeds, uint32_t nseeds, uint32_t levels, uint32_t dirs,
             const uint32_t *relmask, uint8_t *level_out, uint64_t *counts) {
  for (uint32_t i = 0; i < nseeds; ++i) if (seeds[i] >= g->V) return 1;
  for (uint32_t v = 0; v < g->V; ++v) level_out[v] = 255;
  for (uint32_t l = 0; l <= levels; ++l) counts[l] = 0;
  uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * (g->V ? g->V : 1));
  uint64_t head = 0, tail = 0;
  for (uint32_t i = 0; i < nseeds; ++i)
    if (level_out[seeds[i]] == 255) { level_out[seeds[i]] = 0; queue[tail++] = seeds[i]; counts[0]++; }
  while (head < tail) {
    const uint32_t u = queue[head++];
    const uint32_t l = level_out[u];
    if (l >= levels) continue;
    for (int dir = 0; dir < 2; ++dir) {
      if (!((dirs >> dir) & 1u)) continue;
      for (uint64_t t = orc_begin(g, dir, u); t < orc_begin(g, dir, u + 1); ++t) {
        const uint32_t r = orc_rel(g, dir, t), w = orc_nbr(g, dir, t);
        if (!((relmask[r >> 5] >> (r & 31)) & 1u) || level_out[w] != 255) continue;
        level_out[w] = (uint8_t)(l + 1);
        counts[l + 1]++;
        queue[tail++] = w;
      }
    }
  }
  free(queue);
  return 0;
}

/* ================================================ multi-level compression
 * Section 3.4 ("Multi-level Graph Compression") and Section 3.5 (matching on
 * the weighted graph, then expanding through the mapping lists), read for
 * directed graphs whose edges carry relations and whose vertices carry types.
 *
 * Weighted graph G_i (Definition 3.4): its nodes are groups of data vertices
 * (the mapping list M(x) of node x); there is an edge (x, r, y), x != y,
 * when some a in M(x), b in M(y) have (a, r, b) in E.  Edges inside one
 * group are not edges of G_i: the node weight accounts for them.
 *
 * Weights, per direction d (0 = out, 1 = in) and relation r:
 *   - node weight w_{d,r}(x) = max over a in M(x) of the number of distinct
 *     d-neighbours of a over r that lie in M(x) (the thesis's "maximum degree
 *     among nodes in the graph constructed by" the merged lists, per plane);
 *   - edge weights start at 1 on every data edge and, when the nodes p, q of
 *     a level merge into u and n, m into v, become the thesis's
 *     w(u, v) = max(w(p, n), w(q, n)) + max(w(p, m), w(q, m)) (a missing
 *     edge weighs 0, an unmerged node is its own only part).  wout(x, r, y)
 *     bounds the r-out-neighbours in M(y) of any a in M(x); win(x, r, y), the
 *     same recursion with the roles of the two ends swapped, bounds the
 *     r-in-neighbours in M(x) of any b in M(y).
 *
 * Similar nodes (garbled in the thesis: its test max(|adj(u)| / |common|,
 * |adj(v)| / |common|) >= delta always holds for 0 < delta <= 1).  Reading:
 * x and y have the same type and common(x, y) makes up at least delta of
 * each adjacency, |common| >= delta * |adj(x)| and |common| >= delta *
 * |adj(y)|, where adj(x) = the (direction, relation, neighbour node) triples
 * of x's edges in G_i and common(x, y) = adj(x) intersected with adj(y)
 * (Section 3.4: an edge to/from v with the same label from both); with
 * delta = 1 similar nodes have the same adjacency list, as in the thesis's
 * example.  Two nodes without edges are similar; one without edges is
 * similar to no node with edges.  The comparisons are the double-precision
 * products (double)|common| >= delta * (double)|adj|.
 *
 * Each level combines pairs of similar nodes (Section 3.4: a weighted node of
 * G_i is a combination of two nodes of G_{i-1}): nodes are visited in
 * ascending index order, and a node not yet paired is paired with the
 * lowest-indexed later node that is not paired and is similar to it.  The
 * nodes of G_i are numbered by ascending smallest member (level 0: node v =
 * vertex v).
 * ====================================================================== */
typedef struct {
  uint32_t V, T, R, n;  /* data vertices, types, relations, weighted nodes */
  uint32_t *group;      /* [V] node whose mapping list holds v */
  uint32_t *moff;       /* [n+1] mapping lists: mem[moff[x] .. moff[x+1]), ascending */
  uint32_t *mem;        /* [V] */
  uint32_t *type;       /* [n] */
  uint64_t ne;          /* edges between different nodes */
  orc_triple *e;        /* [ne] sorted by (src, rel, dst) */
  uint32_t *wout, *win; /* [ne] */
  uint32_t *wnode;      /* [(d * R + r) * n + x] node weight per direction and relation */
} orc_wgraph;

typedef struct { uint32_t src, rel, dst, wout, win; } orc_wedge;

static int cmp_wedge(const void *a, const void *b) { return cmp_src(a, b); }

typedef struct { uint32_t node; uint64_t key; } orc_adjkey;
static int cmp_adjkey(const void *a, const void *b) {
  const orc_adjkey *x = (const orc_adjkey *)a, *y = (const orc_adjkey *)b;
  if (x->node != y->node) return x->node < y->node ? -1 : 1;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return 0;
}

/* One compression level: pair similar nodes of the weighted graph
 * (n nodes, edges e[ne] with weights, node types) and write the merged
 * level.  newidx[x] = x's node at the next level.  Returns the new node
 * count. */
static uint32_t orc_level_pairs(uint32_t n, const uint32_t *type, const orc_wedge *e, uint64_t ne, double delta,
                                uint32_t *newidx) {
  /* adjacency lists: (out, r, y) for x -> y and (in, r, x) for x -> y at y */
  orc_adjkey *ak = (orc_adjkey *)malloc(sizeof(orc_adjkey) * (2 * ne + 1));
  for (uint64_t i = 0; i < ne; ++i) {
    ak[2 * i].node = e[i].src;
    ak[2 * i].key = ((uint64_t)0 << 40) | ((uint64_t)e[i].rel << 32) | e[i].dst;
    ak[2 * i + 1].node = e[i].dst;
    ak[2 * i + 1].key = ((uint64_t)1 << 40) | ((uint64_t)e[i].rel << 32) | e[i].src;
  }
  qsort(ak, 2 * ne, sizeof(orc_adjkey), cmp_adjkey);
  uint64_t *aoff = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
  for (uint64_t i = 0; i < 2 * ne; ++i) aoff[ak[i].node + 1]++;
  for (uint32_t x = 0; x < n; ++x) aoff[x + 1] += aoff[x];
  int64_t *partner = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
  for (uint32_t x = 0; x < n; ++x) partner[x] = -1;
  for (uint32_t x = 0; x < n; ++x) {
    if (partner[x] >= 0) continue;
    for (uint32_t y = x + 1; y < n; ++y) {
      if (partner[y] >= 0 || type[y] != type[x]) continue;
      const uint64_t a = aoff[x + 1] - aoff[x], b = aoff[y + 1] - aoff[y];
      int similar;
      if (a == 0 || b == 0) {
        similar = a == 0 && b == 0;
      } else {
        uint64_t c = 0, i = aoff[x], j = aoff[y];
        while (i < aoff[x + 1] && j < aoff[y + 1]) {
          if (ak[i].key == ak[j].key) { c++; i++; j++; }
          else if (ak[i].key < ak[j].key) i++;
          else j++;
        }
        similar = (double)c >= delta * (double)a && (double)c >= delta * (double)b;
      }
      if (similar) { partner[x] = y; partner[y] = x; break; }
    }
  }
  uint32_t cnt = 0;
  for (uint32_t x = 0; x < n; ++x) {
    if (partner[x] >= 0 && (uint32_t)partner[x] < x) continue;  /* numbered with its lower partner */
    newidx[x] = cnt;
    if (partner[x] >= 0) newidx[partner[x]] = cnt;
    cnt++;
  }
  free(ak); free(aoff); free(partner);
  return cnt;
}

/* Edges of the merged level with the thesis's weight recursion.  Old edge
 * (A, r, B) -> new edge (U, r, V) with U = newidx[A], V = newidx[B]; U == V
 * (an edge inside a merged node) is dropped.  wout(U, r, V) = sum over the
 * parts B of V of the max over the parts A of U of wout(A, r, B); win(U, r, V)
 * = sum over the parts A of U of the max over the parts B of V of
 * win(A, r, B). */
typedef struct { uint32_t u, rel, v, a, b, wout, win; } orc_lift;
static int cmp_lift_b(const void *p, const void *q) {  /* (u, rel, v, b) */
  const orc_lift *x = (const orc_lift *)p, *y = (const orc_lift *)q;
  if (x->u != y->u) return x->u < y->u ? -1 : 1;
  if (x->rel != y->rel) return x->rel < y->rel ? -1 : 1;
  if (x->v != y->v) return x->v < y->v ? -1 : 1;
  if (x->b != y->b) return x->b < y->b ? -1 : 1;
  return 0;
}
static int cmp_lift_a(const void *p, const void *q) {  /* (u, rel, v, a) */
  const orc_lift *x = (const orc_lift *)p, *y = (const orc_lift *)q;
  if (x->u != y->u) return x->u < y->u ? -1 : 1;
  if (x->rel != y->rel) return x->rel < y->rel ? -1 : 1;
  if (x->v != y->v) return x->v < y->v ? -1 : 1;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  return 0;
}
static orc_wedge *orc_level_edges(const orc_wedge *e, uint64_t ne, const uint32_t *newidx, uint64_t *ne_out) {
  orc_lift *l = (orc_lift *)malloc(sizeof(orc_lift) * (ne ? ne : 1));
  uint64_t nl = 0;
  for (uint64_t i = 0; i < ne; ++i) {
    const uint32_t u = newidx[e[i].src], v = newidx[e[i].dst];
    if (u == v) continue;
    l[nl].u = u; l[nl].rel = e[i].rel; l[nl].v = v; l[nl].a = e[i].src; l[nl].b = e[i].dst;
    l[nl].wout = e[i].wout; l[nl].win = e[i].win; nl++;
  }
  orc_wedge *out = (orc_wedge *)malloc(sizeof(orc_wedge) * (nl ? nl : 1));
  uint64_t no = 0;
  /* wout: per (u, rel, v, b) the max over a, summed over b */
  qsort(l, nl, sizeof(orc_lift), cmp_lift_b);
  for (uint64_t i = 0; i < nl;) {
    uint64_t j = i;
    uint32_t sum = 0;
    while (j < nl && l[j].u == l[i].u && l[j].rel == l[i].rel && l[j].v == l[i].v) {
      uint32_t mx = 0;
      const uint32_t b = l[j].b;
      while (j < nl && l[j].u == l[i].u && l[j].rel == l[i].rel && l[j].v == l[i].v && l[j].b == b) {
        if (l[j].wout > mx) mx = l[j].wout;
        j++;
      }
      sum += mx;
    }
    out[no].src = l[i].u; out[no].rel = l[i].rel; out[no].dst = l[i].v; out[no].wout = sum; out[no].win = 0; no++;
    i = j;
  }
  /* win: per (u, rel, v, a) the max over b, summed over a (same edge order) */
  qsort(l, nl, sizeof(orc_lift), cmp_lift_a);
  uint64_t k = 0;
  for (uint64_t i = 0; i < nl;) {
    uint64_t j = i;
    uint32_t sum = 0;
    while (j < nl && l[j].u == l[i].u && l[j].rel == l[i].rel && l[j].v == l[i].v) {
      uint32_t mx = 0;
      const uint32_t a = l[j].a;
      while (j < nl && l[j].u == l[i].u && l[j].rel == l[i].rel && l[j].v == l[i].v && l[j].a == a) {
        if (l[j].win > mx) mx = l[j].win;
        j++;
      }
      sum += mx;
    }
    out[k++].win = sum;  /* both passes visit the (u, rel, v) groups in the same order */
    i = j;
  }
  free(l);
  *ne_out = no;
  return out;
}

void orc_wgraph_free(orc_wgraph *w) {
  if (!w) return;
  free(w->group); free(w->moff); free(w->mem); free(w->type); free(w->e); free(w->wout); free(w->win);
  free(w->wnode); free(w);
}

/*
 * orc_compress: `levels` levels of compression of g with thresholds
 * delta[0..levels).  Returns the final weighted graph (levels = 0: g itself
 * with unit weights).
 */
orc_wgraph *orc_compress(const orc_graph *g, uint32_t levels, const double *delta) {
  const uint32_t V = g->V, R = g->R;
  uint32_t n = V;
  uint32_t *group = (uint32_t *)malloc(sizeof(uint32_t) * (V ? V : 1));
  uint32_t *type = (uint32_t *)malloc(sizeof(uint32_t) * (V ? V : 1));
  for (uint32_t v = 0; v < V; ++v) { group[v] = v; type[v] = g->vtype[v]; }
  /* level 0: the data edges between different vertices, weight 1 */
  orc_wedge *e = (orc_wedge *)malloc(sizeof(orc_wedge) * (g->E ? g->E : 1));
  uint64_t ne = 0;
  for (uint64_t i = 0; i < g->E; ++i) {
    if (g->by_src[i].src == g->by_src[i].dst) continue;
    e[ne].src = g->by_src[i].src; e[ne].rel = g->by_src[i].rel; e[ne].dst = g->by_src[i].dst;
    e[ne].wout = 1; e[ne].win = 1; ne++;
  }
  uint32_t *newidx = (uint32_t *)malloc(sizeof(uint32_t) * (V ? V : 1));
  for (uint32_t lv = 0; lv < levels; ++lv) {
    const uint32_t n2 = orc_level_pairs(n, type, e, ne, delta[lv], newidx);
    uint64_t ne2 = 0;
    orc_wedge *e2 = orc_level_edges(e, ne, newidx, &ne2);
    uint32_t *type2 = (uint32_t *)malloc(sizeof(uint32_t) * (n2 ? n2 : 1));
    for (uint32_t x = 0; x < n; ++x) type2[newidx[x]] = type[x];
    for (uint32_t v = 0; v < V; ++v) group[v] = newidx[group[v]];
    free(e); free(type);
    e = e2; ne = ne2; type = type2; n = n2;
  }
  free(newidx);
  orc_wgraph *w = (orc_wgraph *)calloc(1, sizeof(orc_wgraph));
  w->V = V; w->T = g->T; w->R = R; w->n = n; w->group = group; w->type = type;
  /* mapping lists (members ascending) */
  w->moff = (uint32_t *)calloc(n + 1, sizeof(uint32_t));
  w->mem = (uint32_t *)malloc(sizeof(uint32_t) * (V ? V : 1));
  for (uint32_t v = 0; v < V; ++v) w->moff[group[v] + 1]++;
  for (uint32_t x = 0; x < n; ++x) w->moff[x + 1] += w->moff[x];
  uint32_t *fill = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  for (uint32_t x = 0; x < n; ++x) fill[x] = w->moff[x];
  for (uint32_t v = 0; v < V; ++v) w->mem[fill[group[v]]++] = v;
  free(fill);
  /* edges sorted by (src, rel, dst) */
  qsort(e, ne, sizeof(orc_wedge), cmp_wedge);
  w->ne = ne;
  w->e = (orc_triple *)malloc(sizeof(orc_triple) * (ne ? ne : 1));
  w->wout = (uint32_t *)malloc(sizeof(uint32_t) * (ne ? ne : 1));
  w->win = (uint32_t *)malloc(sizeof(uint32_t) * (ne ? ne : 1));
  for (uint64_t i = 0; i < ne; ++i) {
    w->e[i].src = e[i].src; w->e[i].rel = e[i].rel; w->e[i].dst = e[i].dst;
    w->wout[i] = e[i].wout; w->win[i] = e[i].win;
  }
  free(e);
  /* node weights, straight from the data graph */
  w->wnode = (uint32_t *)calloc((uint64_t)2 * R * (n ? n : 1), sizeof(uint32_t));
  for (uint32_t a = 0; a < V; ++a) {
    const uint32_t x = group[a];
    for (int dir = 0; dir < 2; ++dir)
      for (uint32_t r = 0; r < R; ++r) {
        uint32_t c = 0;
        for (uint64_t t = orc_begin(g, dir, a); t < orc_begin(g, dir, a + 1); ++t)
          if (orc_rel(g, dir, t) == r && group[orc_nbr(g, dir, t)] == x) c++;
        uint32_t *slot = &w->wnode[((uint64_t)dir * R + r) * n + x];
        if (c > *slot) *slot = c;
      }
  }
  return w;
}

uint32_t orc_wgraph_nodes(const orc_wgraph *w) { return w->n; }
uint64_t orc_wgraph_edges(const orc_wgraph *w) { return w->ne; }
/* Copy out the weighted graph: group[V], moff[n+1], mem[V], type[n],
 * edges src/rel/dst/wout/win [ne], wnode[2 * R * n] (any may be NULL). */
void orc_wgraph_get(const orc_wgraph *w, uint32_t *group, uint32_t *moff, uint32_t *mem, uint32_t *type,
                    uint32_t *src, uint32_t *rel, uint32_t *dst, uint32_t *wout, uint32_t *win, uint32_t *wnode) {
  if (group) memcpy(group, w->group, sizeof(uint32_t) * w->V);
  if (moff) memcpy(moff, w->moff, sizeof(uint32_t) * (w->n + 1));
  if (mem) memcpy(mem, w->mem, sizeof(uint32_t) * w->V);
  if (type) memcpy(type, w->type, sizeof(uint32_t) * w->n);
  for (uint64_t i = 0; i < w->ne; ++i) {
    if (src) src[i] = w->e[i].src;
    if (rel) rel[i] = w->e[i].rel;
    if (dst) dst[i] = w->e[i].dst;
    if (wout) wout[i] = w->wout[i];
    if (win) win[i] = w->win[i];
  }
  if (wnode) memcpy(wnode, w->wnode, sizeof(uint32_t) * 2 * w->R * w->n);
}

/* Is there a weighted edge (x, r, y) (x != y), or, for x == y, an edge of
 * relation r inside x (node weight > 0)?  r = ORC_ANY: any relation. */
static int orc_wedge_exists(const orc_wgraph *w, uint32_t x, uint32_t r, uint32_t y) {
  if (x == y) {
    for (uint32_t rr = 0; rr < w->R; ++rr)
      if ((r == ORC_ANY || rr == r) && w->wnode[(uint64_t)rr * w->n + x] > 0) return 1;
    return 0;
  }
  for (uint64_t i = 0; i < w->ne; ++i)  /* plain scan */
    if (w->e[i].src == x && w->e[i].dst == y && (r == ORC_ANY || w->e[i].rel == r)) return 1;
  return 0;
}

/* Definition 3.5's weight of node x in direction dir over relation r: its
 * node weight plus the weights of its edges (r = ORC_ANY: the sum over
 * every relation). */
static uint64_t orc_wbound(const orc_wgraph *w, uint32_t x, int dir, uint32_t r) {
  uint64_t s = 0;
  for (uint32_t rr = 0; rr < w->R; ++rr) {
    if (r != ORC_ANY && rr != r) continue;
    s += w->wnode[((uint64_t)dir * w->R + rr) * w->n + x];
    for (uint64_t i = 0; i < w->ne; ++i)
      if (w->e[i].rel == rr && (dir == 0 ? w->e[i].src : w->e[i].dst) == x) s += dir == 0 ? w->wout[i] : w->win[i];
  }
  return s;
}

/*
 * orc_wcandidates: Definition 3.5 on the weighted graph: node x is a
 * candidate of query vertex u when its type is u's (or u is untyped), u's
 * binding (a data vertex) lies in M(x), and for every direction and
 * relation the query degree of u is at most x's weight there.
 * sets[u * n + x] = 1 for candidates.  Returns 1 for an invalid query.
 */
int orc_wcandidates(const orc_wgraph *w, uint32_t k, uint32_t m, const uint32_t *vtype, const uint32_t *vbind,
                    const uint32_t *esrc, const uint32_t *edst, const uint32_t *erel, uint8_t *sets) {
  orc_query q;
  if (orc_query_make(&q, k, m, vtype, vbind, esrc, edst, erel) != 0) return 1;
  for (uint32_t u = 0; u < k; ++u)
    for (uint32_t x = 0; x < w->n; ++x) {
      int ok = (vtype[u] == ORC_ANY || w->type[x] == vtype[u]) &&
               (vbind[u] == ORC_UNBOUND || (vbind[u] < w->V && w->group[vbind[u]] == x));
      for (uint32_t e = 0; e < q.m && ok; ++e) {
        if (q.esrc[e] != u && q.edst[e] != u) continue;
        const int dir = q.esrc[e] == u ? 0 : 1;
        uint64_t need = 0;  /* query neighbours of u over this direction and relation */
        for (uint32_t f = 0; f < q.m; ++f)
          need += q.erel[f] == q.erel[e] && (dir == 0 ? q.esrc[f] == u : q.edst[f] == u);
        if (need > orc_wbound(w, x, dir, q.erel[e])) ok = 0;
      }
      sets[(uint64_t)u * w->n + x] = (uint8_t)ok;
    }
  return 0;
}

/*
 * orc_wrefine: the pruning rule of the refinement (Section 3.3.3) on the
 * weighted graph, repeated until nothing changes: candidate x of u stays when
 * every query edge at u has, at its other end w, a candidate y of w joined
 * to x by a weighted edge of that relation and direction, or y == x with an
 * edge of that relation inside x (two query vertices may map to one node of
 * the weighted graph).  sets as orc_wcandidates, refined in place.
 */
int orc_wrefine(const orc_wgraph *w, uint32_t k, uint32_t m, const uint32_t *esrc, const uint32_t *edst,
                const uint32_t *erel, uint8_t *sets) {
  int changed = 1, passes = 0;
  while (changed) {
    changed = 0; passes++;
    for (uint32_t e = 0; e < m; ++e) {
      const uint32_t a = esrc[e], b = edst[e], r = erel[e];
      if (a >= k || b >= k) return -1;
      uint8_t *sa = sets + (uint64_t)a * w->n, *sb = sets + (uint64_t)b * w->n;
      for (uint32_t x = 0; x < w->n; ++x) {
        if (!sa[x]) continue;
        int found = 0;
        for (uint32_t y = 0; y < w->n && !found; ++y) found = sb[y] && orc_wedge_exists(w, x, r, y);
        if (!found) { sa[x] = 0; changed = 1; }
      }
      for (uint32_t y = 0; y < w->n; ++y) {
        if (!sb[y]) continue;
        int found = 0;
        for (uint32_t x = 0; x < w->n && !found; ++x) found = sa[x] && orc_wedge_exists(w, x, r, y);
        if (!found) { sb[y] = 0; changed = 1; }
      }
    }
  }
  return passes;
}

/* Matching on the weighted graph (Section 3.5): every map h from the query
 * vertices to nodes with h(u) among u's refined candidates and every query
 * edge on a weighted edge (or inside a node); for each such h, the injective
 * maps f with f(u) in M(h(u)) that keep types, bindings and every query edge
 * in g go to the sink.  Every embedding f of the query in g arises from
 * exactly one h (h(u) = the node holding f(u)). */
typedef struct {
  const orc_graph *g;
  const orc_wgraph *w;
  const orc_query *q;
  const uint8_t *sets;
  uint32_t h[32], f[32];
  uint8_t *used;
  orc_sink *sink;
  uint64_t homs;
} orc_cbt;

static void orc_expand(orc_cbt *c, uint32_t u) {
  const orc_query *q = c->q;
  if (u == q->k) { orc_sink_put(c->sink, c->f); return; }
  const uint32_t x = c->h[u];
  for (uint32_t i = c->w->moff[x]; i < c->w->moff[x + 1]; ++i) {
    const uint32_t v = c->w->mem[i];
    if (c->used[v] || !orc_unary_ok(c->g, q, u, v)) continue;
    int ok = 1;
    for (uint32_t e = 0; e < q->m && ok; ++e) {
      const uint32_t s = q->esrc[e], d = q->edst[e];
      if ((s == u && d < u) || (d == u && s < u))
        ok = orc_has_edge(c->g, s == u ? v : c->f[s], q->erel[e], d == u ? v : c->f[d]);
    }
    if (!ok) continue;
    c->f[u] = v; c->used[v] = 1;
    orc_expand(c, u + 1);
    c->used[v] = 0;
  }
}

static void orc_hom(orc_cbt *c, uint32_t u) {
  const orc_query *q = c->q;
  if (u == q->k) { c->homs++; orc_expand(c, 0); return; }
  for (uint32_t x = 0; x < c->w->n; ++x) {
    if (!c->sets[(uint64_t)u * c->w->n + x]) continue;
    int ok = 1;
    for (uint32_t e = 0; e < q->m && ok; ++e) {
      const uint32_t s = q->esrc[e], d = q->edst[e];
      if ((s == u && d < u) || (d == u && s < u))
        ok = orc_wedge_exists(c->w, s == u ? x : c->h[s], q->erel[e], d == u ? x : c->h[d]);
    }
    if (!ok) continue;
    c->h[u] = x;
    orc_hom(c, u + 1);
  }
}

/*
 * orc_match_compressed: the embeddings of the query in g found through the
 * weighted graph: Definition 3.5's candidates on w, refined to the fixpoint,
 * every weighted-graph solution h, and each expanded through the mapping
 * lists.  Outputs as orc_match, plus *homs = the number of weighted-graph
 * solutions.  Returns 1 for an invalid query.
 */
int orc_match_compressed(const orc_graph *g, const orc_wgraph *w, uint32_t k, uint32_t m, const uint32_t *vtype,
                         const uint32_t *vbind, const uint32_t *esrc, const uint32_t *edst, const uint32_t *erel,
                         uint64_t cap, uint64_t *count, uint64_t *fp, uint32_t *rows_out, uint64_t *nrows,
                         uint64_t *homs) {
  orc_query q;
  if (orc_query_make(&q, k, m, vtype, vbind, esrc, edst, erel) != 0) return 1;
  for (uint32_t u = 0; u < k; ++u) {
    if (vbind[u] != ORC_UNBOUND && vbind[u] >= g->V) return 1;
    if (vtype[u] != ORC_ANY && vtype[u] >= g->T) return 1;
  }
  for (uint32_t e = 0; e < q.m; ++e) if (q.erel[e] >= g->R && q.erel[e] != ORC_ANY) return 1;
  uint8_t *sets = (uint8_t *)malloc((uint64_t)k * (w->n ? w->n : 1));
  orc_wcandidates(w, k, m, vtype, vbind, esrc, edst, erel, sets);
  orc_wrefine(w, k, q.m, q.esrc, q.edst, q.erel, sets);
  orc_sink sink;
  memset(&sink, 0, sizeof sink);
  sink.k = k; sink.cap = cap; sink.w = k;
  for (uint32_t u = 0; u < k; ++u) sink.proj[u] = u;
  sink.room = cap == 0 ? 0 : (cap < (1u << 20) ? 2 * cap : cap + (1u << 20));
  sink.rows = cap ? (uint32_t *)malloc(sizeof(uint32_t) * k * sink.room) : NULL;
  orc_cbt c;
  memset(&c, 0, sizeof c);
  c.g = g; c.w = w; c.q = &q; c.sets = sets; c.sink = &sink;
  c.used = (uint8_t *)calloc(g->V ? g->V : 1, 1);
  orc_hom(&c, 0);
  free(c.used); free(sets);
  if (cap) orc_sink_trim(&sink);
  *count = sink.count; *fp = sink.fp; *nrows = sink.n; *homs = c.homs;
  if (cap && rows_out) memcpy(rows_out, sink.rows, sizeof(uint32_t) * k * sink.n);
  free(sink.rows);
  return 0;
}
