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
