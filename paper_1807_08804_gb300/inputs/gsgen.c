/*
 * Seeded synthetic inputs for labeled subgraph matching: data graphs, query
 * graphs and query arrival times.  This file holds no matching arithmetic;
 * both the CUDA engine and the CPU oracle consume what it produces.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both written here from their
 * published definitions.
 *
 * Shapes follow the workloads the thesis evaluates on (Ch. 3, Section
 * "Performance Evaluation"): large directed graphs with relation-labelled
 * edges and typed vertices, and small query graphs grown from a seed vertex
 * so that they are not only trees.  The distributions themselves (power-law
 * out-degree, Zipf types and relations, uniform targets) are this project's
 * stand-ins for the thesis's datasets, which are not available.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ PRNG */
typedef struct { uint64_t s[4]; } gsg_rng;

static uint64_t gsg_splitmix64(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static uint64_t gsg_rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static void gsg_seed(gsg_rng *r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = gsg_splitmix64(&x);
}
static uint64_t gsg_next(gsg_rng *r) {
  uint64_t *s = r->s;
  uint64_t res = gsg_rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = gsg_rotl(s[3], 45);
  return res;
}
/* uniform double in [0,1) with 53 random bits */
static double gsg_unif(gsg_rng *r) { return (double)(gsg_next(r) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0,n) by Lemire's multiply-shift with rejection */
static uint64_t gsg_below(gsg_rng *r, uint64_t n) {
  if (n <= 1) return 0;
  for (;;) {
    uint64_t x = gsg_next(r);
    __uint128_t m = (__uint128_t)x * n;
    uint64_t lo = (uint64_t)m;
    if (lo >= n) return (uint64_t)(m >> 64);
    uint64_t thr = (0 - n) % n;
    if (lo >= thr) return (uint64_t)(m >> 64);
  }
}

/* Stream ids keep graph, queries and arrivals independent for one seed. */
static void gsg_stream(gsg_rng *r, uint64_t seed, uint64_t stream) {
  gsg_seed(r, seed ^ (0xA0761D6478BD642Full * (stream + 1)));
}

/* ---------------------------------------------------------- Zipf tables */
/* P(i) proportional to 1/(i+1)^s over n labels; sampled by CDF search. */
static double *gsg_zipf_cdf(uint32_t n, double s) {
  double *c = (double *)malloc(sizeof(double) * n);
  double acc = 0;
  for (uint32_t i = 0; i < n; ++i) { acc += pow((double)(i + 1), -s); c[i] = acc; }
  for (uint32_t i = 0; i < n; ++i) c[i] /= acc;
  c[n - 1] = 1.0;
  return c;
}
static uint32_t gsg_zipf(gsg_rng *r, const double *cdf, uint32_t n) {
  double u = gsg_unif(r);
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) { uint32_t mid = (lo + hi) / 2; if (cdf[mid] > u) hi = mid; else lo = mid + 1; }
  return lo;
}

/* ------------------------------------------------------------ the graph */
static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : x > y;
}

/*
 * Out-degrees: x_i i.i.d. continuous Pareto with density exponent alpha
 * (x >= 1), d_i = clamp(round(c * x_i), 1, dmax), with c found by bisection so
 * that sum d_i is as close to E as the rounding allows; the remainder is
 * settled by +-1 steps on random vertices that stay inside [1, dmax].
 * Returns 0 on success, -1 if E cannot be reached.
 */
static int gsg_degrees(gsg_rng *r, uint32_t V, uint64_t E, double alpha, uint32_t dmax,
                       uint32_t *deg) {
  if ((uint64_t)V > E || (uint64_t)V * dmax < E) return -1;
  double *x = (double *)malloc(sizeof(double) * V);
  for (uint32_t i = 0; i < V; ++i) x[i] = pow(1.0 - gsg_unif(r), -1.0 / (alpha - 1.0));
  double lo = 0.0, hi = (double)dmax;
  for (int it = 0; it < 200; ++it) {
    double c = 0.5 * (lo + hi);
    uint64_t s = 0;
    for (uint32_t i = 0; i < V; ++i) {
      double d = floor(c * x[i] + 0.5);
      s += d < 1 ? 1 : (d > dmax ? dmax : (uint64_t)d);
    }
    if (s < E) lo = c; else hi = c;
  }
  uint64_t s = 0;
  for (uint32_t i = 0; i < V; ++i) {
    double d = floor(hi * x[i] + 0.5);
    deg[i] = d < 1 ? 1 : (d > dmax ? dmax : (uint32_t)d);
    s += deg[i];
  }
  free(x);
  while (s != E) {
    uint32_t v = (uint32_t)gsg_below(r, V);
    if (s > E && deg[v] > 1) { deg[v]--; s--; }
    else if (s < E && deg[v] < dmax) { deg[v]++; s++; }
  }
  return 0;
}

/*
 * gsg_graph: V vertices, E directed edges.  Outputs an out-CSR in draw order
 * (not sorted, so that consumers canonicalise it themselves):
 *   row_off[V+1] (uint64), col[E] (uint32), rel[E] (uint32), vtype[V] (uint32).
 * Types ~ Zipf(type_s) over T labels, relations ~ Zipf(rel_s) over R labels,
 * targets uniform over V \ {src} (target_s = 0) or, with target_s > 0,
 * Zipf(target_s) over the vertices in a seeded random order, a vertex taking
 * at most dmax incoming edges (popular concepts take most incoming edges);
 * with copy_p > 0 a vertex copies, with
 * that probability, the whole out-list (relations and targets) of the last
 * earlier vertex of its type and out-degree, so families of concepts share
 * their adjacency as in commonsense graphs (a copied target equal to the
 * vertex itself is redrawn); duplicate (src, rel, dst) triples are redrawn.
 * Returns 0 or -1 (parameters impossible).
 */
static uint32_t gsg_target(gsg_rng *r, uint32_t V, uint32_t v, const double *tcdf, const uint32_t *perm,
                           const uint32_t *indeg, uint32_t dmax) {
  if (!tcdf) {
    uint32_t t = (uint32_t)gsg_below(r, V - 1);
    return t >= v ? t + 1 : t;
  }
  for (;;) {  /* popular targets fill up to dmax incoming edges, like out-degrees */
    const uint32_t t = perm[gsg_zipf(r, tcdf, V)];
    if (t != v && indeg[t] < dmax) return t;
  }
}

int gsg_graph(uint32_t V, uint64_t E, uint32_t T, double type_s, uint32_t R, double rel_s,
              double alpha, uint32_t dmax, uint64_t seed,
              uint64_t *row_off, uint32_t *col, uint32_t *rel, uint32_t *vtype, double target_s,
              double copy_p) {
  if (V < 2 || T == 0 || R == 0) return -1;
  uint64_t cap = (uint64_t)R * (V - 1);
  if (dmax > cap) dmax = (uint32_t)cap;
  gsg_rng rt, rd, re;
  gsg_stream(&rt, seed, 1);
  gsg_stream(&rd, seed, 2);
  gsg_stream(&re, seed, 3);
  double *tc = gsg_zipf_cdf(T, type_s), *rc = gsg_zipf_cdf(R, rel_s);
  for (uint32_t v = 0; v < V; ++v) vtype[v] = gsg_zipf(&rt, tc, T);
  double *tcdf = NULL;
  uint32_t *perm = NULL, *indeg = NULL;
  if (target_s > 0) {  /* popularity order: a seeded Fisher-Yates shuffle */
    gsg_rng rp;
    gsg_stream(&rp, seed, 4);
    tcdf = gsg_zipf_cdf(V, target_s);
    indeg = (uint32_t *)calloc(V, sizeof(uint32_t));
    perm = (uint32_t *)malloc(sizeof(uint32_t) * V);
    for (uint32_t v = 0; v < V; ++v) perm[v] = v;
    for (uint32_t v = V - 1; v > 0; --v) {
      const uint32_t j = (uint32_t)gsg_below(&rp, (uint64_t)v + 1);
      const uint32_t t = perm[v]; perm[v] = perm[j]; perm[j] = t;
    }
  }
  uint32_t *deg = (uint32_t *)malloc(sizeof(uint32_t) * V);
  if (gsg_degrees(&rd, V, E, alpha, dmax, deg) != 0) { free(deg); free(tc); free(rc); return -1; }
  row_off[0] = 0;
  for (uint32_t v = 0; v < V; ++v) row_off[v + 1] = row_off[v] + deg[v];
  uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (dmax + 1));
  uint64_t *srt = (uint64_t *)malloc(sizeof(uint64_t) * (dmax + 1));
  /* copy model: last vertex of each (type, out-degree), -1 if none yet */
  int64_t *last = NULL;
  gsg_rng rcp;
  if (copy_p > 0) {
    gsg_stream(&rcp, seed, 5);
    last = (int64_t *)malloc(sizeof(int64_t) * (uint64_t)T * (dmax + 1));
    for (uint64_t i = 0; i < (uint64_t)T * (dmax + 1); ++i) last[i] = -1;
  }
  for (uint32_t v = 0; v < V; ++v) {
    uint32_t d = deg[v];
    /* key = rel << 32 | dst; redraw duplicates until the list is distinct */
    int64_t proto = -1;
    if (last) {
      int64_t *slot = &last[(uint64_t)vtype[v] * (dmax + 1) + d];
      if (*slot >= 0 && gsg_unif(&rcp) < copy_p) proto = *slot;
      *slot = v;
    }
    for (uint32_t j = 0; j < d; ++j) {
      if (proto >= 0) {
        const uint64_t o = row_off[proto] + j;
        key[j] = ((uint64_t)rel[o] << 32) | col[o];
        if (col[o] != v && (!indeg || indeg[col[o]] < dmax)) continue;
      }
      uint32_t t = gsg_target(&re, V, v, tcdf, perm, indeg, dmax);
      key[j] = ((uint64_t)gsg_zipf(&re, rc, R) << 32) | t;
    }
    for (;;) {
      memcpy(srt, key, sizeof(uint64_t) * d);
      qsort(srt, d, sizeof(uint64_t), cmp_u64);
      int dup = 0;
      for (uint32_t j = 1; j < d; ++j) if (srt[j] == srt[j - 1]) { dup = 1; break; }
      if (!dup) break;
      /* redraw every later occurrence of a repeated key, in draw order */
      for (uint32_t j = 0; j < d; ++j) {
        int seen = 0;
        for (uint32_t i = 0; i < j; ++i) if (key[i] == key[j]) { seen = 1; break; }
        if (seen) {
          uint32_t t = gsg_target(&re, V, v, tcdf, perm, indeg, dmax);
          key[j] = ((uint64_t)gsg_zipf(&re, rc, R) << 32) | t;
        }
      }
    }
    uint64_t o = row_off[v];
    for (uint32_t j = 0; j < d; ++j) { col[o + j] = (uint32_t)key[j]; rel[o + j] = (uint32_t)(key[j] >> 32); }
    if (indeg)
      for (uint32_t j = 0; j < d; ++j) indeg[(uint32_t)key[j]]++;
  }
  free(key); free(srt); free(deg); free(tc); free(rc); free(tcdf); free(perm); free(last); free(indeg);
  return 0;
}

/* ------------------------------------------------------------- queries */
/*
 * Incoming CSR built by counting sort, for walks over the undirected view.
 */
typedef struct {
  uint32_t V; const uint64_t *ro; const uint32_t *col, *rel;
  uint64_t *ri; uint32_t *icol, *irel;
} gsg_view;

static void gsg_view_build(gsg_view *g, uint32_t V, const uint64_t *ro, const uint32_t *col,
                           const uint32_t *rel) {
  g->V = V; g->ro = ro; g->col = col; g->rel = rel;
  uint64_t E = ro[V];
  g->ri = (uint64_t *)calloc(V + 1, sizeof(uint64_t));
  g->icol = (uint32_t *)malloc(sizeof(uint32_t) * (E ? E : 1));
  g->irel = (uint32_t *)malloc(sizeof(uint32_t) * (E ? E : 1));
  for (uint64_t e = 0; e < E; ++e) g->ri[col[e] + 1]++;
  for (uint32_t v = 0; v < V; ++v) g->ri[v + 1] += g->ri[v];
  uint64_t *pos = (uint64_t *)malloc(sizeof(uint64_t) * (V + 1));
  memcpy(pos, g->ri, sizeof(uint64_t) * (V + 1));
  for (uint32_t s = 0; s < V; ++s)
    for (uint64_t e = ro[s]; e < ro[s + 1]; ++e) {
      uint64_t p = pos[col[e]]++;
      g->icol[p] = s; g->irel[p] = rel[e];
    }
  free(pos);
}
static void gsg_view_free(gsg_view *g) { free(g->ri); free(g->icol); free(g->irel); }

/* is (a, r, b) a data edge?  (linear scan of a's out-list; lists are short) */
static int gsg_has_edge(const gsg_view *g, uint32_t a, uint32_t r, uint32_t b) {
  for (uint64_t e = g->ro[a]; e < g->ro[a + 1]; ++e)
    if (g->col[e] == b && g->rel[e] == r) return 1;
  return 0;
}

#define GSG_UNBOUND 0xFFFFFFFFu
#define GSG_ANY 0xFFFFFFFFu

/*
 * gsg_walk_queries: n queries grown by seeded random walks over the undirected
 * view of the graph.  Query i has k_i vertices, k_i uniform in [kmin, kmax].
 * Tree edges are the traversed data edges (direction and relation kept);
 * every other data triple among the walked vertices is added with p_close.
 * cyclic_mode: 0 = as above; 1 = even-indexed queries must hold >= 1 closing
 * edge (redraw up to 32 times), odd-indexed ones get none.
 * Each vertex is bound to its walked id with p_bind (type ANY), else typed
 * with its walked vertex's type.  The walked identity map is always a match.
 *
 * Output (flat, caller-allocated with room for n*kmax vertices and
 * n*kmax*(kmax-1)*R edges at most — use gsg_walk_queries_bound for sizes):
 *   qk[n], qm[n], vtype[], vbind[], walked[] (the walked data ids),
 *   esrc[], edst[], erel[] (query-local endpoints).
 * Returns the total number of edges written, or -1.
 */
int64_t gsg_walk_queries(uint32_t V, const uint64_t *ro, const uint32_t *col, const uint32_t *rel,
                         const uint32_t *gtype, uint32_t n, uint32_t kmin, uint32_t kmax,
                         double p_close, double p_bind, int cyclic_mode, uint64_t seed,
                         uint64_t max_edges,
                         uint32_t *qk, uint32_t *qm, uint32_t *vtype, uint32_t *vbind,
                         uint32_t *walked, uint32_t *esrc, uint32_t *edst, uint32_t *erel) {
  if (kmin < 2 || kmax < kmin || kmax > 32 || V < kmax) return -1;
  gsg_view g;
  gsg_view_build(&g, V, ro, col, rel);
  gsg_rng r;
  gsg_stream(&r, seed, 10);
  uint64_t vout = 0, eout = 0;
  uint32_t tsrc[32], tdst[32], trel[32];
  uint32_t cs[4096], cd[4096], cr[4096];
  for (uint32_t q = 0; q < n; ++q) {
    uint32_t k = kmin + (uint32_t)gsg_below(&r, kmax - kmin + 1);
    uint32_t ids[32], nt = 0, nv = 0, nc = 0;
    int want_cycle = cyclic_mode == 1 && (q % 2 == 0);
    int no_close = cyclic_mode == 1 && (q % 2 == 1);
    for (int attempt = 0;; ++attempt) {
      /* the walk */
      for (;;) {
        nv = 0; nt = 0;
        uint32_t cur = (uint32_t)gsg_below(&r, V);
        ids[nv++] = cur;
        uint32_t stall = 0;
        while (nv < k && stall < 64 * k) {
          uint64_t dout = ro[cur + 1] - ro[cur], din = g.ri[cur + 1] - g.ri[cur];
          if (dout + din == 0) break;
          uint64_t pick = gsg_below(&r, dout + din);
          uint32_t nxt, a, b, rr;
          if (pick < dout) { uint64_t e = ro[cur] + pick; nxt = col[e]; a = cur; b = nxt; rr = rel[e]; }
          else { uint64_t e = g.ri[cur] + (pick - dout); nxt = g.icol[e]; a = nxt; b = cur; rr = g.irel[e]; }
          int known = 0;
          for (uint32_t i = 0; i < nv; ++i) if (ids[i] == nxt) { known = 1; break; }
          if (!known) {
            ids[nv] = nxt;
            uint32_t ia = 0, ib = 0;
            for (uint32_t i = 0; i <= nv; ++i) { if (ids[i] == a) ia = i; if (ids[i] == b) ib = i; }
            tsrc[nt] = ia; tdst[nt] = ib; trel[nt] = rr; nt++;
            nv++; stall = 0;
          } else stall++;
          cur = nxt;
        }
        if (nv == k) break;
      }
      /* closing edges: every other triple among the walked vertices */
      nc = 0;
      if (!no_close) {
        for (uint32_t i = 0; i < k; ++i)
          for (uint64_t e = ro[ids[i]]; e < ro[ids[i] + 1]; ++e) {
            uint32_t j = 0; int in = 0;
            for (j = 0; j < k; ++j) if (ids[j] == col[e]) { in = 1; break; }
            if (!in) continue;
            int is_tree = 0;
            for (uint32_t t = 0; t < nt; ++t)
              if (tsrc[t] == i && tdst[t] == j && trel[t] == rel[e]) { is_tree = 1; break; }
            if (is_tree) continue;
            if (gsg_unif(&r) < p_close && nc < 4096) { cs[nc] = i; cd[nc] = j; cr[nc] = rel[e]; nc++; }
          }
      }
      if (!want_cycle || nc > 0 || attempt >= 31) break;
    }
    if (eout + nt + nc > max_edges) { gsg_view_free(&g); return -1; }
    qk[q] = k; qm[q] = nt + nc;
    for (uint32_t i = 0; i < k; ++i) {
      walked[vout + i] = ids[i];
      if (gsg_unif(&r) < p_bind) { vbind[vout + i] = ids[i]; vtype[vout + i] = GSG_ANY; }
      else { vbind[vout + i] = GSG_UNBOUND; vtype[vout + i] = gtype[ids[i]]; }
    }
    for (uint32_t t = 0; t < nt; ++t) { esrc[eout] = tsrc[t]; edst[eout] = tdst[t]; erel[eout] = trel[t]; eout++; }
    for (uint32_t t = 0; t < nc; ++t) { esrc[eout] = cs[t]; edst[eout] = cd[t]; erel[eout] = cr[t]; eout++; }
    vout += k;
  }
  gsg_view_free(&g);
  (void)gsg_has_edge;
  return (int64_t)eout;
}

/*
 * gsg_shape_queries: n unbound typed queries of fixed shapes, in equal shares
 * and in this order of shapes: directed 4-cycle, directed 5-cycle, 4-clique
 * (edge i->j for i<j), 6-vertex random tree (random parent, random direction).
 * Edge relations are drawn uniformly from rels[0..nr), vertex types from
 * types[0..nt).  Output as gsg_walk_queries (vbind all unbound).
 * Returns the number of edges written.
 */
int64_t gsg_shape_queries(uint32_t n, const uint32_t *rels, uint32_t nr, const uint32_t *types,
                          uint32_t nt, uint64_t seed,
                          uint32_t *qk, uint32_t *qm, uint32_t *vtype, uint32_t *vbind,
                          uint32_t *esrc, uint32_t *edst, uint32_t *erel) {
  gsg_rng r;
  gsg_stream(&r, seed, 20);
  uint64_t vout = 0, eout = 0;
  for (uint32_t q = 0; q < n; ++q) {
    uint32_t shape = (uint32_t)((uint64_t)q * 4 / (n ? n : 1));
    uint32_t k = 0, m = 0, s[16], d[16];
    if (shape == 0 || shape == 1) {
      k = shape == 0 ? 4 : 5;
      for (uint32_t i = 0; i < k; ++i) { s[m] = i; d[m] = (i + 1) % k; m++; }
    } else if (shape == 2) {
      k = 4;
      for (uint32_t i = 0; i < k; ++i) for (uint32_t j = i + 1; j < k; ++j) { s[m] = i; d[m] = j; m++; }
    } else {
      k = 6;
      for (uint32_t i = 1; i < k; ++i) {
        uint32_t p = (uint32_t)gsg_below(&r, i);
        if (gsg_below(&r, 2)) { s[m] = p; d[m] = i; } else { s[m] = i; d[m] = p; }
        m++;
      }
    }
    qk[q] = k; qm[q] = m;
    for (uint32_t i = 0; i < k; ++i) {
      vbind[vout + i] = GSG_UNBOUND;
      vtype[vout + i] = types[gsg_below(&r, nt)];
    }
    for (uint32_t j = 0; j < m; ++j) {
      esrc[eout + j] = s[j]; edst[eout + j] = d[j]; erel[eout + j] = rels[gsg_below(&r, nr)];
    }
    vout += k; eout += m;
  }
  return (int64_t)eout;
}

/* gsg_arrivals: n Poisson arrival times (seconds) at rate qps, starting at 0. */
void gsg_arrivals(uint32_t n, double qps, uint64_t seed, double *t) {
  gsg_rng r;
  gsg_stream(&r, seed, 30);
  double now = 0;
  for (uint32_t i = 0; i < n; ++i) { now += -log(1.0 - gsg_unif(&r)) / qps; t[i] = now; }
}
