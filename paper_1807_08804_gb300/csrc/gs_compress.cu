// Multi-level graph compression (Section 3.4) and matching through the
// compressed graph (Section 3.5).
//
// Offline, on the host (the thesis compresses offline on the CPU): levels of
// pairwise merges of similar nodes build a weighted graph G_w whose nodes
// stand for groups of data vertices (mapping lists).  Online, on the device:
//   1. the queries, with each binding replaced by the node holding it, run
//      the filtering phase on G_w with Definition 3.5's candidate test (the
//      weights are loaded as G_w's degree signatures) and exploration and
//      refinement to the fixpoint;
//   2. the full pipeline runs on the data graph with every candidate test
//      also requiring that the vertex's node is a G_w candidate of the same
//      query vertex (Theorem 3.2: no other vertex can match), which is the
//      expansion of the G_w sets through the mapping lists.
// The result is every embedding of the query in the data graph, exactly as
// without compression.
//
// Definitions, read for directed graphs with relation labels and vertex
// types:
//   - adjacency of a node x of a level: the (direction, relation, other node)
//     triples of its edges to other nodes; common(x, y) = the triples both
//     have; x, y are similar when they have one type and |common| >= delta *
//     |adj| for both (double-precision products), or both have no edges;
//   - a level visits nodes in index order and pairs each unpaired node with
//     the lowest-indexed later unpaired node similar to it; the merged nodes
//     are numbered by ascending smallest member;
//   - edge weights start at 1 and follow the thesis's recursion
//     w(u, v) = max(w(p, n), w(q, n)) + max(w(p, m), w(q, m)) per relation,
//     wout over the parts of the target node, win over the parts of the
//     source node; edges inside a node are not edges of G_w;
//   - node weight per direction and relation: the most neighbours a member
//     has inside its own node, counted in the data graph;
//   - Definition 3.5 per direction and relation: a query vertex with c
//     neighbours there needs node weight + edge weights >= c (the plane of
//     variable edges sums every relation).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "gs_host.h"

using namespace gs;

namespace {

struct WEdge {
  uint32_t src, rel, dst, wout, win;
};

// A compressed graph held on the host: mapping lists and weights.
struct Compression {
  uint32_t V = 0, R = 0, n = 0;
  std::vector<uint32_t> group;   // [V] node holding each data vertex
  std::vector<uint32_t> moff;    // [n+1]
  std::vector<uint32_t> mem;     // [V] members of each node, ascending
  std::vector<uint32_t> type;    // [n]
  std::vector<WEdge> edges;      // between different nodes, by (src, rel, dst)
  std::vector<uint32_t> wnode;   // [(dir * R + rel) * n + x]
};

// (direction, relation, other node) packed so that sorting orders by all three.
inline uint64_t adj_key(uint32_t dir, uint32_t rel, uint32_t other) {
  return ((uint64_t)dir << 32) | ((uint64_t)rel << 24) | other;
}

// One level of pairing.  Returns the node count of the next level and
// fills next[x] for every node x of this level.
uint32_t pair_nodes(uint32_t n, const std::vector<uint32_t> &type, const std::vector<WEdge> &edges, double delta,
                    std::vector<uint32_t> &next) {
  // adjacency of every node as a sorted key list
  std::vector<std::pair<uint32_t, uint64_t>> ends;
  ends.reserve(2 * edges.size());
  for (const WEdge &e : edges) {
    ends.emplace_back(e.src, adj_key(0, e.rel, e.dst));
    ends.emplace_back(e.dst, adj_key(1, e.rel, e.src));
  }
  std::sort(ends.begin(), ends.end());
  std::vector<uint64_t> aoff(n + 1, 0), keys(ends.size());
  for (size_t i = 0; i < ends.size(); ++i) {
    aoff[ends[i].first + 1]++;
    keys[i] = ends[i].second;
  }
  for (uint32_t x = 0; x < n; ++x) aoff[x + 1] += aoff[x];
  // Candidates by prefix filtering (the exact filter of all-pairs set
  // similarity joins): order keys by how many nodes hold them (fewest
  // first); node x's prefix is its first a - cmin(a) + 1 keys in that order,
  // cmin(a) = the least overlap its side of the test accepts.  Two similar
  // nodes share at least max(cmin(a), cmin(b)) keys, so their prefixes
  // meet: only nodes holding one of x's prefix keys in their own prefix are
  // tried, in ascending index order, and the first similar one is x's mate.
  // held[i] = how many nodes hold keys[i] (positions grouped by key)
  std::vector<uint64_t> held(keys.size());
  {
    std::vector<uint64_t> at(keys.size());
    for (uint64_t i = 0; i < at.size(); ++i) at[i] = i;
    std::sort(at.begin(), at.end(), [&](uint64_t p, uint64_t q) { return keys[p] < keys[q]; });
    for (uint64_t i = 0; i < at.size();) {
      uint64_t j = i;
      while (j < at.size() && keys[at[j]] == keys[at[i]]) ++j;
      for (uint64_t t = i; t < j; ++t) held[at[t]] = j - i;
      i = j;
    }
  }
  auto cmin_of = [&](uint64_t a) {
    uint64_t c = 0;
    while (!((double)c >= delta * (double)a)) ++c;
    return c;
  };
  std::vector<std::pair<uint64_t, uint32_t>> pre;  // (key, node) over every node's prefix keys
  std::vector<std::pair<uint64_t, uint64_t>> order;
  std::vector<uint64_t> poff(n + 1, 0);
  std::vector<uint64_t> pkeys;
  for (uint32_t x = 0; x < n; ++x) {
    const uint64_t a = aoff[x + 1] - aoff[x];
    order.clear();
    for (uint64_t i = aoff[x]; i < aoff[x + 1]; ++i) order.emplace_back(held[i], keys[i]);
    std::sort(order.begin(), order.end());
    const uint64_t plen = a ? a - cmin_of(a) + 1 : 0;
    for (uint64_t j = 0; j < plen; ++j) {
      pre.emplace_back(order[j].second, x);
      pkeys.push_back(order[j].second);
    }
    poff[x + 1] = pkeys.size();
  }
  std::sort(pre.begin(), pre.end());
  // nodes without edges, per type (similar only to each other)
  uint32_t T = 0;
  for (uint32_t t : type) T = std::max(T, t + 1);
  std::vector<std::vector<uint32_t>> bare(T);
  for (uint32_t x = 0; x < n; ++x)
    if (aoff[x + 1] == aoff[x]) bare[type[x]].push_back(x);
  std::vector<size_t> bare_at(T, 0);

  // classes of nodes with one type and equal adjacency lists, each in
  // ascending index order: when the test admits only equal lists (every key
  // of x shared, and one key more already too many for x's side), x's mate
  // is the next unpaired node of its class
  std::vector<uint32_t> by_adj(n);
  for (uint32_t x = 0; x < n; ++x) by_adj[x] = x;
  auto adj_less = [&](uint32_t x, uint32_t y) {
    if (type[x] != type[y]) return type[x] < type[y];
    const uint64_t a = aoff[x + 1] - aoff[x], b = aoff[y + 1] - aoff[y];
    if (a != b) return a < b;
    for (uint64_t i = 0; i < a; ++i)
      if (keys[aoff[x] + i] != keys[aoff[y] + i]) return keys[aoff[x] + i] < keys[aoff[y] + i];
    return x < y;
  };
  std::sort(by_adj.begin(), by_adj.end(), adj_less);
  auto same_adj = [&](uint32_t x, uint32_t y) {
    const uint64_t a = aoff[x + 1] - aoff[x];
    return type[x] == type[y] && a == aoff[y + 1] - aoff[y] &&
           std::equal(keys.begin() + aoff[x], keys.begin() + aoff[x + 1], keys.begin() + aoff[y]);
  };
  std::vector<uint32_t> cls_pos(n);   // position of each node in by_adj
  std::vector<uint32_t> cls_end(n);   // end of its class in by_adj
  for (uint32_t i = 0; i < n; ++i) cls_pos[by_adj[i]] = i;
  for (uint32_t i = n; i-- > 0;)
    cls_end[by_adj[i]] = (i + 1 < n && same_adj(by_adj[i], by_adj[i + 1])) ? cls_end[by_adj[i + 1]] : i + 1;

  std::vector<int64_t> mate(n, -1);
  std::vector<uint32_t> cand;
  for (uint32_t x = 0; x < n; ++x) {
    if (mate[x] >= 0) continue;
    const uint64_t a = aoff[x + 1] - aoff[x];
    if (a > 0 && cmin_of(a) == a && !((double)a >= delta * (double)(a + 1))) {
      for (uint32_t i = cls_pos[x] + 1; i < cls_end[x]; ++i) {  // later members of x's class, ascending
        const uint32_t y = by_adj[i];
        if (mate[y] < 0) {
          mate[x] = y;
          mate[y] = x;
          break;
        }
      }
      continue;
    }
    if (a == 0) {
      auto &L = bare[type[x]];
      size_t &c = bare_at[type[x]];
      while (c < L.size() && (L[c] <= x || mate[L[c]] >= 0)) ++c;
      if (c < L.size()) {
        mate[x] = L[c];
        mate[L[c]] = x;
      }
      continue;
    }
    cand.clear();
    for (uint64_t j = poff[x]; j < poff[x + 1]; ++j) {
      auto lo = std::upper_bound(pre.begin(), pre.end(), std::make_pair(pkeys[j], x));
      for (auto h = lo; h != pre.end() && h->first == pkeys[j]; ++h) {
        const uint32_t y = h->second;
        if (mate[y] < 0 && type[y] == type[x]) cand.push_back(y);
      }
    }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (uint32_t y : cand) {
      const uint64_t b = aoff[y + 1] - aoff[y];
      uint64_t c = 0;
      for (uint64_t i = aoff[x], j = aoff[y]; i < aoff[x + 1] && j < aoff[y + 1];) {
        if (keys[i] == keys[j]) { ++c; ++i; ++j; }
        else if (keys[i] < keys[j]) ++i;
        else ++j;
      }
      if ((double)c >= delta * (double)a && (double)c >= delta * (double)b) {
        mate[x] = y;
        mate[y] = x;
        break;
      }
    }
  }
  next.assign(n, 0);
  uint32_t cnt = 0;
  for (uint32_t x = 0; x < n; ++x) {
    if (mate[x] >= 0 && (uint32_t)mate[x] < x) continue;
    next[x] = cnt;
    if (mate[x] >= 0) next[mate[x]] = cnt;
    ++cnt;
  }
  return cnt;
}

// Edges of the next level with the weight recursion.
std::vector<WEdge> merge_edges(const std::vector<WEdge> &edges, const std::vector<uint32_t> &next) {
  struct Part { uint32_t u, rel, v, from, to, wout, win; };
  std::vector<Part> parts;
  parts.reserve(edges.size());
  for (const WEdge &e : edges) {
    const uint32_t u = next[e.src], v = next[e.dst];
    if (u != v) parts.push_back({u, e.rel, v, e.src, e.dst, e.wout, e.win});
  }
  auto same_edge = [](const Part &a, const Part &b) { return a.u == b.u && a.rel == b.rel && a.v == b.v; };
  std::vector<WEdge> out;
  // wout: for each part `to` of the target, the heaviest part of the source
  std::sort(parts.begin(), parts.end(), [](const Part &a, const Part &b) {
    return std::tie(a.u, a.rel, a.v, a.to) < std::tie(b.u, b.rel, b.v, b.to);
  });
  for (size_t i = 0; i < parts.size();) {
    WEdge w{parts[i].u, parts[i].rel, parts[i].v, 0, 0};
    size_t j = i;
    while (j < parts.size() && same_edge(parts[j], parts[i])) {
      uint32_t best = 0;
      const uint32_t to = parts[j].to;
      for (; j < parts.size() && same_edge(parts[j], parts[i]) && parts[j].to == to; ++j)
        best = std::max(best, parts[j].wout);
      w.wout += best;
    }
    out.push_back(w);
    i = j;
  }
  // win: for each part `from` of the source, the heaviest part of the target
  std::sort(parts.begin(), parts.end(), [](const Part &a, const Part &b) {
    return std::tie(a.u, a.rel, a.v, a.from) < std::tie(b.u, b.rel, b.v, b.from);
  });
  size_t k = 0;
  for (size_t i = 0; i < parts.size(); ++k) {
    size_t j = i;
    while (j < parts.size() && same_edge(parts[j], parts[i])) {
      uint32_t best = 0;
      const uint32_t from = parts[j].from;
      for (; j < parts.size() && same_edge(parts[j], parts[i]) && parts[j].from == from; ++j)
        best = std::max(best, parts[j].win);
      out[k].win += best;
    }
    i = j;
  }
  return out;
}

// The compression of a host out-CSR.
Compression compress(const gs_graph_desc &d, uint32_t levels, const double *delta) {
  Compression c;
  c.V = d.num_vertices;
  c.R = d.num_rels;
  const uint32_t V = c.V, R = c.R;
  // distinct data triples (src << 32 | rel << 24 | dst)
  std::vector<uint64_t> tri;
  tri.reserve(d.num_edges);
  for (uint32_t s = 0; s < V; ++s)
    for (uint64_t e = d.row_offsets[s]; e < d.row_offsets[s + 1]; ++e)
      tri.push_back(((uint64_t)s << 32) | ((uint64_t)d.edge_rel[e] << 24) | d.col_targets[e]);
  std::sort(tri.begin(), tri.end());
  tri.erase(std::unique(tri.begin(), tri.end()), tri.end());
  auto t_src = [](uint64_t t) { return (uint32_t)(t >> 32); };
  auto t_rel = [](uint64_t t) { return (uint32_t)((t >> 24) & 0xFFu); };
  auto t_dst = [](uint64_t t) { return (uint32_t)(t & kNbrMask); };

  uint32_t n = V;
  std::vector<uint32_t> type(d.vertex_type, d.vertex_type + V), group(V);
  for (uint32_t v = 0; v < V; ++v) group[v] = v;
  std::vector<WEdge> edges;
  edges.reserve(tri.size());
  for (uint64_t t : tri)
    if (t_src(t) != t_dst(t)) edges.push_back({t_src(t), t_rel(t), t_dst(t), 1, 1});
  std::vector<uint32_t> next;
  for (uint32_t l = 0; l < levels; ++l) {
    const uint32_t n2 = pair_nodes(n, type, edges, delta[l], next);
    edges = merge_edges(edges, next);
    std::vector<uint32_t> type2(n2);
    for (uint32_t x = 0; x < n; ++x) type2[next[x]] = type[x];
    for (uint32_t &g : group) g = next[g];
    type.swap(type2);
    n = n2;
  }
  std::sort(edges.begin(), edges.end(), [](const WEdge &a, const WEdge &b) {
    return std::tie(a.src, a.rel, a.dst) < std::tie(b.src, b.rel, b.dst);
  });
  c.n = n;
  c.group = group;
  c.type = type;
  c.edges = std::move(edges);
  c.moff.assign(n + 1, 0);
  for (uint32_t v = 0; v < V; ++v) c.moff[group[v] + 1]++;
  for (uint32_t x = 0; x < n; ++x) c.moff[x + 1] += c.moff[x];
  c.mem.resize(V);
  std::vector<uint32_t> at(c.moff.begin(), c.moff.end() - 1);
  for (uint32_t v = 0; v < V; ++v) c.mem[at[group[v]]++] = v;
  // node weights: per member and relation, its neighbours inside its node
  c.wnode.assign((uint64_t)2 * R * n, 0);
  auto bump = [&](uint32_t dir, uint32_t r, uint32_t x, uint32_t cnt) {
    uint32_t &w = c.wnode[((uint64_t)dir * R + r) * n + x];
    w = std::max(w, cnt);
  };
  for (size_t i = 0; i < tri.size();) {  // out: runs of one (src, rel)
    size_t j = i;
    uint32_t cnt = 0;
    for (; j < tri.size() && (tri[j] >> 24) == (tri[i] >> 24); ++j) cnt += group[t_dst(tri[j])] == group[t_src(tri[i])];
    bump(0, t_rel(tri[i]), group[t_src(tri[i])], cnt);
    i = j;
  }
  std::vector<uint64_t> rev(tri.size());  // (dst, rel, src)
  for (size_t i = 0; i < tri.size(); ++i)
    rev[i] = ((uint64_t)t_dst(tri[i]) << 32) | ((uint64_t)t_rel(tri[i]) << 24) | t_src(tri[i]);
  std::sort(rev.begin(), rev.end());
  for (size_t i = 0; i < rev.size();) {  // in: runs of one (dst, rel)
    size_t j = i;
    uint32_t cnt = 0;
    for (; j < rev.size() && (rev[j] >> 24) == (rev[i] >> 24); ++j) cnt += group[t_dst(rev[j])] == group[t_src(rev[i])];
    bump(1, t_rel(rev[i]), group[t_src(rev[i])], cnt);
    i = j;
  }
  return c;
}

}  // namespace

struct gs_cgraph {
  gs_graph *g = nullptr;    // the data graph (device)
  gs_graph *gw = nullptr;   // the weighted graph (device, weights as degree signatures)
  uint32_t *d_group = nullptr;
  Compression c;
  uint32_t levels = 0;
  uint64_t E = 0;           // distinct data triples
  uint64_t inner = 0;       // (node, relation) pairs with edges inside the node
  cudaStream_t stream = nullptr;
  gs_batch *wb = nullptr;   // weighted-graph stage
  gs_batch *gb = nullptr;   // data-graph stage
  std::mutex mu;
};

namespace {

void cgraph_release(gs_cgraph *cg) {
  if (cg->wb) batch_destroy(cg->wb);
  if (cg->gb) batch_destroy(cg->gb);
  if (cg->d_group) cudaFree(cg->d_group);
  if (cg->gw) gs_graph_free(cg->gw);
  if (cg->g) gs_graph_free(cg->g);
  if (cg->stream) cudaStreamDestroy(cg->stream);
  delete cg;
}

// The weighted graph as a data graph for the device pipeline: its edges,
// plus an edge (x, r, x) where relation-r edges lie inside x, and its
// Definition 3.5 weights as the degree signatures.
gs_status load_weighted(gs_cgraph *cg, uint32_t T) {
  const Compression &c = cg->c;
  const uint32_t n = c.n, R = c.R;
  std::vector<std::vector<std::pair<uint32_t, uint32_t>>> rows(n);  // (rel, dst)
  for (const WEdge &e : c.edges) rows[e.src].emplace_back(e.rel, e.dst);
  cg->inner = 0;
  for (uint32_t r = 0; r < R; ++r)
    for (uint32_t x = 0; x < n; ++x)
      if (c.wnode[(uint64_t)r * n + x]) {
        rows[x].emplace_back(r, x);
        cg->inner++;
      }
  std::vector<uint64_t> ro(n + 1, 0);
  std::vector<uint32_t> col, rel;
  for (uint32_t x = 0; x < n; ++x) {
    ro[x + 1] = ro[x] + rows[x].size();
    for (auto &p : rows[x]) {
      rel.push_back(p.first);
      col.push_back(p.second);
    }
  }
  gs_graph_desc wd;
  memset(&wd, 0, sizeof(wd));
  wd.num_vertices = n;
  wd.num_edges = ro[n];
  wd.row_offsets = ro.data();
  wd.col_targets = col.data();
  wd.edge_rel = rel.data();
  wd.vertex_type = c.type.data();
  wd.num_types = T;
  wd.num_rels = R;
  gs_status st = gs_graph_load(&wd, &cg->gw);
  if (st != GS_OK) return st;
  // Definition 3.5 per plane: node weight + weights of the node's edges
  const uint64_t P = 2ull * R + 2;
  std::vector<uint64_t> bound(P * n, 0);
  for (uint32_t dir = 0; dir < 2; ++dir)
    for (uint32_t r = 0; r < R; ++r)
      for (uint32_t x = 0; x < n; ++x) bound[((uint64_t)dir * R + r) * n + x] = c.wnode[((uint64_t)dir * R + r) * n + x];
  for (const WEdge &e : c.edges) {
    bound[(uint64_t)e.rel * n + e.src] += e.wout;
    bound[((uint64_t)R + e.rel) * n + e.dst] += e.win;
  }
  for (uint32_t dir = 0; dir < 2; ++dir)
    for (uint32_t r = 0; r < R; ++r)
      for (uint32_t x = 0; x < n; ++x) bound[(2ull * R + dir) * n + x] += bound[((uint64_t)dir * R + r) * n + x];
  std::vector<uint8_t> cnt(P * n);
  for (uint64_t i = 0; i < P * n; ++i) cnt[i] = (uint8_t)std::min<uint64_t>(bound[i], 255);
  return graph_set_signatures(cg->gw, cnt.data());
}

// Queries for the weighted graph: each binding replaced by the node holding it.
struct WQueries {
  std::vector<uint32_t> vbind;
  std::vector<gs_query> qs;
};
void weighted_queries(const gs_cgraph *cg, const gs_query *qs, uint32_t n, WQueries *w) {
  uint64_t nv = 0;
  for (uint32_t i = 0; i < n; ++i) nv += qs[i].vbind ? qs[i].k : 0;
  w->vbind.resize(nv);
  w->qs.assign(qs, qs + n);
  uint64_t at = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (!qs[i].vbind) continue;
    uint32_t *b = w->vbind.data() + at;
    for (uint32_t u = 0; u < qs[i].k; ++u) {
      const uint32_t x = qs[i].vbind[u];
      b[u] = (x != GS_UNBOUND && x < cg->c.V) ? cg->c.group[x] : x;
    }
    w->qs[i].vbind = b;
    at += qs[i].k;
  }
}

}  // namespace

// Host checks of a host out-CSR and the compression parameters.
static gs_status check_compression_args(const gs_graph_desc *desc, uint32_t levels, const double *delta) {
  if (desc->flags & GS_DEVICE_PTRS)
    return fail(GS_ERR_UNSUPPORTED, "compression runs on the host: pass host arrays");
  if (levels > 32) return fail(GS_ERR_INVALID, "at most 32 compression levels");
  for (uint32_t l = 0; l < levels; ++l)
    if (!(delta[l] > 0.0 && delta[l] <= 1.0)) return fail(GS_ERR_INVALID, "each threshold must be in (0, 1]");
  const uint32_t V = desc->num_vertices;
  if (V == 0 || V > (1u << kNbrBits) || desc->num_types == 0 || desc->num_types > 256 || desc->num_rels == 0 ||
      desc->num_rels > 255 || !desc->row_offsets || !desc->vertex_type ||
      (desc->num_edges && (!desc->col_targets || !desc->edge_rel)))
    return fail(GS_ERR_INVALID, "graph sizes or arrays out of range");
  if (desc->row_offsets[0] != 0 || desc->row_offsets[V] != desc->num_edges)
    return fail(GS_ERR_INVALID, "row_offsets must start at 0 and end at num_edges");
  for (uint32_t v = 0; v < V; ++v)
    if (desc->row_offsets[v + 1] < desc->row_offsets[v] || desc->vertex_type[v] >= desc->num_types)
      return fail(GS_ERR_INVALID, "row_offsets must not decrease; types must be < num_types");
  for (uint64_t e = 0; e < desc->num_edges; ++e)
    if (desc->col_targets[e] >= V || desc->edge_rel[e] >= desc->num_rels)
      return fail(GS_ERR_INVALID, "an edge's target or relation is out of range");
  return GS_OK;
}

extern "C" gs_status gs_compress_host(const gs_graph_desc *desc, uint32_t levels, const double *delta,
                                      uint32_t *nodes, uint64_t *weighted_edges, uint32_t *group, uint32_t *src,
                                      uint32_t *rel, uint32_t *dst, uint32_t *wout, uint32_t *win, uint32_t *wnode) {
  if (!desc || !nodes || !weighted_edges || (levels && !delta)) return fail(GS_ERR_INVALID, "gs_compress_host: null argument");
  gs_status st = check_compression_args(desc, levels, delta);
  if (st != GS_OK) return st;
  const Compression c = compress(*desc, levels, delta);
  *nodes = c.n;
  *weighted_edges = c.edges.size();
  if (group) memcpy(group, c.group.data(), sizeof(uint32_t) * c.V);
  for (size_t i = 0; i < c.edges.size(); ++i) {
    if (src) src[i] = c.edges[i].src;
    if (rel) rel[i] = c.edges[i].rel;
    if (dst) dst[i] = c.edges[i].dst;
    if (wout) wout[i] = c.edges[i].wout;
    if (win) win[i] = c.edges[i].win;
  }
  if (wnode) memcpy(wnode, c.wnode.data(), sizeof(uint32_t) * c.wnode.size());
  return GS_OK;
}

extern "C" gs_status gs_cgraph_build(const gs_graph_desc *desc, uint32_t levels, const double *delta, gs_cgraph **out) {
  if (!desc || !out || (levels && !delta)) return fail(GS_ERR_INVALID, "gs_cgraph_build: null argument");
  *out = nullptr;
  gs_status st = check_compression_args(desc, levels, delta);
  if (st != GS_OK) return st;
  gs_cgraph *cg = new gs_cgraph();
  cg->levels = levels;
  st = gs_graph_load(desc, &cg->g);
  if (st != GS_OK) {
    cgraph_release(cg);
    return st;
  }
  cg->E = cg->g->d.E;
  cg->c = compress(*desc, levels, delta);
  st = load_weighted(cg, desc->num_types);
  if (st == GS_OK) {
    cudaError_t e = gs::dev_malloc(&cg->d_group, sizeof(uint32_t) * cg->c.V);
    if (e == cudaSuccess) e = cudaMemcpy(cg->d_group, cg->c.group.data(), sizeof(uint32_t) * cg->c.V, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cg->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) st = cuda_fail(e, "compressed graph set-up");
  }
  if (st != GS_OK) {
    cgraph_release(cg);
    return st;
  }
  *out = cg;
  return GS_OK;
}

extern "C" void gs_cgraph_free(gs_cgraph *cg) {
  if (cg) cgraph_release(cg);
}

extern "C" gs_status gs_cgraph_get_info(const gs_cgraph *cg, gs_cgraph_info *out) {
  if (!cg || !out) return fail(GS_ERR_INVALID, "gs_cgraph_get_info: null argument");
  out->levels = cg->levels;
  out->vertices = cg->c.V;
  out->edges = cg->E;
  out->nodes = cg->c.n;
  out->weighted_edges = cg->c.edges.size();
  out->inner_edges = cg->inner;
  out->ratio = (double)(cg->c.n + cg->c.edges.size() + cg->inner) / (double)(cg->c.V + cg->E);
  return GS_OK;
}

extern "C" gs_status gs_cgraph_export(const gs_cgraph *cg, uint32_t *group, uint32_t *src, uint32_t *rel, uint32_t *dst,
                                      uint32_t *wout, uint32_t *win, uint32_t *wnode) {
  if (!cg) return fail(GS_ERR_INVALID, "gs_cgraph_export: null graph");
  const Compression &c = cg->c;
  if (group) memcpy(group, c.group.data(), sizeof(uint32_t) * c.V);
  for (size_t i = 0; i < c.edges.size(); ++i) {
    if (src) src[i] = c.edges[i].src;
    if (rel) rel[i] = c.edges[i].rel;
    if (dst) dst[i] = c.edges[i].dst;
    if (wout) wout[i] = c.edges[i].wout;
    if (win) win[i] = c.edges[i].win;
  }
  if (wnode) memcpy(wnode, c.wnode.data(), sizeof(uint32_t) * c.wnode.size());
  return GS_OK;
}

extern "C" gs_status gs_cgraph_candidates(gs_cgraph *cg, const gs_query *q, uint64_t *off, uint32_t *ids,
                                          uint64_t cap_ids, uint64_t *n_ids) {
  if (!cg || !q) return fail(GS_ERR_INVALID, "gs_cgraph_candidates: null argument");
  std::lock_guard<std::mutex> lk(cg->mu);
  WQueries w;
  weighted_queries(cg, q, 1, &w);
  return gs_inspect_candidates(cg->gw, w.qs.data(), GS_STAGE_FIXPOINT, off, ids, cap_ids, n_ids);
}

extern "C" gs_status gs_match_batch_compressed(gs_cgraph *cg, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                                               gs_result *outs) {
  if (!cg || !outs || (n && !qs)) return fail(GS_ERR_INVALID, "gs_match_batch_compressed: null argument");
  if (n == 0) return GS_OK;
  if (opts && opts->mode == GS_CHUNKED)
    return fail(GS_ERR_UNSUPPORTED, "GS_CHUNKED is not offered through a compressed graph");
  std::lock_guard<std::mutex> lk(cg->mu);
  GS_CUDA(cudaSetDevice(cg->g->device));
  // 1. the weighted graph: filter (Definition 3.5), exploration, refinement to the fixpoint
  WQueries w;
  weighted_queries(cg, qs, n, &w);
  gs_match_opts wo;
  memset(&wo, 0, sizeof(wo));
  wo.mode = GS_COUNT_ONLY;
  wo.cuda_stream = cg->stream;
  if (!cg->wb || !batch_rearm(cg->wb, w.qs.data(), n, &wo)) {
    if (cg->wb) batch_destroy(cg->wb);
    cg->wb = nullptr;
    gs_status st = batch_create(cg->gw, w.qs.data(), n, &wo, 0, &cg->wb);
    if (st != GS_OK) return st;
  }
  gs_batch *wb = cg->wb;
  if (wb->waves.size() != 1) return fail(GS_ERR_UNSUPPORTED, "the weighted-graph stage needs the batch in one wave");
  wb->use_graph = false;
  wb->fixpoint = true;
  if (wb->refine_rounds == 0) wb->refine_rounds = 1;
  const cudaStream_t s = cg->stream;
  GS_CUDA(cudaMemsetAsync(&wb->W.ctrl->wave, 0, sizeof(uint32_t), s));
  enqueue_wave(wb, wb->wave_k[0], false, &wb->evs);
  gs_status st = refine_to_fixpoint(wb);
  if (st != GS_OK) return st;
  std::vector<uint32_t> wst(n);  // a query the stage could not finish gets no restriction
  GS_CUDA(cudaMemcpy2DAsync(wst.data(), 4, &wb->W.dq[0].status, sizeof(DQuery), 4, n, cudaMemcpyDeviceToHost, s));
  GS_CUDA(cudaStreamSynchronize(s));
  // 2. the data graph, every candidate test restricted to the stage's sets
  gs_match_opts go;
  if (opts) go = *opts;
  else memset(&go, 0, sizeof(go));
  go.cuda_stream = cg->stream;
  if (!cg->gb || !batch_rearm(cg->gb, qs, n, &go)) {
    if (cg->gb) batch_destroy(cg->gb);
    cg->gb = nullptr;
    st = batch_create(cg->g, qs, n, &go, 0, &cg->gb);
    if (st != GS_OK) return st;
  }
  gs_batch *gb = cg->gb;
  std::vector<uint64_t> masks(n, 0);
  for (uint32_t i = 0; i < n; ++i)
    if (wb->hstatus[i] == GS_OK && wst[i] == QS_OK)
      masks[i] = (uint64_t)(uintptr_t)(wb->W.bm + (uint64_t)wb->hq[i].qv_base * wb->W.slot_words);
  st = batch_set_wmasks(gb, masks.data(), (uint32_t)wb->W.slot_words, cg->d_group);
  if (st == GS_OK) st = run_waves(gb);
  gb->ran = st == GS_OK;
  if (st == GS_OK) st = batch_finish(gb);
  if (st == GS_OK) st = batch_fetch(gb, outs);
  // 3. the stage's bitmaps back to zero for the next call
  launch_clear(wb->W, s, wb->sms);
  GS_CUDA(cudaStreamSynchronize(s));
  return st;
}
