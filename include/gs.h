/*
 * gs.h — C ABI of the GB300 engine for exact labeled subgraph matching
 * (the filtering-and-joining method of thesis arXiv:1807.08804, Ch. 3,
 * Algorithm "FilteringAndJoining").
 *
 * What a match is (Definition 3.2, read for directed graphs whose edges carry
 * relation labels, Section 3.2 "Commonsense Graph Transformation"): given a
 * data graph G = (V, E subset of V x R x V, type: V -> [0,T)) and a query with
 * k vertices and m directed labeled edges, an embedding is an injective map
 * f: [0,k) -> V such that
 *   - a bound query vertex i (a "concept node", Section 3.2) has f(i) = vbind[i];
 *   - a typed query vertex i has type(f(i)) = vtype[i] (GS_ANY: no constraint);
 *   - every query edge (i -> j, r) has (f(i), r, f(j)) in E; a variable edge
 *     (r = GS_ANY, Section 3.2: a relation may be a variable) needs
 *     (f(i), r', f(j)) in E for some relation r'.  An embedding is a map of
 *     vertices, so a pair joined under several relations counts once.
 * The engine returns every embedding: the exact count always, plus the
 * lexicographically smallest `cap` embeddings written in query-vertex order.
 * With a projection (gs_match_opts.project, Section 3.5: only the matches
 * of a subset of the query vertices are wanted) the rows are instead the
 * lexicographically smallest `cap` DISTINCT tuples (f(u)) over the
 * projected vertices u, in ascending u; count and fingerprint still cover
 * every embedding.
 *
 * Conventions for every call:
 *   - Return value: a gs_status.  On failure nothing is returned through the
 *     output arguments and gs_last_error() holds a message for this thread.
 *   - Pointers are host pointers unless a flag says they are device pointers.
 *   - The library copies every input; the caller keeps ownership of its arrays.
 *   - Memory the library returns (gs_result.rows) is freed with gs_result_free.
 *   - All ids are uint32.  Limits: V < 2^24, num_rels <= 255, num_types <= 255,
 *     1 <= k <= 16, m <= 120 edges per query.
 *   - Work runs on the CUDA device that is current when gs_graph_load is
 *     called; later calls on that graph must run with the same device current.
 */
#ifndef GS_H_
#define GS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID = 1,      /* bad argument or query; nothing was done */
  GS_ERR_OOM = 2,          /* device or host allocation failed */
  GS_ERR_CUDA = 3,         /* a CUDA call failed; see gs_last_error() */
  GS_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
  GS_ERR_UNSUPPORTED = 5,  /* valid but outside this build (e.g. disconnected query) */
  GS_ERR_BUSY = 6,         /* serving queue full; retry later */
  GS_ERR_NOT_READY = 7     /* serving result not finished yet */
} gs_status;

#define GS_UNBOUND 0xFFFFFFFFu  /* vbind[i]: variable vertex (no binding) */
#define GS_ANY 0xFFFFFFFFu      /* vtype[i]: no type constraint; erel[j]: any relation */

/* gs_graph_desc.flags */
#define GS_DEVICE_PTRS 1u       /* the arrays are device pointers (read on cuda_stream) */

/*
 * A data graph as an out-CSR (Section 3.3.1: "nodes array" of start offsets
 * and "edges array" of neighbours, plus label arrays of length |V| and |E|).
 * Rows may be in any order and may repeat a (src, rel, dst) triple; the
 * library sorts each row by (relation, neighbour), drops repeats and builds
 * the incoming CSR as well (Section 3.5, "incoming and outgoing graph
 * representations"), plus, per direction, the rows of distinct neighbours
 * over all relations that variable edges read.
 */
typedef struct {
  uint32_t num_vertices;        /* V */
  uint64_t num_edges;           /* E = row_offsets[V] */
  const uint64_t *row_offsets;  /* [V+1], non-decreasing, row_offsets[0] = 0 */
  const uint32_t *col_targets;  /* [E], each < V, no self-loops required (they never match) */
  const uint32_t *edge_rel;     /* [E], each < num_rels */
  const uint32_t *vertex_type;  /* [V], each < num_types */
  uint32_t num_types, num_rels;
  uint32_t flags;               /* GS_DEVICE_PTRS or 0 */
  void *cuda_stream;            /* cudaStream_t for device inputs; NULL = default stream */
} gs_graph_desc;

typedef struct gs_graph gs_graph;

/* Canonicalise and upload a graph (untimed setup; a few device sorts).
 * Errors: GS_ERR_INVALID (sizes, ids, labels out of range), GS_ERR_OOM,
 * GS_ERR_CUDA.  *out is owned by the caller; free it with gs_graph_free. */
gs_status gs_graph_load(const gs_graph_desc *desc, gs_graph **out);
void gs_graph_free(gs_graph *g);
/* Distinct (src, rel, dst) triples after canonicalisation. */
uint64_t gs_graph_num_edges(const gs_graph *g);
/* The canonical graph as loaded on the device, for checks: plane 0 = out,
 * 1 = in (rows of rel << 24 | neighbour, ascending), 2 = out, 3 = in
 * (distinct neighbours over every relation, ascending); off[V+1] and adj[off[V]]
 * of that plane (host arrays; adj may be NULL to ask for the size, which *n
 * receives).  sig (may be NULL) receives the degree signatures, one byte per
 * (signature plane, vertex) = the distinct neighbours in that direction over
 * that relation saturated at 15, planes dir * num_rels + rel, then
 * 2 * num_rels + dir over every relation: (2 * num_rels + 2) * V bytes.
 * Errors: GS_ERR_INVALID (plane > 3, null graph), GS_ERR_CUDA. */
gs_status gs_graph_export(const gs_graph *g, uint32_t plane, uint64_t *off, uint32_t *adj, uint64_t *n,
                          uint8_t *sig);

/*
 * Domain-graph exploration (Ch. 5, "Domain-specific knowledge graph
 * generation": the knowledge graph is explored a few levels out from chosen
 * seed concepts to collect the concepts of a domain).  level_out[v] = the hop
 * count of a shortest path from any seed to v when it is at most `levels`,
 * else 255 (seeds are level 0).  A hop follows an edge forwards
 * (GS_KHOP_OUT) and/or backwards (GS_KHOP_IN) over the listed relations.
 * counts[l] = vertices at level l (host array of levels + 1); edges_scanned
 * (may be NULL) = adjacency entries read.  Errors: levels > 254, directions
 * 0 or unknown, a relation or a seed out of range -> GS_ERR_INVALID.  Host
 * seeds are checked before any work; device seeds (GS_DEVICE_PTRS) are
 * checked on the device, so on that error the device level_out may already
 * have been written (counts and edges_scanned are not).  Calls on one graph
 * are serialised.
 */
#define GS_KHOP_OUT 1u
#define GS_KHOP_IN 2u
typedef struct {
  uint32_t levels;         /* hops to explore, 0..254 */
  uint32_t directions;     /* GS_KHOP_OUT, GS_KHOP_IN or both */
  const uint32_t *rels;    /* host array of the relations to follow; NULL = every relation */
  uint32_t nrels;
  uint32_t flags;          /* GS_DEVICE_PTRS: seeds and level_out are device pointers */
  void *cuda_stream;       /* stream for the work; NULL = the library's own */
} gs_khop_opts;
gs_status gs_khop(gs_graph *g, const uint32_t *seeds, uint32_t nseeds, const gs_khop_opts *opts,
                  uint8_t *level_out /* [V] */, uint64_t *counts /* [levels + 1] */, uint64_t *edges_scanned);

/*
 * A query graph (Section 3.2: concept nodes, variable nodes, labeled edges).
 * Edges are directed esrc[j] -> edst[j] with relation erel[j].  Repeated
 * edges are dropped.  Errors: k = 0 or k > 16, m > 120, an endpoint >= k, a
 * self-loop, a type/relation/binding out of range -> GS_ERR_INVALID; a
 * disconnected query -> GS_ERR_UNSUPPORTED.  Host pointers.
 */
typedef struct {
  uint32_t k, m;
  const uint32_t *vtype;  /* [k], < num_types or GS_ANY */
  const uint32_t *vbind;  /* [k], < V or GS_UNBOUND */
  const uint32_t *esrc;   /* [m] */
  const uint32_t *edst;   /* [m] */
  const uint32_t *erel;   /* [m], < num_rels or GS_ANY (variable edge) */
} gs_query;

/* gs_match_opts.mode */
#define GS_ENUMERATE 0u    /* count + fingerprint + smallest `cap` rows */
#define GS_COUNT_ONLY 1u   /* count + fingerprint, no rows */
#define GS_CHUNKED 2u      /* count + fingerprint, and EVERY embedding streamed to on_chunk */

/* Chunk callback of GS_CHUNKED: `rows` is a DEVICE pointer to num_rows rows
 * of k uint32 ids each (row-major, query-vertex order; rows in no particular
 * order), valid only during the call (copy with gs_memcpy_d2h or a kernel
 * of the caller's).  `query` is the index of the query in the batch.  The
 * callback runs on the thread that called gs_match / gs_match_batch /
 * gs_batch_finish, after the chunk's kernels have completed; it must not
 * call back into the library except gs_memcpy_d2h. */
typedef void (*gs_chunk_cb)(const uint32_t *rows, uint64_t num_rows, uint32_t k, uint32_t query, void *user);

typedef struct {
  uint64_t cap;               /* rows to return (0 = none); the count is always exact */
  uint32_t mode;              /* GS_ENUMERATE, GS_COUNT_ONLY or GS_CHUNKED */
  uint32_t max_refine_rounds; /* 0 = refine until nothing changes (Section 3.3.3) */
  uint64_t chunk_bytes;       /* partial-embedding budget per join level before the
                                 join switches to chunked depth-first expansion, and
                                 (GS_CHUNKED) the size bound of each streamed chunk;
                                 0 = library default (1 GiB) */
  void *cuda_stream;          /* cudaStream_t; NULL = the library's own stream */
  gs_chunk_cb on_chunk;       /* GS_CHUNKED: required; otherwise ignored */
  void *user;                 /* passed to on_chunk */
  uint32_t project;           /* bit u set: return f(u); 0 (or every vertex) = whole
                                 embeddings.  A bit >= k -> GS_ERR_INVALID; with
                                 GS_CHUNKED -> GS_ERR_UNSUPPORTED */
  uint32_t refine;            /* refinement variant (Section 3.3.3 and the refinement
                                 experiments of Section 3.6): 0 = every query vertex
                                 at once; GS_REFINE_OFF, GS_REFINE_REVERSED, and
                                 GS_REFINE_LOW(d) (may be or-ed).  Results never depend
                                 on it: refinement only prunes candidates */
} gs_match_opts;

/* gs_match_opts.refine */
#define GS_REFINE_OFF 1u       /* no refinement after exploration */
#define GS_REFINE_REVERSED 2u  /* one query vertex at a time, in the reverse of the order in
                                  which exploration gave the vertices candidate sets */
#define GS_REFINE_LOW(d) (((uint32_t)(d) & 0xFFu) << 8)  /* skip "low connectivity" query
                                  vertices (at most d incident edges): not refined, and
                                  their edges not used to refine others */
#define GS_REFINE_BASELINE 4u  /* the comparison baseline of Section 3.6's refinement
                                  experiments: only the outgoing graph filters (a spanning-tree
                                  child reached against an edge's direction gets its whole
                                  Definition 3.3 candidate set, as by a scan of every vertex),
                                  exploration checks and expands spanning-tree edges only, no
                                  neighbour-type test, no refinement */

/* Synchronous copy of `bytes` bytes from device memory to host memory, for
 * chunk callbacks.  Returns GS_ERR_CUDA if the copy fails. */
gs_status gs_memcpy_d2h(void *dst, const void *src, uint64_t bytes);

typedef struct {
  uint64_t count;        /* exact number of embeddings */
  uint64_t num_rows;     /* rows returned = min(count, cap) (projected: min(distinct
                            tuples, cap)); 0 for GS_CHUNKED */
  uint64_t fingerprint;  /* sum over ALL embeddings of an order-free 64-bit row hash */
  uint32_t k;            /* row width: query vertices, or projected vertices */
  uint32_t truncated;    /* 1 if count > cap (projected: more distinct tuples than cap) */
  uint32_t *rows;        /* [num_rows * k] row-major, query-vertex order, ascending; owned
                            unless `shared` */
  uint32_t status;       /* gs_status of this query (batch calls) */
  uint32_t shared;       /* 1: rows lie in a block shared by the results of one
                            gs_match_batch_shared call (gs_result_free leaves them) */
} gs_result;

/* Match one query (a batch of one).  Blocks until the result is on the host. */
gs_status gs_match(gs_graph *g, const gs_query *q, const gs_match_opts *opts, gs_result *out);

/* Match n queries as one batch: every phase runs once for all of them.
 * outs[n] receive per-query results (outs[i].status says whether query i was
 * valid).  Returns GS_OK unless the call itself failed. */
gs_status gs_match_batch(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                         gs_result *outs);

/* gs_match_batch without a copy of the rows on the host: the results' rows
 * lie in page-locked host buffers that the device wrote directly (one per
 * sub-batch: a call of 4,096 queries or more, without a stream of the
 * caller's, runs as four sub-batches at once on streams of their own), and
 * each such result has shared = 1.  *block receives the buffers (NULL when
 * no row is shared); the rows stay valid until gs_rows_release(block), which
 * returns the buffers to a library pool for later calls.  gs_rows_count
 * gives the number of buffers, gs_rows_base/gs_rows_words buffer i's address
 * and size in uint32 words.  Results of queries finished on the chunked path
 * own their rows as usual.  Errors as gs_match_batch. */
typedef struct gs_rows gs_rows;
gs_status gs_match_batch_shared(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                                gs_result *outs, gs_rows **block);
uint32_t gs_rows_count(const gs_rows *block);
const uint32_t *gs_rows_base(const gs_rows *block, uint32_t i);
uint64_t gs_rows_words(const gs_rows *block, uint32_t i);
void gs_rows_release(gs_rows *block);

void gs_result_free(gs_result *r);
/* gs_result_free on each of r[0..n). */
void gs_results_free(gs_result *r, uint32_t n);
/* Copy the rows of r[0..n) into dst back to back: r[0]'s num_rows*k words,
 * then r[1]'s, and so on (dst holds the sum; host memory).  The results keep
 * their rows.  Errors: GS_ERR_INVALID for a null pointer. */
gs_status gs_results_copy_rows(const gs_result *r, uint32_t n, uint32_t *dst);
const char *gs_last_error(void);

/* Bytes copied host->device and device->host by all gs_match and
 * gs_match_batch calls on this graph so far (query descriptors in; counts,
 * fingerprints and rows out). */
gs_status gs_graph_io_bytes(gs_graph *g, uint64_t *h2d, uint64_t *d2h);

/* ------------------------------------------------------------------------
 * Prepared batches: the queries are validated, packed and uploaded once; each
 * gs_batch_run then executes the whole device pipeline (plan, filter,
 * refinement, edge tables, join, sort) from device-resident inputs, replaying
 * a captured CUDA graph.  Results stay in device memory until gs_batch_fetch.
 * ------------------------------------------------------------------------ */
typedef struct gs_batch gs_batch;
gs_status gs_batch_create(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                          gs_batch **out);
/* Enqueue one run on the batch's stream (asynchronous). */
gs_status gs_batch_run(gs_batch *b);
/* Run nb prepared batches at once, each on its own stream (their streams
 * must differ): every batch starts after the work queued so far on
 * cuda_stream (NULL = the legacy default stream), their kernels overlap on
 * the device, and cuda_stream waits for all of them.  Finish and fetch each
 * batch as after gs_batch_run.  Errors: GS_ERR_INVALID (no batch, a null
 * batch, two batches on one stream), GS_ERR_CUDA. */
gs_status gs_batch_run_all(gs_batch **bs, uint32_t nb, void *cuda_stream);
/* Wait for the last run, finish queries that overflowed the device budgets
 * (chunked join on the host-driven path), and make results fetchable. */
gs_status gs_batch_finish(gs_batch *b);
/* Copy results of the last finished run to the host (outs[n]). */
gs_status gs_batch_fetch(gs_batch *b, gs_result *outs);

/* Partial-embedding words of each query in the last finished run, for
 * measuring refinement (Section 3.6: "intermediate results"): words_total[i]
 * = sum over the join levels before the last of rows x width, words_peak[i]
 * = the largest of those levels (uint32 words; the device pipeline's levels,
 * not those of a query finished on the chunked path).  Host arrays of the
 * batch's n entries.  Errors: GS_ERR_INVALID before gs_batch_finish. */
gs_status gs_batch_join_sizes(gs_batch *b, uint64_t *words_total, uint64_t *words_peak);
void gs_batch_destroy(gs_batch *b);
/* Waves of `wave_queries` queries each: every phase runs per wave (1 = one
 * query at a time through the same device pipeline). */
gs_status gs_batch_create_waves(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                                uint32_t wave_queries, gs_batch **out);
/* Execution knobs: captured graph or direct launches, lanes per work item
 * (4, 8, 16 or 32), refinement rounds (0 = until nothing changes;
 * GS_ROUNDS_NONE = no refinement round after exploration). */
#define GS_ROUNDS_NONE 0xFFFFFFFFu
gs_status gs_batch_set(gs_batch *b, int use_graph, int group, uint32_t refine_rounds);
/* Sort of the outputs above the one-block limit (more than 2,048 rows) into
 * the ascending lexicographic row order in which results are returned: by
 * default a sample sort (buckets bounded by splitters drawn from the
 * query's rows, each bucket sorted in shared memory), with the tile sort and
 * merge passes for a query whose bucket overflows.  GS_SORT_MERGE_ONLY sorts
 * every large output by the tile sort and merge passes (same results; for
 * tests of that path).  Applies to the batch's later runs.  Errors:
 * GS_ERR_INVALID (null batch, unknown flag). */
#define GS_SORT_MERGE_ONLY 1u
gs_status gs_batch_set_sort(gs_batch *b, uint32_t flags);
/* Bound on the one device-side wait of the pipeline: the look-back of the
 * single-pass prefix scans that size every output (Section 3.3.4's two-step
 * output scheme: count, prefix sum, write).  A block waits there only on
 * tiles that earlier, running blocks claimed, so the wait ends; it is bounded
 * all the same.  max_polls = reads of a predecessor tile's state before the
 * wait gives up (0 = the default, 2^22).  A wait that gives up sums the scan's
 * inputs before its tile directly, so every result stays exact, and records
 * the event; the next gs_batch_finish then returns GS_ERR_TIMEOUT and clears
 * the record (fetch nothing from that run).  GS_WAIT_WITHHOLD_FIRST_TILE is
 * for tests of this path: the first tile of every scan of more than one tile
 * (2,048 counts) publishes nothing, so each later tile's wait runs to the
 * bound.  Applies to the batch's later runs, in stream order.  Errors:
 * GS_ERR_INVALID (null batch, unknown flag), GS_ERR_CUDA. */
#define GS_WAIT_WITHHOLD_FIRST_TILE 1u
gs_status gs_batch_set_wait(gs_batch *b, uint32_t max_polls, uint32_t flags);
/* Kernels launched by runs so far, bytes moved between host and device, and
 * queries finished on the host-driven chunked path by the last finish. */
gs_status gs_batch_counters(gs_batch *b, uint64_t *kernel_launches, uint64_t *h2d, uint64_t *d2h,
                            uint64_t *fallback_queries);

/* Per-kernel statistics accumulated by runs since the last reset:
 * launches, device time (CUDA events) and algorithmic bytes.  Timing is
 * recorded only while enabled (adds events around each launch). */
#define GS_NUM_KERNEL_KINDS 16
typedef struct {
  const char *name[GS_NUM_KERNEL_KINDS];
  uint64_t launches[GS_NUM_KERNEL_KINDS];
  double ms[GS_NUM_KERNEL_KINDS];
  uint64_t bytes[GS_NUM_KERNEL_KINDS];
} gs_kernel_stats;
gs_status gs_stats_enable(gs_batch *b, int on);
gs_status gs_stats_get(gs_batch *b, gs_kernel_stats *out);
gs_status gs_stats_reset(gs_batch *b);
/* Per kernel kind, the device time during which at least one launch of that
 * kind was running, over the timed runs of the nb batches since their last
 * resets: the union of the launches' intervals (CUDA events on the streams
 * they ran on, taken from an anchor event recorded before each run's first
 * launch; batches run together by gs_batch_run_all share one anchor), summed
 * over runs.  Launches of one kind that overlap, as those of batches run
 * together do, count once.  busy_ms: GS_NUM_KERNEL_KINDS doubles, written.
 * Errors: GS_ERR_INVALID (null argument or batch). */
gs_status gs_stats_busy(gs_batch *const *bs, uint32_t nb, double *busy_ms);

/* ------------------------------------------------------------------------
 * Autotuning.  Times the captured pipeline on the given queries for each
 * lanes-per-work-item setting (4, 8, 16, 32: the lanes that share one
 * candidate vertex, edge-table key or partial embedding) and each number of
 * refinement rounds (none, 1, 2, 4), then 4 or 8 lanes per partial embedding
 * for the join alone, and keeps the fastest for batches created on this
 * graph afterwards.  Results never depend on these settings.  With
 * cache_path != NULL the choice is read from / appended to that text file,
 * keyed by graph content hash, GPU name and a signature of the query load
 * (batch size class, mean k and m, bound fraction, mode).
 * ------------------------------------------------------------------------ */
typedef struct {
  uint32_t group;          /* lanes per work item */
  uint32_t refine_rounds;  /* refinement rounds in captured runs */
  double ms;               /* best time of one run of the given queries */
  uint32_t from_cache;     /* 1 if read from cache_path */
  uint32_t configs_tried;
  uint32_t join_group;     /* lanes per partial row in the join */
  uint32_t reserved;
} gs_tuning;
gs_status gs_tune(gs_graph *g, const gs_query *qs, uint32_t n, const gs_match_opts *opts, const char *cache_path,
                  gs_tuning *out);
/* Set the tuned values by hand (0 = library default; refine_rounds may be
 * GS_ROUNDS_NONE); the join takes the same lanes per work item. */
gs_status gs_tune_set(gs_graph *g, uint32_t group, uint32_t refine_rounds);

/* ------------------------------------------------------------------------
 * Inspection of the filtering phase and the candidate-edge tables of one
 * query, for per-kernel parity checks.
 * ------------------------------------------------------------------------ */
#define GS_STAGE_FILTER 0u    /* C0(u): binding, type, per-(direction, relation) degree */
#define GS_STAGE_FIXPOINT 1u  /* after exploration and refinement to a fixpoint */

/* Candidate sets of query q at `stage` as sorted lists: for query vertex u,
 * ids[off[u] .. off[u+1]) ascending.  off has k+1 entries; ids has room for
 * `cap_ids`; *n_ids receives the total (GS_ERR_INVALID if cap_ids is too
 * small; ids may be NULL to ask for the size).  Host pointers. */
gs_status gs_inspect_candidates(gs_graph *g, const gs_query *q, uint32_t stage, uint64_t *off,
                                uint32_t *ids, uint64_t cap_ids, uint64_t *n_ids);

/* Candidate-edge table of query edge e after the fixpoint (Section 3.3.4),
 * oriented from esrc[e] (from_src = 1: keys = C(esrc), lists of out-neighbours
 * in C(edst)) or from edst[e] (from_src = 0: keys = C(edst), lists of
 * in-neighbours in C(esrc)).  keys[nkeys], off[nkeys+1], vals[off[nkeys]].
 * With keys == NULL only *nkeys and *nvals are written. */
gs_status gs_inspect_edge_table(gs_graph *g, const gs_query *q, uint32_t e, uint32_t from_src, uint32_t *keys,
                                uint64_t *off, uint32_t *vals, uint64_t cap_keys, uint64_t cap_vals,
                                uint64_t *nkeys, uint64_t *nvals);

/* ------------------------------------------------------------------------
 * Candidate filter without allocation.  The thesis has no counterpart: this
 * is an interface for callers that must not let the library allocate (a
 * process that reserved its device memory budget up front, or one whose own
 * allocator owns the device; cudaMalloc/cudaFree can also stall the device).
 *
 * Writes the candidates of query vertex u (binding, type and the
 * per-direction, per-relation degree test; the same set gs_inspect_candidates
 * reports at GS_STAGE_FILTER) in ascending order to d_ids[0 .. min(n, cap_ids))
 * and their number n to *d_count, both device pointers owned by the caller,
 * asynchronously on cuda_stream (NULL = default stream).
 *
 * It calls no allocating routine.  Its scratch is one fixed array inside the
 * library (196,616 bytes per device, held until the process exits), which
 * limits the graph to 2^24 vertices (larger graphs: GS_ERR_INVALID).  Every
 * call on a device shares that array, so calls that overlap on the GPU race:
 * serialise them.  The first call on each device looks up the array's device
 * address; make that first call before any stream capture.
 * Errors: GS_ERR_INVALID (null pointers, bad query, u >= k, too many vertices).
 * ------------------------------------------------------------------------ */
gs_status gs_filter_candidates_static(gs_graph *g, const gs_query *q, uint32_t u, uint32_t *d_ids, uint64_t cap_ids,
                                      uint64_t *d_count, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Multi-level graph compression (Section 3.4) and matching through it
 * (Section 3.5).  gs_cgraph_build compresses a data graph offline, on the
 * host: `levels` levels (0-32), each pairing similar nodes with threshold
 * delta[l] in (0, 1], into a weighted graph whose nodes stand for groups of
 * data vertices (mapping lists).  Readings, for directed graphs with
 * relations and vertex types:
 *   - adj(x) = the (direction, relation, other node) triples of x's edges to
 *     other nodes; x and y are similar when they have one type and the
 *     triples both have number at least delta * |adj(x)| and at least
 *     delta * |adj(y)| (double-precision products; the thesis's test as
 *     printed always holds), or when neither has edges; with delta = 1 similar
 *     nodes have equal adjacency lists;
 *   - a level visits nodes in index order and pairs each unpaired node with
 *     the lowest-indexed later unpaired node similar to it; merged nodes are
 *     numbered by ascending smallest member;
 *   - edge weights start at 1 and follow w(u, v) = max(w(p, n), w(q, n)) +
 *     max(w(p, m), w(q, m)) per relation (Definition 3.4's recursion), wout
 *     bounding the out-neighbours in M(v) of any member of M(u), win the
 *     in-neighbours in M(u) of any member of M(v); edges inside a node are not
 *     edges of the weighted graph; the node weight per direction and relation
 *     is the most neighbours a member has inside its own node;
 *   - Definition 3.5, per direction and relation: a node is a candidate of a
 *     query vertex with c neighbours there when its node weight plus the
 *     weights of its edges there is at least c (variable edges: the sum over
 *     every relation).
 * The data graph and the weighted graph are both loaded on the current
 * device; the arrays must be host pointers (GS_DEVICE_PTRS ->
 * GS_ERR_UNSUPPORTED).  Errors as gs_graph_load, and GS_ERR_INVALID for more
 * than 32 levels or a threshold outside (0, 1].
 * ------------------------------------------------------------------------ */
/* The compression alone, on the host (no CUDA call, no device needed):
 * *nodes and *weighted_edges receive the sizes; then, for each non-NULL
 * array, group[V], src/rel/dst/wout/win[*weighted_edges] and
 * wnode[2 * num_rels * *nodes] as gs_cgraph_export writes them.  Arrays
 * sized for the bounds (num_edges entries, 2 * num_rels * V words) are
 * always large enough.  The graph's arrays are checked on the host. */
gs_status gs_compress_host(const gs_graph_desc *desc, uint32_t levels, const double *delta, uint32_t *nodes,
                           uint64_t *weighted_edges, uint32_t *group, uint32_t *src, uint32_t *rel, uint32_t *dst,
                           uint32_t *wout, uint32_t *win, uint32_t *wnode);
typedef struct gs_cgraph gs_cgraph;
gs_status gs_cgraph_build(const gs_graph_desc *desc, uint32_t levels, const double *delta, gs_cgraph **out);
void gs_cgraph_free(gs_cgraph *cg);
typedef struct {
  uint32_t levels;
  uint32_t vertices;        /* V of the data graph */
  uint64_t edges;           /* distinct data triples */
  uint32_t nodes;           /* nodes of the weighted graph */
  uint32_t reserved;
  uint64_t weighted_edges;  /* its edges between different nodes */
  uint64_t inner_edges;     /* (node, relation) pairs with edges inside the node */
  double ratio;             /* (nodes + weighted_edges + inner_edges) / (vertices + edges),
                               the thesis's compression ratio */
} gs_cgraph_info;
gs_status gs_cgraph_get_info(const gs_cgraph *cg, gs_cgraph_info *out);
/* The compression itself, for checks: group[vertices] = the node holding
 * each data vertex; the weighted edges src/rel/dst/wout/win[weighted_edges]
 * sorted by (src, rel, dst); wnode[(dir * num_rels + rel) * nodes + x]
 * (dir 0 = out, 1 = in).  Host arrays; any may be NULL. */
gs_status gs_cgraph_export(const gs_cgraph *cg, uint32_t *group, uint32_t *src, uint32_t *rel, uint32_t *dst,
                           uint32_t *wout, uint32_t *win, uint32_t *wnode);
/* Candidate sets of a query on the weighted graph (Definition 3.5, then
 * exploration and refinement to the fixpoint, two query vertices allowed on
 * one node), as gs_inspect_candidates: node ids per query vertex.  Bindings
 * are data vertices; each is replaced by the node holding it. */
gs_status gs_cgraph_candidates(gs_cgraph *cg, const gs_query *q, uint64_t *off, uint32_t *ids, uint64_t cap_ids,
                               uint64_t *n_ids);
/* gs_match_batch through the compressed graph: the queries' candidate sets
 * on the weighted graph (as gs_cgraph_candidates) restrict every candidate
 * test of the device pipeline on the data graph to the vertices of their
 * nodes' mapping lists (Theorem 3.2: no other vertex is a match), so the
 * results are every embedding in the data graph, the same as gs_match_batch
 * on it.  GS_CHUNKED -> GS_ERR_UNSUPPORTED; a batch too large for one wave
 * of the weighted-graph stage -> GS_ERR_UNSUPPORTED.  Calls on one compressed
 * graph are serialised. */
gs_status gs_match_batch_compressed(gs_cgraph *cg, const gs_query *qs, uint32_t n, const gs_match_opts *opts,
                                    gs_result *outs);

/* ------------------------------------------------------------------------
 * Serving: a request loop that keeps the graph device-resident and admits
 * queries while slots and the working-set budget allow (continuous batching:
 * requests that arrive while others run are admitted as slots free up).
 * ------------------------------------------------------------------------ */
typedef struct {
  uint64_t budget_bytes;  /* working-set budget for admitted queries (0 = 40 GB) */
  uint32_t slots;         /* concurrent micro-batches in flight (0 = 4) */
  uint32_t max_batch;     /* queries per micro-batch (0 = 256) */
  uint32_t queue_depth;   /* pending requests before submit says GS_ERR_BUSY (0 = 65536) */
  uint32_t reserved;
} gs_serve_opts;

typedef struct gs_server gs_server;
gs_status gs_serve_create(gs_graph *g, const gs_serve_opts *opts, gs_server **out);
/* Queue one query; *ticket identifies it.  The query is copied. */
gs_status gs_serve_submit(gs_server *s, const gs_query *q, const gs_match_opts *opts, uint64_t *ticket);
/* Non-blocking: GS_ERR_NOT_READY until the result is done; then fills *out
 * (free with gs_result_free) and forgets the ticket.  *latency_s (may be NULL)
 * receives submit-to-completion time in seconds. */
gs_status gs_serve_poll(gs_server *s, uint64_t ticket, gs_result *out, double *latency_s);
gs_status gs_serve_destroy(gs_server *s);

/* ------------------------------------------------------------------------
 * Failure injection for tests, on the host side only: no kernel is made to
 * fault.  The thesis has no counterpart.
 * ------------------------------------------------------------------------ */
/* After `after` more device allocations by the library (any thread, any
 * graph), the next one fails as if the device were out of memory, without
 * allocating; the call that made it returns GS_ERR_OOM (or reports it per
 * request) and frees what it had allocated.  One-shot; after < 0 disarms. */
void gs_debug_fail_alloc(int64_t after);
/* Serving: the next n completion checks of in-flight micro-batches (across
 * servers) report a CUDA error, as a failed kernel would.  Each such
 * micro-batch is dropped after its work drains and its requests complete with
 * GS_ERR_CUDA; the server keeps serving.  n = 0 disarms. */
void gs_debug_fail_serve_wait(uint32_t n);

#ifdef __cplusplus
}
#endif
#endif /* GS_H_ */
