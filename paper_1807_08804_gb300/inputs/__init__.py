"""Seeded synthetic inputs: data graphs, query graphs and arrival times.

This module holds no matching arithmetic.  Both the CUDA engine and the CPU
oracle are fed from it; neither one imports the other.

The thesis's datasets (SenticNet, Gowalla, Enron; Ch. 3, "Performance
Evaluation") are not available, so seeded synthetic graphs with their shape
stand in for them: large directed graphs whose edges carry relation labels and
whose vertices carry types, and small query graphs grown from a seed vertex so
that they are not only trees.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsgen.c")
_LIB = os.path.join(_HERE, "libgsgen.so")
_lib = None

UNBOUND = 0xFFFFFFFF
ANY = 0xFFFFFFFF


def build() -> str:
    """Compile the generator library in place (plain C, host only)."""
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.gsg_graph.restype = ctypes.c_int
        _lib.gsg_graph.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                   ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_uint32,
                                   ctypes.c_uint64, P, P, P, P, ctypes.c_double, ctypes.c_double]
        _lib.gsg_walk_queries.restype = ctypes.c_int64
        _lib.gsg_walk_queries.argtypes = [ctypes.c_uint32, P, P, P, P, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_uint64, ctypes.c_uint64, P, P, P, P, P, P, P, P]
        _lib.gsg_shape_queries.restype = ctypes.c_int64
        _lib.gsg_shape_queries.argtypes = [ctypes.c_uint32, P, ctypes.c_uint32, P, ctypes.c_uint32,
                                           ctypes.c_uint64, P, P, P, P, P, P, P]
        _lib.gsg_arrivals.restype = None
        _lib.gsg_arrivals.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64, P]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Graph:
    """A directed graph as an out-CSR (row_offsets, col_targets, edge_rel) in
    draw order (unsorted, duplicates already excluded), plus vertex types."""
    num_vertices: int
    row_offsets: np.ndarray  # uint64 [V+1]
    col_targets: np.ndarray  # uint32 [E]
    edge_rel: np.ndarray     # uint32 [E]
    vertex_type: np.ndarray  # uint32 [V]
    num_types: int
    num_rels: int

    @property
    def num_edges(self) -> int:
        return int(self.row_offsets[-1])


@dataclass
class Query:
    """One query graph: k vertices, m directed labeled edges esrc->edst."""
    vtype: np.ndarray  # uint32 [k]; ANY = no type constraint
    vbind: np.ndarray  # uint32 [k]; UNBOUND = variable vertex
    esrc: np.ndarray   # uint32 [m]
    edst: np.ndarray   # uint32 [m]
    erel: np.ndarray   # uint32 [m]
    walked: np.ndarray | None = None  # data ids the query was grown from (a known match)

    @property
    def k(self) -> int:
        return int(self.vtype.shape[0])

    @property
    def m(self) -> int:
        return int(self.esrc.shape[0])


def make_graph(V: int, E: int, T: int = 64, type_s: float = 1.0, R: int = 34, rel_s: float = 1.1,
               alpha: float = 2.1, dmax: int = 1000, seed: int = 1, target_s: float = 0.0,
               copy_p: float = 0.0) -> Graph:
    """Power-law out-degree (density exponent alpha, scaled so the degrees sum
    to E, clamped to [1, dmax]), Zipf types and relations, and uniform
    targets (target_s = 0) or Zipf(target_s) targets over a seeded vertex
    order; with copy_p a vertex copies, with that probability, the out-list
    of the last earlier vertex of its type and out-degree."""
    lib = _load()
    ro = np.zeros(V + 1, np.uint64)
    col = np.zeros(max(E, 1), np.uint32)
    rel = np.zeros(max(E, 1), np.uint32)
    vt = np.zeros(V, np.uint32)
    rc = lib.gsg_graph(V, E, T, type_s, R, rel_s, alpha, dmax, seed, _p(ro), _p(col), _p(rel), _p(vt), target_s,
                       copy_p)
    if rc != 0:
        raise ValueError(f"graph parameters impossible: V={V} E={E} dmax={dmax} R={R}")
    return Graph(V, ro, col[:E], rel[:E], vt, T, R)


def _split(qk, qm, vtype, vbind, walked, esrc, edst, erel):
    out = []
    vo = eo = 0
    for k, m in zip(qk.tolist(), qm.tolist()):
        out.append(Query(vtype[vo:vo + k].copy(), vbind[vo:vo + k].copy(), esrc[eo:eo + m].copy(),
                         edst[eo:eo + m].copy(), erel[eo:eo + m].copy(),
                         None if walked is None else walked[vo:vo + k].copy()))
        vo += k
        eo += m
    return out


def make_walk_queries(g: Graph, n: int, kmin: int, kmax: int, p_close: float = 0.3, p_bind: float = 0.2,
                      cyclic_half: bool = False, seed: int = 1) -> list[Query]:
    """Queries grown by random walks over the undirected view (tree edges =
    traversed data edges), plus every other triple among the walked vertices
    with probability p_close; vertices bound with p_bind, else typed."""
    lib = _load()
    max_e = n * kmax * kmax * 8 + 64
    qk = np.zeros(n, np.uint32)
    qm = np.zeros(n, np.uint32)
    nv = n * kmax
    vtype = np.zeros(nv, np.uint32)
    vbind = np.zeros(nv, np.uint32)
    walked = np.zeros(nv, np.uint32)
    esrc = np.zeros(max_e, np.uint32)
    edst = np.zeros(max_e, np.uint32)
    erel = np.zeros(max_e, np.uint32)
    rc = lib.gsg_walk_queries(g.num_vertices, _p(g.row_offsets), _p(g.col_targets), _p(g.edge_rel),
                              _p(g.vertex_type), n, kmin, kmax, p_close, p_bind, 1 if cyclic_half else 0,
                              seed, max_e, _p(qk), _p(qm), _p(vtype), _p(vbind), _p(walked), _p(esrc),
                              _p(edst), _p(erel))
    if rc < 0:
        raise ValueError("query generation failed")
    return _split(qk, qm, vtype, vbind, walked, esrc, edst, erel)


def top_labels(counts: np.ndarray, n: int) -> np.ndarray:
    """The n most frequent labels (ties to the lower label)."""
    order = np.lexsort((np.arange(counts.shape[0]), -counts.astype(np.int64)))
    return order[:n].astype(np.uint32)


def make_shape_queries(g: Graph, n: int, seed: int = 1, ntop: int = 4) -> list[Query]:
    """Unbound typed shapes in equal shares: directed 4-cycles, directed
    5-cycles, 4-cliques (i->j for i<j) and 6-vertex random trees, over the
    ntop most frequent relations and types."""
    lib = _load()
    rels = top_labels(np.bincount(g.edge_rel, minlength=g.num_rels), ntop)
    types = top_labels(np.bincount(g.vertex_type, minlength=g.num_types), ntop)
    qk = np.zeros(n, np.uint32)
    qm = np.zeros(n, np.uint32)
    vtype = np.zeros(n * 6, np.uint32)
    vbind = np.zeros(n * 6, np.uint32)
    esrc = np.zeros(n * 6, np.uint32)
    edst = np.zeros(n * 6, np.uint32)
    erel = np.zeros(n * 6, np.uint32)
    lib.gsg_shape_queries(n, _p(rels), len(rels), _p(types), len(types), seed, _p(qk), _p(qm), _p(vtype),
                          _p(vbind), _p(esrc), _p(edst), _p(erel))
    return _split(qk, qm, vtype, vbind, None, esrc, edst, erel)


def with_variable_edges(queries: list[Query], p_var: float, seed: int = 1) -> list[Query]:
    """The same queries with each edge's relation replaced by ANY (a variable
    edge) with probability p_var; the walked vertices still match."""
    rng = np.random.default_rng(seed)
    out = []
    for q in queries:
        erel = q.erel.copy()
        erel[rng.random(q.m) < p_var] = ANY
        out.append(Query(q.vtype, q.vbind, q.esrc, q.edst, erel, q.walked))
    return out


def anchor_untyped(queries: list[Query]) -> list[Query]:
    """The same query shapes with one concept node: vertex 0 (where the walk
    started) bound to its walked vertex, every other vertex an untyped
    variable."""
    out = []
    for q in queries:
        vt = np.full(q.k, ANY, np.uint32)
        vb = np.full(q.k, UNBOUND, np.uint32)
        vb[0] = q.walked[0]
        out.append(Query(vt, vb, q.esrc, q.edst, q.erel, q.walked))
    return out


def make_arrivals(n: int, qps: float, seed: int = 1) -> np.ndarray:
    """Poisson arrival times in seconds (exponential inter-arrival gaps)."""
    lib = _load()
    t = np.zeros(n, np.float64)
    lib.gsg_arrivals(n, qps, seed, _p(t))
    return t


@dataclass
class Workload:
    """A named workload: graph sizes and distributions plus its query recipe."""
    name: str
    V: int
    E: int
    n_queries: int
    kmin: int
    kmax: int
    p_bind: float
    cap: int
    seed: int
    cyclic_half: bool = False
    shapes: bool = False
    qps: tuple = field(default_factory=tuple)
    p_var: float = 0.0  # share of query edges made variable (relation ANY)
    anchored: bool = False  # one bound vertex (the walk start), every other vertex untyped
    graph_seed: int | None = None  # the graph's seed when it differs from the queries' seed
    target_s: float = 0.0  # Zipf exponent of edge targets (0 = uniform)
    copy_p: float = 0.0  # share of vertices copying the out-list of an earlier vertex of their type and degree
    deltas: tuple = ()  # compression thresholds per level (matching through a compressed graph)
    count_only: bool = False  # measured in count-only mode

    def graph(self) -> Graph:
        return make_graph(self.V, self.E, seed=self.seed if self.graph_seed is None else self.graph_seed,
                          target_s=self.target_s, copy_p=self.copy_p)

    def queries(self, g: Graph, n: int | None = None) -> list[Query]:
        n = self.n_queries if n is None else n
        if self.shapes:
            qs = make_shape_queries(g, n, seed=self.seed)
        else:
            qs = make_walk_queries(g, n, self.kmin, self.kmax, p_close=0.3, p_bind=self.p_bind,
                                   cyclic_half=self.cyclic_half, seed=self.seed)
        if self.anchored:
            qs = anchor_untyped(qs)
        return with_variable_edges(qs, self.p_var, self.seed + 0x76) if self.p_var > 0 else qs


# The workloads: sizes, label distributions and query recipes.
WORKLOADS = {
    # 10k vertices / 60k edges; 100 queries of 3-6 vertices; cap 2^20
    "single-10k": Workload("single-10k", 10_000, 60_000, 100, 3, 6, 0.2, 1 << 20, 0x6753001),
    # 1M vertices / 8M edges; 1,000 queries of 4-10 vertices; cap 2^22
    "single-1m": Workload("single-1m", 1_000_000, 8_000_000, 1000, 4, 10, 0.2, 1 << 22, 0x6753002),
    # 4M vertices / 32M edges; 10,000 queries of 3-12 vertices, half cyclic
    "batch-4m": Workload("batch-4m", 4_000_000, 32_000_000, 10_000, 3, 12, 0.1, 1 << 20, 0x6753003,
                         cyclic_half=True),
    # the batch-4m graph kept device-resident; Poisson arrivals of queries of 3-12 vertices
    "serve-4m": Workload("serve-4m", 4_000_000, 32_000_000, 20_000, 3, 12, 0.2, 1 << 20, 0x6753004,
                         qps=(1000.0, 5000.0, 20000.0, 50000.0), graph_seed=0x6753003),
    # 16M vertices / 200M edges; 200 unbound shape queries
    "stress-16m": Workload("stress-16m", 16_000_000, 200_000_000, 200, 4, 6, 0.0, 1 << 20, 0x6753005,
                           shapes=True),
    # the single-1m graph with 200 queries of 10-12 vertices, half of them cyclic, each with one
    # concept node and untyped variables elsewhere (refinement measurements, count only)
    "ablation-1m": Workload("ablation-1m", 1_000_000, 8_000_000, 200, 10, 12, 0.0, 1 << 20, 0x6753002,
                            cyclic_half=True, anchored=True),
    # matching through a multi-level compression (three levels at the thesis's SenticNet thresholds
    # 0.8, 0.7, 0.7) of graphs with concept families: edge targets follow Zipf(1.3) over a seeded
    # vertex order (rarely-cited concepts have few incoming edges) and 80% of the vertices copy the
    # out-list of the last earlier vertex of their type and out-degree
    "compress-10k": Workload("compress-10k", 10_000, 60_000, 100, 3, 6, 0.2, 1 << 20, 0x6753006, target_s=1.3,
                             copy_p=0.8, deltas=(0.8, 0.7, 0.7)),
    "compress-1m": Workload("compress-1m", 1_000_000, 8_000_000, 1000, 4, 10, 0.2, 1 << 22, 0x6753007,
                            target_s=1.3, copy_p=0.8, deltas=(0.8, 0.7, 0.7)),
    # the single-1m graph with 200 queries of 16 vertices (the most the engine takes), half of them
    # cyclic, typed or bound as in single-1m (refinement measurements against the thesis's baseline)
    "ablation16-1m": Workload("ablation16-1m", 1_000_000, 8_000_000, 200, 16, 16, 0.2, 1 << 20, 0x6753002,
                              cyclic_half=True, count_only=True),
    # the single-10k and single-1m workloads with 30% of query edges variable
    "single-10k-var": Workload("single-10k-var", 10_000, 60_000, 100, 3, 6, 0.2, 1 << 20, 0x6753001, p_var=0.3),
    "single-1m-var": Workload("single-1m-var", 1_000_000, 8_000_000, 1000, 4, 10, 0.2, 1 << 22, 0x6753002,
                              p_var=0.3),
}
