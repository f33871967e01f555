"""CPU oracle for exact labeled subgraph matching — TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA engine:
the C source `oracle.c` is compiled here with gcc into `liborc.so` and driven
through ctypes.  Each function restates a definition or step of the thesis's
Ch. 3 (see the header of `oracle.c` for the passages).

Parity status: every function here is pinned by `tests/test_oracle_pins.py`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None

UNBOUND = 0xFFFFFFFF
ANY = 0xFFFFFFFF


def build() -> str:
    """Compile the oracle (plain C, OpenMP across queries only)."""
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, U32, U64, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        lib.orc_graph_build.restype = P
        lib.orc_graph_build.argtypes = [U32, U64, P, P, P, P, U32, U32]
        lib.orc_graph_free.argtypes = [P]
        lib.orc_graph_num_edges.restype = U64
        lib.orc_graph_num_edges.argtypes = [P]
        lib.orc_mix64.restype = U64
        lib.orc_mix64.argtypes = [U64]
        lib.orc_row_hash.restype = U64
        lib.orc_row_hash.argtypes = [U32, P]
        lib.orc_fingerprint.restype = U64
        lib.orc_fingerprint.argtypes = [U32, P, U64]
        lib.orc_match.restype = I
        lib.orc_match.argtypes = [P, U32, U32, P, P, P, P, P, U64, P, P, P, P, ctypes.c_double]
        lib.orc_match_proj.restype = I
        lib.orc_match_proj.argtypes = [P, U32, U32, P, P, P, P, P, U32, U64, P, P, P, P, P, ctypes.c_double]
        lib.orc_match_many.restype = I
        lib.orc_match_many.argtypes = [P, U32, P, P, P, P, P, P, P, P, P, I, ctypes.c_double, P, P, P]
        lib.orc_brute.restype = I
        lib.orc_brute.argtypes = [P, U32, U32, P, P, P, P, P, U64, P, P, P, P]
        lib.orc_candidates.restype = I
        lib.orc_candidates.argtypes = [P, U32, U32, P, P, P, P, P, I, P]
        lib.orc_refine.restype = I
        lib.orc_refine.argtypes = [P, U32, U32, P, P, P, P, P, P]
        lib.orc_edge_table.restype = I
        lib.orc_edge_table.argtypes = [P, U32, U32, P, P, P, P, U32, I, P, P, P, P, P]
        lib.orc_khop.restype = I
        lib.orc_khop.argtypes = [P, P, U32, U32, U32, P, P, P]
        lib.orc_compress.restype = P
        lib.orc_compress.argtypes = [P, U32, P]
        lib.orc_wgraph_free.argtypes = [P]
        lib.orc_wgraph_nodes.restype = U32
        lib.orc_wgraph_nodes.argtypes = [P]
        lib.orc_wgraph_edges.restype = U64
        lib.orc_wgraph_edges.argtypes = [P]
        lib.orc_wgraph_get.restype = None
        lib.orc_wgraph_get.argtypes = [P] + [P] * 10
        lib.orc_wcandidates.restype = I
        lib.orc_wcandidates.argtypes = [P, U32, U32, P, P, P, P, P, P]
        lib.orc_wrefine.restype = I
        lib.orc_wrefine.argtypes = [P, U32, U32, P, P, P, P]
        lib.orc_match_compressed.restype = I
        lib.orc_match_compressed.argtypes = [P, P, U32, U32, P, P, P, P, P, U64, P, P, P, P, P]
        lib.orc_verify.restype = ctypes.c_int64
        lib.orc_verify.argtypes = [P, U32, U32, P, P, P, P, P, P, U64]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


class OracleGraph:
    """The oracle's own copy of a data graph (triples sorted and de-duplicated)."""

    def __init__(self, num_vertices, row_offsets, col_targets, edge_rel, vertex_type, num_types, num_rels):
        lib = _load()
        self.V = int(num_vertices)
        self.T = int(num_types)
        self.R = int(num_rels)
        ro = np.ascontiguousarray(np.asarray(row_offsets, dtype=np.uint64))
        col, rel, vt = _u32(col_targets), _u32(edge_rel), _u32(vertex_type)
        self._h = lib.orc_graph_build(self.V, int(ro[-1]), _p(ro), _p(col), _p(rel), _p(vt), self.T, self.R)
        self.E = int(lib.orc_graph_num_edges(self._h))

    @classmethod
    def from_graph(cls, g):
        return cls(g.num_vertices, g.row_offsets, g.col_targets, g.edge_rel, g.vertex_type, g.num_types,
                   g.num_rels)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_graph_free(self._h)
            self._h = None


def _q(q):
    vt, vb = _u32(q.vtype), _u32(q.vbind)
    es, ed, er = _u32(q.esrc), _u32(q.edst), _u32(q.erel)
    return vt, vb, es, ed, er


class Result:
    def __init__(self, status, count, fingerprint, rows, truncated=None):
        self.status = status  # 0 ok, 1 invalid query, 2 time-out
        self.count = count
        self.fingerprint = fingerprint
        self.rows = rows      # uint32 [nrows, w], lexicographically ascending
        self.truncated = truncated  # more distinct rows than returned


def project_mask(project) -> int:
    """Bit mask of projected query vertices from a mask or a vertex list."""
    if project is None:
        return 0
    if isinstance(project, (int, np.integer)):
        return int(project)
    m = 0
    for u in project:
        m |= 1 << int(u)
    return m


def match(g: OracleGraph, q, cap: int = 1 << 20, time_limit_s: float = 0.0, project=None) -> Result:
    """Every embedding (count, fingerprint) and the smallest `cap` distinct
    rows over the projected vertices (all vertices when project is None)."""
    lib = _load()
    vt, vb, es, ed, er = _q(q)
    k = vt.shape[0]
    pm = project_mask(project)
    w = k if pm == 0 else bin(pm & ((1 << k) - 1)).count("1")
    cnt, fp, nr, tr = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint32()
    rows = np.zeros((max(cap, 0), w), np.uint32) if cap else np.zeros((0, w), np.uint32)
    st = lib.orc_match_proj(g._h, k, es.shape[0], _p(vt), _p(vb), _p(es), _p(ed), _p(er), pm, cap,
                            ctypes.byref(cnt), ctypes.byref(fp), _p(rows) if cap else None, ctypes.byref(nr),
                            ctypes.byref(tr), time_limit_s)
    return Result(st, cnt.value, fp.value, rows[: nr.value].copy(), bool(tr.value))


def match_many(g: OracleGraph, queries, threads: int = 0, time_limit_s: float = 0.0):
    """Counts and fingerprints for many queries on `threads` OpenMP threads.
    Returns (count[n], fingerprint[n], status[n], threads_used)."""
    lib = _load()
    n = len(queries)
    qk = np.array([q.k for q in queries], np.uint32)
    qm = np.array([q.m for q in queries], np.uint32)
    voff = np.zeros(n, np.uint64)
    eoff = np.zeros(n, np.uint64)
    if n:
        voff[1:] = np.cumsum(qk[:-1], dtype=np.uint64)
        eoff[1:] = np.cumsum(qm[:-1], dtype=np.uint64)
    cat = lambda f: _u32(np.concatenate([np.asarray(getattr(q, f), np.uint32) for q in queries] + [np.zeros(1, np.uint32)]))
    vt, vb, es, ed, er = cat("vtype"), cat("vbind"), cat("esrc"), cat("edst"), cat("erel")
    cnt = np.zeros(n, np.uint64)
    fp = np.zeros(n, np.uint64)
    st = np.zeros(n, np.int32)
    used = lib.orc_match_many(g._h, n, _p(qk), _p(qm), _p(voff), _p(eoff), _p(vt), _p(vb), _p(es), _p(ed), _p(er),
                              threads, time_limit_s, _p(cnt), _p(fp), _p(st))
    return cnt, fp, st, used


def brute(g: OracleGraph, q, cap: int = 1 << 20) -> Result:
    """Every injective map tried in lexicographic order (tiny graphs only)."""
    lib = _load()
    vt, vb, es, ed, er = _q(q)
    k = vt.shape[0]
    cnt, fp, nr = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    rows = np.zeros((max(cap, 1), k), np.uint32)
    st = lib.orc_brute(g._h, k, es.shape[0], _p(vt), _p(vb), _p(es), _p(ed), _p(er), cap, ctypes.byref(cnt),
                       ctypes.byref(fp), _p(rows), ctypes.byref(nr))
    return Result(st, cnt.value, fp.value, rows[: nr.value].copy())


def candidates(g: OracleGraph, q, signature: bool = True) -> np.ndarray:
    """C0: bool [k, V] (binding, type and, with signature, the per-direction,
    per-relation degree test)."""
    lib = _load()
    vt, vb, es, ed, er = _q(q)
    k = vt.shape[0]
    out = np.zeros((k, g.V), np.uint8)
    st = lib.orc_candidates(g._h, k, es.shape[0], _p(vt), _p(vb), _p(es), _p(ed), _p(er), 1 if signature else 0,
                            _p(out))
    if st:
        raise ValueError("invalid query")
    return out.astype(bool)


def refine(g: OracleGraph, q, sets: np.ndarray) -> tuple[np.ndarray, int]:
    """Prune `sets` (bool [k, V]) until no candidate lacks support on some
    query edge.  Returns (fixpoint sets, number of passes)."""
    lib = _load()
    vt, vb, es, ed, er = _q(q)
    s = np.ascontiguousarray(sets.astype(np.uint8))
    passes = lib.orc_refine(g._h, vt.shape[0], es.shape[0], _p(vt), _p(vb), _p(es), _p(ed), _p(er), _p(s))
    if passes < 0:
        raise ValueError("invalid query")
    return s.astype(bool), passes


def fixpoint(g: OracleGraph, q) -> np.ndarray:
    """Candidate sets after refinement to a fixpoint, starting from C0."""
    return refine(g, q, candidates(g, q, True))[0]


def edge_table(g: OracleGraph, q, sets: np.ndarray, e: int, from_src: bool):
    """Candidate edges of query edge e: (keys, off, vals)."""
    lib = _load()
    es, ed, er = _u32(q.esrc), _u32(q.edst), _u32(q.erel)
    s = np.ascontiguousarray(sets.astype(np.uint8))
    nk, nv = ctypes.c_uint64(), ctypes.c_uint64()
    k = sets.shape[0]
    st = lib.orc_edge_table(g._h, k, es.shape[0], _p(es), _p(ed), _p(er), _p(s), e, 1 if from_src else 0, None,
                            None, None, ctypes.byref(nk), ctypes.byref(nv))
    if st:
        raise ValueError("invalid edge")
    keys = np.zeros(max(nk.value, 1), np.uint32)
    off = np.zeros(nk.value + 1, np.uint64)
    vals = np.zeros(max(nv.value, 1), np.uint32)
    lib.orc_edge_table(g._h, k, es.shape[0], _p(es), _p(ed), _p(er), _p(s), e, 1 if from_src else 0, _p(keys),
                       _p(off), _p(vals), ctypes.byref(nk), ctypes.byref(nv))
    return keys[: nk.value], off, vals[: nv.value]


def verify(g: OracleGraph, q, rows: np.ndarray) -> int:
    """Index of the first row that is not an embedding, or -1."""
    lib = _load()
    vt, vb, es, ed, er = _q(q)
    r = np.ascontiguousarray(np.asarray(rows, np.uint32).reshape(-1, vt.shape[0]))
    return int(lib.orc_verify(g._h, vt.shape[0], es.shape[0], _p(vt), _p(vb), _p(es), _p(ed), _p(er), _p(r),
                              r.shape[0]))


def row_hash(row) -> int:
    lib = _load()
    r = _u32(row)
    return int(lib.orc_row_hash(r.shape[0], _p(r)))


def mix64(z: int) -> int:
    """The splitmix64 finaliser the row hash is built from."""
    return int(_load().orc_mix64(z & 0xFFFFFFFFFFFFFFFF))


def fingerprint(rows: np.ndarray) -> int:
    """Sum (mod 2^64) of row_hash over rows [n, k]."""
    r = np.ascontiguousarray(np.asarray(rows, np.uint32))
    if r.ndim != 2 or r.shape[0] == 0:
        return 0
    return int(_load().orc_fingerprint(r.shape[1], _p(r), r.shape[0]))


def relmask(rels=None) -> np.ndarray:
    """256-bit relation mask (8 uint32 words): every relation when None."""
    m = np.zeros(8, np.uint32)
    if rels is None:
        m[:] = 0xFFFFFFFF
    else:
        for r in rels:
            m[int(r) >> 5] |= np.uint32(1 << (int(r) & 31))
    return m


def khop(g: OracleGraph, seeds, levels: int, dirs: int = 3, rels=None):
    """Domain-graph exploration: (status, level[V] uint8 with 255 = not
    reached, counts[levels + 1])."""
    lib = _load()
    s = _u32(seeds)
    lv = np.zeros(g.V, np.uint8)
    cnt = np.zeros(levels + 1, np.uint64)
    st = lib.orc_khop(g._h, _p(s), s.shape[0], levels, dirs, _p(relmask(rels)), _p(lv), _p(cnt))
    return st, lv, cnt


class WeightedGraph:
    """The oracle's multi-level compression of a graph (Section 3.4): the
    weighted graph, its mapping lists and its weights, as numpy arrays."""

    def __init__(self, g: OracleGraph, deltas):
        lib = _load()
        d = np.ascontiguousarray(np.asarray(list(deltas), np.float64))
        self.g = g
        self.levels = d.shape[0]
        self._h = lib.orc_compress(g._h, self.levels, _p(d) if self.levels else None)
        self.n = int(lib.orc_wgraph_nodes(self._h))
        self.ne = int(lib.orc_wgraph_edges(self._h))
        V, n, ne, R = g.V, self.n, self.ne, g.R
        self.group = np.zeros(V, np.uint32)
        self.moff = np.zeros(n + 1, np.uint32)
        self.mem = np.zeros(V, np.uint32)
        self.type = np.zeros(max(n, 1), np.uint32)
        self.src, self.rel, self.dst = (np.zeros(max(ne, 1), np.uint32) for _ in range(3))
        self.wout, self.win = np.zeros(max(ne, 1), np.uint32), np.zeros(max(ne, 1), np.uint32)
        self.wnode = np.zeros(max(2 * R * n, 1), np.uint32)
        lib.orc_wgraph_get(self._h, _p(self.group), _p(self.moff), _p(self.mem), _p(self.type), _p(self.src),
                           _p(self.rel), _p(self.dst), _p(self.wout), _p(self.win), _p(self.wnode))
        self.type, self.src, self.rel, self.dst = self.type[:n], self.src[:ne], self.rel[:ne], self.dst[:ne]
        self.wout, self.win = self.wout[:ne], self.win[:ne]
        self.wnode = self.wnode[: 2 * R * n].reshape(2, R, n)

    def ratio(self) -> float:
        """(nodes + edges) of the weighted graph over (vertices + edges) of the
        data graph; an edge inside a node counts once per relation."""
        inner = int((self.wnode[0] > 0).sum())
        return (self.n + self.ne + inner) / (self.g.V + self.g.E)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_wgraph_free(self._h)
            self._h = None


def wcandidates(w: WeightedGraph, q) -> np.ndarray:
    """Definition 3.5 on the weighted graph: bool [k, n]."""
    lib = _load()
    vt, vb, es, ed, er = _q(q)
    out = np.zeros((vt.shape[0], max(w.n, 1)), np.uint8)
    if lib.orc_wcandidates(w._h, vt.shape[0], es.shape[0], _p(vt), _p(vb), _p(es), _p(ed), _p(er), _p(out)):
        raise ValueError("invalid query")
    return out[:, : w.n].astype(bool)


def wrefine(w: WeightedGraph, q, sets: np.ndarray) -> np.ndarray:
    """The refinement rule on the weighted graph, to its fixpoint."""
    lib = _load()
    es, ed, er = _u32(q.esrc), _u32(q.edst), _u32(q.erel)
    s = np.ascontiguousarray(sets.astype(np.uint8))
    if lib.orc_wrefine(w._h, s.shape[0], es.shape[0], _p(es), _p(ed), _p(er), _p(s)) < 0:
        raise ValueError("invalid query")
    return s.astype(bool)


def match_compressed(g: OracleGraph, w: WeightedGraph, q, cap: int = 1 << 20):
    """Embeddings found through the weighted graph and the mapping lists:
    (Result, number of weighted-graph solutions)."""
    lib = _load()
    vt, vb, es, ed, er = _q(q)
    k = vt.shape[0]
    cnt, fp, nr, homs = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    rows = np.zeros((max(cap, 1), k), np.uint32)
    st = lib.orc_match_compressed(g._h, w._h, k, es.shape[0], _p(vt), _p(vb), _p(es), _p(ed), _p(er), cap,
                                  ctypes.byref(cnt), ctypes.byref(fp), _p(rows) if cap else None, ctypes.byref(nr),
                                  ctypes.byref(homs))
    return Result(st, cnt.value, fp.value, rows[: nr.value].copy()), homs.value
