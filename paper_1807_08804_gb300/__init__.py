"""GB300 engine for exact labeled subgraph matching (thesis arXiv:1807.08804,
Ch. 3, the filtering-and-joining method).

This module is a thin ctypes binding over the C ABI in `include/gs.h`
(`libgs.so`, built by `build.py`).  It only marshals arguments: every step of
the matching runs in the library's CUDA kernels.  There is no CPU fallback: if
the library or a CUDA device is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs  # noqa: F401  (seeded input generators)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs.so")

GS_OK, GS_ERR_INVALID, GS_ERR_OOM, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_UNSUPPORTED, GS_ERR_BUSY, GS_ERR_NOT_READY = range(8)
STATUS_NAMES = ["OK", "INVALID", "OOM", "CUDA", "TIMEOUT", "UNSUPPORTED", "BUSY", "NOT_READY"]
UNBOUND = 0xFFFFFFFF
ANY = 0xFFFFFFFF
GS_DEVICE_PTRS = 1
GS_ENUMERATE, GS_COUNT_ONLY, GS_CHUNKED = 0, 1, 2
GS_STAGE_FILTER, GS_STAGE_FIXPOINT = 0, 1
GS_REFINE_OFF, GS_REFINE_REVERSED, GS_REFINE_BASELINE = 1, 2, 4
GS_KHOP_OUT, GS_KHOP_IN = 1, 2
GS_WAIT_WITHHOLD_FIRST_TILE = 1
GS_ROUNDS_NONE = 0xFFFFFFFF
GS_SORT_MERGE_ONLY = 1


def GS_REFINE_LOW(d: int) -> int:
    """Refinement flag: skip query vertices with at most d incident edges."""
    return (int(d) & 0xFF) << 8
NUM_KERNEL_KINDS = 16


class GSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


P = ctypes.c_void_p
U32, U64 = ctypes.c_uint32, ctypes.c_uint64


class GraphDesc(ctypes.Structure):
    _fields_ = [("num_vertices", U32), ("num_edges", U64), ("row_offsets", P), ("col_targets", P),
                ("edge_rel", P), ("vertex_type", P), ("num_types", U32), ("num_rels", U32), ("flags", U32),
                ("cuda_stream", P)]


class QueryDesc(ctypes.Structure):
    _fields_ = [("k", U32), ("m", U32), ("vtype", P), ("vbind", P), ("esrc", P), ("edst", P), ("erel", P)]


# void (*)(const uint32_t *rows_dev, uint64_t num_rows, uint32_t k, uint32_t query, void *user)
ChunkCallback = ctypes.CFUNCTYPE(None, ctypes.c_void_p, U64, U32, U32, ctypes.c_void_p)


class MatchOpts(ctypes.Structure):
    _fields_ = [("cap", U64), ("mode", U32), ("max_refine_rounds", U32), ("chunk_bytes", U64), ("cuda_stream", P),
                ("on_chunk", ChunkCallback), ("user", P), ("project", U32), ("refine", U32)]


class KhopOpts(ctypes.Structure):
    _fields_ = [("levels", U32), ("directions", U32), ("rels", P), ("nrels", U32), ("flags", U32),
                ("cuda_stream", P)]


class ResultDesc(ctypes.Structure):
    _fields_ = [("count", U64), ("num_rows", U64), ("fingerprint", U64), ("k", U32), ("truncated", U32),
                ("rows", ctypes.POINTER(U32)), ("status", U32), ("shared", U32)]


class KernelStats(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p * NUM_KERNEL_KINDS), ("launches", U64 * NUM_KERNEL_KINDS),
                ("ms", ctypes.c_double * NUM_KERNEL_KINDS), ("bytes", U64 * NUM_KERNEL_KINDS)]


class Tuning(ctypes.Structure):
    _fields_ = [("group", U32), ("refine_rounds", U32), ("ms", ctypes.c_double), ("from_cache", U32),
                ("configs_tried", U32), ("join_group", U32), ("reserved", U32)]


class ServeOpts(ctypes.Structure):
    _fields_ = [("budget_bytes", U64), ("slots", U32), ("max_batch", U32), ("queue_depth", U32), ("reserved", U32)]


class CGraphInfo(ctypes.Structure):
    _fields_ = [("levels", U32), ("vertices", U32), ("edges", U64), ("nodes", U32), ("reserved", U32),
                ("weighted_edges", U64), ("inner_edges", U64), ("ratio", ctypes.c_double)]


# Every entry point of include/gs.h with its argument types.
SIGNATURES = {
    "gs_graph_load": (ctypes.c_int, [ctypes.POINTER(GraphDesc), ctypes.POINTER(P)]),
    "gs_graph_free": (None, [P]),
    "gs_graph_num_edges": (U64, [P]),
    "gs_match": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), ctypes.POINTER(MatchOpts), ctypes.POINTER(ResultDesc)]),
    "gs_match_batch": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), U32, ctypes.POINTER(MatchOpts),
                                      ctypes.POINTER(ResultDesc)]),
    "gs_memcpy_d2h": (ctypes.c_int, [P, ctypes.c_void_p, U64]),
    "gs_result_free": (None, [ctypes.POINTER(ResultDesc)]),
    "gs_results_free": (None, [ctypes.POINTER(ResultDesc), U32]),
    "gs_last_error": (ctypes.c_char_p, []),
    "gs_batch_create": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), U32, ctypes.POINTER(MatchOpts), ctypes.POINTER(P)]),
    "gs_batch_run": (ctypes.c_int, [P]),
    "gs_batch_finish": (ctypes.c_int, [P]),
    "gs_batch_fetch": (ctypes.c_int, [P, ctypes.POINTER(ResultDesc)]),
    "gs_batch_join_sizes": (ctypes.c_int, [P, P, P]),
    "gs_results_copy_rows": (ctypes.c_int, [P, U32, P]),
    "gs_khop": (ctypes.c_int, [P, P, U32, ctypes.POINTER(KhopOpts), P, P, P]),
    "gs_batch_destroy": (None, [P]),
    "gs_stats_enable": (ctypes.c_int, [P, ctypes.c_int]),
    "gs_stats_get": (ctypes.c_int, [P, ctypes.POINTER(KernelStats)]),
    "gs_stats_reset": (ctypes.c_int, [P]),
    "gs_stats_busy": (ctypes.c_int, [ctypes.POINTER(P), U32, ctypes.POINTER(ctypes.c_double)]),
    "gs_inspect_candidates": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), U32, P, P, U64, ctypes.POINTER(U64)]),
    "gs_inspect_edge_table": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), U32, U32, P, P, P, U64, U64,
                                             ctypes.POINTER(U64), ctypes.POINTER(U64)]),
    "gs_serve_create": (ctypes.c_int, [P, ctypes.POINTER(ServeOpts), ctypes.POINTER(P)]),
    "gs_serve_submit": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), ctypes.POINTER(MatchOpts), ctypes.POINTER(U64)]),
    "gs_serve_poll": (ctypes.c_int, [P, U64, ctypes.POINTER(ResultDesc), ctypes.POINTER(ctypes.c_double)]),
    "gs_serve_destroy": (ctypes.c_int, [P]),
}
# Entry points beyond include/gs.h's core list, used by tests and the benchmark.
EXTRA_SIGNATURES = {
    "gs_batch_create_waves": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), U32, ctypes.POINTER(MatchOpts), U32,
                                             ctypes.POINTER(P)]),
    "gs_batch_set": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, U32]),
    "gs_batch_counters": (ctypes.c_int, [P, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U64),
                                         ctypes.POINTER(U64)]),
    "gs_graph_io_bytes": (ctypes.c_int, [P, ctypes.POINTER(U64), ctypes.POINTER(U64)]),
    "gs_filter_candidates_static": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), U32, P, U64, P, P]),
    "gs_tune": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), U32, ctypes.POINTER(MatchOpts), ctypes.c_char_p,
                               ctypes.POINTER(Tuning)]),
    "gs_tune_set": (ctypes.c_int, [P, U32, U32]),
    "gs_batch_set_wait": (ctypes.c_int, [P, U32, U32]),
    "gs_batch_set_sort": (ctypes.c_int, [P, U32]),
    "gs_batch_run_all": (ctypes.c_int, [P, U32, P]),
    "gs_graph_export": (ctypes.c_int, [P, U32, P, P, ctypes.POINTER(U64), P]),
    "gs_match_batch_shared": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), U32, ctypes.POINTER(MatchOpts),
                                             ctypes.POINTER(ResultDesc), ctypes.POINTER(P)]),
    "gs_rows_count": (U32, [P]),
    "gs_rows_base": (P, [P, U32]),
    "gs_rows_words": (U64, [P, U32]),
    "gs_rows_release": (None, [P]),
    "gs_compress_host": (ctypes.c_int, [ctypes.POINTER(GraphDesc), U32, P, ctypes.POINTER(U32), ctypes.POINTER(U64),
                                        P, P, P, P, P, P, P]),
    "gs_cgraph_build": (ctypes.c_int, [ctypes.POINTER(GraphDesc), U32, P, ctypes.POINTER(P)]),
    "gs_cgraph_free": (None, [P]),
    "gs_cgraph_get_info": (ctypes.c_int, [P, ctypes.POINTER(CGraphInfo)]),
    "gs_cgraph_export": (ctypes.c_int, [P, P, P, P, P, P, P, P]),
    "gs_cgraph_candidates": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), P, P, U64, ctypes.POINTER(U64)]),
    "gs_match_batch_compressed": (ctypes.c_int, [P, ctypes.POINTER(QueryDesc), U32, ctypes.POINTER(MatchOpts),
                                                 ctypes.POINTER(ResultDesc)]),
    "gs_debug_fail_alloc": (None, [ctypes.c_int64]),
    "gs_debug_fail_serve_wait": (None, [U32]),
}

_lib = None


def build(verbose: bool = False) -> str:
    from .buildlib import build as _build
    return _build(verbose=verbose)


def lib() -> ctypes.CDLL:
    """The loaded engine library.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GSError(GS_ERR_UNSUPPORTED, f"{LIB_PATH} is missing; run paper_1807_08804_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in {**SIGNATURES, **EXTRA_SIGNATURES}.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int):
    if st != GS_OK:
        raise GSError(st, lib().gs_last_error().decode(errors="replace"))


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(P)


_QDESC_DTYPE = np.dtype({"names": ["k", "m", "vtype", "vbind", "esrc", "edst", "erel"],
                         "formats": ["<u4", "<u4", "<u8", "<u8", "<u8", "<u8", "<u8"],
                         "offsets": [0, 4, 8, 16, 24, 32, 40], "itemsize": 48})


class _QueryPack:
    """Queries as an array of gs_query structs over five flat id arrays (built
    with vectorised numpy, no per-query ctypes objects)."""

    def __init__(self, queries):
        n = len(queries)
        cols = ([], [], [], [], [])  # one pass over the queries, one concatenation per field
        for q in queries:
            cols[0].append(q.vtype)
            cols[1].append(q.vbind)
            cols[2].append(q.esrc)
            cols[3].append(q.edst)
            cols[4].append(q.erel)
        ks = np.fromiter(map(len, cols[0]), np.int64, n)
        ms = np.fromiter(map(len, cols[2]), np.int64, n)
        z = np.zeros(1, np.uint32)
        self.flat = [np.ascontiguousarray(np.concatenate(c + [z]).astype(np.uint32, copy=False)) for c in cols]
        voff = np.zeros(n, np.uint64)
        eoff = np.zeros(n, np.uint64)
        if n:
            voff[1:] = np.cumsum(ks[:-1]) * 4
            eoff[1:] = np.cumsum(ms[:-1]) * 4
        d = np.zeros(max(n, 1), _QDESC_DTYPE)
        if n:
            d["k"][:n] = ks
            d["m"][:n] = ms
            for name, arr, o in zip(("vtype", "vbind", "esrc", "edst", "erel"), self.flat,
                                    (voff, voff, eoff, eoff, eoff)):
                d[name][:n] = np.uint64(arr.ctypes.data) + o
        self.desc = d
        self.arr = ctypes.cast(d.ctypes.data, ctypes.POINTER(QueryDesc))


# Lower-level names for callers of the C ABI through lib(): queries packed
# once as gs_query structs over host arrays, match options, chunk callbacks,
# the gs_result layout as a numpy dtype, and the status check.
QueryPack = _QueryPack


def project_mask(project) -> int:
    """Projection as the library's bit mask: None = whole embeddings, an int
    is taken as the mask, else an iterable of query vertices."""
    if project is None:
        return 0
    if isinstance(project, (int, np.integer)):
        return int(project)
    m = 0
    for u in project:
        m |= 1 << int(u)
    return m


def _opts(cap=1 << 20, mode=GS_ENUMERATE, max_refine_rounds=0, chunk_bytes=0, stream=None, on_chunk=None,
          project=None, refine=0) -> MatchOpts:
    o = MatchOpts(cap, mode, max_refine_rounds, chunk_bytes, stream)
    if on_chunk is not None:
        o.on_chunk = on_chunk
    o.project = project_mask(project)
    o.refine = refine
    return o


def match_opts(*a, **kw) -> MatchOpts:
    """gs_match_opts from cap, mode, max_refine_rounds, chunk_bytes, stream,
    on_chunk (a wrapped callback), project and refine."""
    return _opts(*a, **kw)


def _chunk_callback(fn, raw=False):
    """Wrap fn as the library's chunk callback.  By default fn(rows, query)
    gets each chunk copied to a uint32 [n, k] array while the call lasts;
    with raw=True, fn(ptr, n, k, query) gets the device pointer (valid only
    during the call) and nothing is copied.  The wrapper must stay
    referenced until the match call returns."""
    if fn is None:
        return None

    def cb(ptr, n, k, query, user):
        if raw:
            fn(ptr, n, k, query)
            return
        rows = np.empty((n, k), np.uint32)
        if n:
            _check(lib().gs_memcpy_d2h(rows.ctypes.data_as(P), ctypes.c_void_p(ptr), 4 * n * k))
        fn(rows, query)

    return ChunkCallback(cb)


class MatchResult:
    """One query's result: count, fingerprint, rows (uint32 [num_rows, k],
    query-vertex order, ascending), truncated, status.  Results of a batch
    share one host array; each `rows` view is made on first access."""
    __slots__ = ("count", "fingerprint", "truncated", "status", "_rows", "_src")

    def __init__(self, count, fingerprint, rows, truncated, status):
        self.count, self.fingerprint, self.truncated, self.status = count, fingerprint, truncated, status
        self._rows, self._src = rows, None

    @classmethod
    def _view(cls, count, fingerprint, big, o0, o1, nrows, k, truncated, status):
        r = cls.__new__(cls)
        r.count, r.fingerprint, r.truncated, r.status = count, fingerprint, truncated, status
        r._rows, r._src = None, (big, o0, o1, nrows, k)
        return r

    @property
    def rows(self) -> np.ndarray:
        if self._rows is None:
            big, o0, o1, nrows, k = self._src
            self._rows, self._src = big[o0:o1].reshape(nrows, k), None
        return self._rows

    def __repr__(self):
        return (f"MatchResult(count={self.count}, fingerprint={self.fingerprint}, rows={self.rows!r}, "
                f"truncated={self.truncated}, status={self.status})")


def _take(r: ResultDesc) -> MatchResult:
    n, k = int(r.num_rows), int(r.k)
    rows = np.zeros((n, k), np.uint32)
    if n:
        ctypes.memmove(rows.ctypes.data, r.rows, 4 * n * k)
    out = MatchResult(int(r.count), int(r.fingerprint), rows, bool(r.truncated), int(r.status))
    lib().gs_result_free(ctypes.byref(r))
    return out


_RES_DTYPE = np.dtype({"names": ["count", "num_rows", "fingerprint", "k", "truncated", "rows", "status", "shared"],
                       "formats": ["<u8", "<u8", "<u8", "<u4", "<u4", "<u8", "<u4", "<u4"],
                       "offsets": [0, 8, 16, 24, 28, 32, 40, 44], "itemsize": 48})
RES_DTYPE = _RES_DTYPE
chunk_callback = _chunk_callback
check = _check



def _take_all(res, n: int) -> list[MatchResult]:
    """Results of a batch call: one copy of all rows into one array (views per
    query), fields read as a structured array, then one free call."""
    if n == 0:
        return []
    a = np.frombuffer(res, dtype=_RES_DTYPE, count=n)
    nr, ks = a["num_rows"].astype(np.int64), a["k"].astype(np.int64)
    off = np.zeros(n + 1, np.int64)
    np.cumsum(nr * ks, out=off[1:])
    big = np.empty(int(off[-1]), np.uint32)
    _check(lib().gs_results_copy_rows(res, n, big.ctypes.data_as(P)))  # every result's rows, back to back
    offl, nrl, kl = off.tolist(), nr.tolist(), ks.tolist()
    view = MatchResult._view
    out = [view(c, f, big, o0, o1, r, k, t != 0, s)
           for c, f, o0, o1, r, k, t, s in zip(a["count"].tolist(), a["fingerprint"].tolist(), offl, offl[1:], nrl,
                                                kl, a["truncated"].tolist(), a["status"].tolist())]
    lib().gs_results_free(res, n)
    return out


class _RowsBlock:
    """Owner of a row block of gs_match_batch_shared: the block goes back to
    the library when the last array viewing it is gone."""

    def __init__(self, h):
        self._h = h

    def __del__(self):
        try:
            lib().gs_rows_release(self._h)
        except Exception:
            pass


def _take_shared(res, n: int, blk) -> list[MatchResult]:
    """Results of gs_match_batch_shared: shared rows are views of the
    library's page-locked buffers (no copy); rows a result owns are copied
    and freed."""
    if n == 0:
        if blk:
            lib().gs_rows_release(blk)
        return []
    a = np.frombuffer(res, dtype=_RES_DTYPE, count=n)
    nbuf = int(lib().gs_rows_count(blk)) if blk else 0
    owner = _RowsBlock(blk) if blk else None  # the buffers go back with the last view
    bases, arrays = [], []
    for i in range(nbuf):
        base, words = int(lib().gs_rows_base(blk, i) or 0), int(lib().gs_rows_words(blk, i))
        if not words:
            continue
        buf = (ctypes.c_uint32 * words).from_address(base)
        buf._owner = owner
        bases.append(base)
        arrays.append(np.frombuffer(buf, np.uint32))
    order = np.argsort(np.array(bases, np.uint64)) if bases else np.zeros(0, np.int64)
    sorted_bases = np.array(bases, np.uint64)[order] if bases else np.zeros(0, np.uint64)
    nr, ks = a["num_rows"].astype(np.int64), a["k"].astype(np.int64)
    shared = a["shared"].astype(bool) & (nr > 0)
    ptr = a["rows"].astype(np.uint64)
    which = np.searchsorted(sorted_bases, ptr, side="right").astype(np.int64) - 1
    which = np.where(shared, which, 0)
    buf_of = order[which] if len(order) else np.zeros(n, np.int64)
    o0 = np.where(shared, (ptr.astype(np.int64) - sorted_bases[which].astype(np.int64)) // 4
                  if len(order) else 0, 0)
    o1 = o0 + nr * ks
    empty = np.empty(0, np.uint32)
    view = MatchResult._view
    out = [view(c, f, arrays[b] if sh else empty, x0, x1, r, k, t != 0, st)
           for c, f, b, sh, x0, x1, r, k, t, st in zip(a["count"].tolist(), a["fingerprint"].tolist(),
                                                       buf_of.tolist(), shared.tolist(), o0.tolist(), o1.tolist(),
                                                       nr.tolist(), ks.tolist(), a["truncated"].tolist(),
                                                       a["status"].tolist())]
    for i in np.flatnonzero(~a["shared"].astype(bool) & (nr > 0)).tolist():  # rows the result owns
        rows = np.empty(int(nr[i] * ks[i]), np.uint32)
        ctypes.memmove(rows.ctypes.data, int(a["rows"][i]), 4 * rows.shape[0])
        out[i] = MatchResult(out[i].count, out[i].fingerprint, rows.reshape(int(nr[i]), int(ks[i])),
                             out[i].truncated, out[i].status)
    lib().gs_results_free(res, n)  # frees owned rows only
    del owner
    return out


class DeviceGraph:
    """A data graph canonicalised and resident on the current CUDA device."""

    def __init__(self, g=None, *, num_vertices=None, num_edges=None, row_offsets=None, col_targets=None, edge_rel=None,
                 vertex_type=None, num_types=None, num_rels=None, device_ptrs=False, stream=None):
        if g is not None:
            num_vertices, row_offsets, col_targets = g.num_vertices, g.row_offsets, g.col_targets
            edge_rel, vertex_type, num_types, num_rels = g.edge_rel, g.vertex_type, g.num_types, g.num_rels
        self._h = P()
        if device_ptrs:  # device addresses (e.g. tensor.data_ptr()) and an explicit edge count
            d = GraphDesc(int(num_vertices), int(num_edges), row_offsets, col_targets, edge_rel, vertex_type,
                          int(num_types), int(num_rels), GS_DEVICE_PTRS, stream)
            keep = ()
        else:
            ro = np.ascontiguousarray(np.asarray(row_offsets, dtype=np.uint64))
            keep = (ro, _u32(col_targets), _u32(edge_rel), _u32(vertex_type))
            d = GraphDesc(int(num_vertices), int(ro[-1]), *[_ptr(x) for x in keep], int(num_types), int(num_rels),
                          0, stream)
        _check(lib().gs_graph_load(ctypes.byref(d), ctypes.byref(self._h)))
        del keep
        self.num_vertices = int(num_vertices)
        self.num_rels = int(num_rels)

    @property
    def num_edges(self) -> int:
        return int(lib().gs_graph_num_edges(self._h))

    def export(self, plane: int, signatures: bool = False):
        """The canonical CSR plane on the device (0 out, 1 in, 2 out and 3 in
        over distinct neighbours) as (off, adj), and with signatures the
        per-(plane, vertex) degree signatures [2R + 2, V]."""
        off = np.zeros(self.num_vertices + 1, np.uint64)
        n = U64()
        _check(lib().gs_graph_export(self._h, plane, _ptr(off), None, ctypes.byref(n), None))
        adj = np.zeros(max(n.value, 1), np.uint32)
        sig = None
        if signatures:
            R = int(self.num_rels)
            sig = np.zeros((2 * R + 2, self.num_vertices), np.uint8)
        _check(lib().gs_graph_export(self._h, plane, _ptr(off), _ptr(adj), ctypes.byref(n),
                                     _ptr(sig) if sig is not None else None))
        return (off, adj[: n.value], sig) if signatures else (off, adj[: n.value])

    def io_bytes(self) -> tuple[int, int]:
        h, d = U64(), U64()
        _check(lib().gs_graph_io_bytes(self._h, ctypes.byref(h), ctypes.byref(d)))
        return h.value, d.value

    def free(self):
        if self._h:
            lib().gs_graph_free(self._h)
            self._h = P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def match(dg: DeviceGraph, q, cap=1 << 20, mode=GS_ENUMERATE, max_refine_rounds=0, chunk_bytes=0,
          on_chunk=None, project=None, refine=0) -> MatchResult:
    """on_chunk(rows, query): with mode=GS_CHUNKED, called with every chunk
    of embeddings (uint32 [n, k], query-vertex order) as it is produced.
    project: query vertices whose distinct tuples are returned as rows."""
    pack = _QueryPack([q])
    cb = _chunk_callback(on_chunk)
    o = _opts(cap, mode, max_refine_rounds, chunk_bytes, on_chunk=cb, project=project, refine=refine)
    r = ResultDesc()
    _check(lib().gs_match(dg._h, pack.arr, ctypes.byref(o), ctypes.byref(r)))
    return _take(r)


def match_batch(dg: DeviceGraph, queries, cap=1 << 20, mode=GS_ENUMERATE, max_refine_rounds=0,
                chunk_bytes=0, on_chunk=None, raw_chunks=False, project=None, refine=0) -> list[MatchResult]:
    pack = _QueryPack(queries)
    cb = _chunk_callback(on_chunk, raw_chunks)
    o = _opts(cap, mode, max_refine_rounds, chunk_bytes, on_chunk=cb, project=project, refine=refine)
    res = (ResultDesc * max(len(queries), 1))()
    blk = P()
    _check(lib().gs_match_batch_shared(dg._h, pack.arr, len(queries), ctypes.byref(o), res, ctypes.byref(blk)))
    return _take_shared(res, len(queries), blk)


def khop(dg: "DeviceGraph", seeds, levels: int, directions: int = GS_KHOP_OUT | GS_KHOP_IN, rels=None,
         device=None, stream=None):
    """Domain-graph exploration from `seeds`: (level uint8 [V], 255 = not
    reached; counts per level; adjacency entries scanned).  With
    device=(seeds_ptr, nseeds, level_ptr) the seeds and the level array are
    device memory (level is then written there and None is returned for it)."""
    rl = None if rels is None else np.ascontiguousarray(np.asarray(rels, np.uint32))
    o = KhopOpts(levels, directions, rl.ctypes.data if rl is not None else None, 0 if rl is None else rl.shape[0],
                 GS_DEVICE_PTRS if device else 0, stream)
    counts = np.zeros(levels + 1, np.uint64)
    edges = U64()
    if device:
        sp, n, lp = device
        _check(lib().gs_khop(dg._h, ctypes.c_void_p(sp), n, ctypes.byref(o), ctypes.c_void_p(lp),
                             counts.ctypes.data_as(P), ctypes.byref(edges)))
        return None, counts, edges.value
    sd = np.ascontiguousarray(np.asarray(seeds, np.uint32))
    level = np.zeros(dg.num_vertices, np.uint8)
    _check(lib().gs_khop(dg._h, sd.ctypes.data_as(P), sd.shape[0], ctypes.byref(o), level.ctypes.data_as(P),
                         counts.ctypes.data_as(P), ctypes.byref(edges)))
    return level, counts, edges.value


class Batch:
    """A prepared batch (device-resident queries, captured pipeline graph)."""

    def __init__(self, dg: DeviceGraph, queries, cap=1 << 20, mode=GS_ENUMERATE, max_refine_rounds=0, chunk_bytes=0,
                 wave_queries=0, stream=None, on_chunk=None, raw_chunks=False, project=None, refine=0):
        self.dg = dg
        self.n = len(queries)
        self._pack = _QueryPack(queries)
        self._cb = _chunk_callback(on_chunk, raw_chunks)  # kept alive: every finish() may call it
        o = _opts(cap, mode, max_refine_rounds, chunk_bytes, stream, on_chunk=self._cb, project=project,
                  refine=refine)
        self._h = P()
        if wave_queries:
            _check(lib().gs_batch_create_waves(dg._h, self._pack.arr, self.n, ctypes.byref(o), wave_queries,
                                               ctypes.byref(self._h)))
        else:
            _check(lib().gs_batch_create(dg._h, self._pack.arr, self.n, ctypes.byref(o), ctypes.byref(self._h)))

    def configure(self, use_graph=True, group=32, refine_rounds=0):
        _check(lib().gs_batch_set(self._h, 1 if use_graph else 0, group, refine_rounds))

    def set_wait(self, max_polls=0, withhold_first_tile=False):
        """Bound of the prefix scans' look-back waits (0 = default); with
        withhold_first_tile the first tile of every multi-tile scan publishes
        nothing (tests of the timeout path)."""
        _check(lib().gs_batch_set_wait(self._h, max_polls,
                                       GS_WAIT_WITHHOLD_FIRST_TILE if withhold_first_tile else 0))

    def set_sort(self, merge_only=False):
        """Large outputs by the sample sort (default) or, with merge_only,
        by the tile sort and merge passes only."""
        _check(lib().gs_batch_set_sort(self._h, GS_SORT_MERGE_ONLY if merge_only else 0))

    def run(self):
        _check(lib().gs_batch_run(self._h))

    def finish(self):
        _check(lib().gs_batch_finish(self._h))

    def fetch(self) -> list[MatchResult]:
        res = (ResultDesc * max(self.n, 1))()
        _check(lib().gs_batch_fetch(self._h, res))
        return _take_all(res, self.n)

    def join_sizes(self):
        """(words_total, words_peak) per query: partial-embedding words of the
        last finished run over the join levels before the last."""
        tot = np.zeros(max(self.n, 1), np.uint64)
        peak = np.zeros(max(self.n, 1), np.uint64)
        _check(lib().gs_batch_join_sizes(self._h, tot.ctypes.data_as(P), peak.ctypes.data_as(P)))
        return tot[: self.n], peak[: self.n]

    def counters(self) -> dict:
        k, h, d, f = U64(), U64(), U64(), U64()
        _check(lib().gs_batch_counters(self._h, ctypes.byref(k), ctypes.byref(h), ctypes.byref(d), ctypes.byref(f)))
        return {"kernel_launches": k.value, "h2d_bytes": h.value, "d2h_bytes": d.value, "fallback_queries": f.value}

    def stats_enable(self, on=True):
        _check(lib().gs_stats_enable(self._h, 1 if on else 0))

    def stats_reset(self):
        _check(lib().gs_stats_reset(self._h))

    def stats(self) -> dict:
        s = KernelStats()
        _check(lib().gs_stats_get(self._h, ctypes.byref(s)))
        out = {}
        for i in range(NUM_KERNEL_KINDS):
            name = s.name[i].decode() if s.name[i] else ""
            if name:
                out[name] = {"launches": int(s.launches[i]), "ms": float(s.ms[i]), "bytes": int(s.bytes[i])}
        return out

    def close(self):
        if self._h:
            lib().gs_batch_destroy(self._h)
            self._h = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune(dg: DeviceGraph, queries, cap=1 << 20, mode=GS_ENUMERATE, cache_path: str | None = None) -> dict:
    """Pick lanes per work item, the join's lanes per partial row and
    refinement rounds for this graph and query load (gs_tune); later batches
    on the graph use them."""
    pack = _QueryPack(queries)
    o = _opts(cap, mode)
    t = Tuning()
    _check(lib().gs_tune(dg._h, pack.arr, len(queries), ctypes.byref(o),
                         cache_path.encode() if cache_path else None, ctypes.byref(t)))
    return {"group": t.group, "refine_rounds": t.refine_rounds, "ms": t.ms, "from_cache": bool(t.from_cache),
            "configs_tried": t.configs_tried, "join_group": t.join_group}


def tune_set(dg: DeviceGraph, group: int = 0, refine_rounds: int = 0) -> None:
    """Set lanes per work item (4, 8, 16 or 32; 0 = default) and refinement
    rounds (0 = default) for batches created on the graph afterwards."""
    _check(lib().gs_tune_set(dg._h, group, refine_rounds))


def inspect_candidates(dg: DeviceGraph, q, stage=GS_STAGE_FIXPOINT) -> list[np.ndarray]:
    pack = _QueryPack([q])
    k = len(q.vtype)
    off = np.zeros(k + 1, np.uint64)
    n = U64()
    _check(lib().gs_inspect_candidates(dg._h, pack.arr, stage, _ptr(off), None, 0, ctypes.byref(n)))
    ids = np.zeros(max(n.value, 1), np.uint32)
    _check(lib().gs_inspect_candidates(dg._h, pack.arr, stage, _ptr(off), _ptr(ids), ids.shape[0], ctypes.byref(n)))
    return [ids[int(off[u]):int(off[u + 1])].copy() for u in range(k)]


def inspect_edge_table(dg: DeviceGraph, q, e: int, from_src: bool):
    pack = _QueryPack([q])
    nk, nv = U64(), U64()
    _check(lib().gs_inspect_edge_table(dg._h, pack.arr, e, 1 if from_src else 0, None, None, None, 0, 0,
                                       ctypes.byref(nk), ctypes.byref(nv)))
    keys = np.zeros(max(nk.value, 1), np.uint32)
    off = np.zeros(nk.value + 1, np.uint64)
    vals = np.zeros(max(nv.value, 1), np.uint32)
    _check(lib().gs_inspect_edge_table(dg._h, pack.arr, e, 1 if from_src else 0, _ptr(keys), _ptr(off), _ptr(vals),
                                       keys.shape[0], vals.shape[0], ctypes.byref(nk), ctypes.byref(nv)))
    return keys[: nk.value], off, vals[: nv.value]


def compress_host(g, deltas) -> dict:
    """The library's multi-level compression of g, computed on the host
    (no device needed): node of each vertex, weighted edges and weights."""
    d = np.ascontiguousarray(np.asarray(list(deltas), np.float64))
    ro = np.ascontiguousarray(np.asarray(g.row_offsets, dtype=np.uint64))
    keep = (ro, _u32(g.col_targets), _u32(g.edge_rel), _u32(g.vertex_type))
    desc = GraphDesc(int(g.num_vertices), int(ro[-1]), *[_ptr(x) for x in keep], int(g.num_types), int(g.num_rels),
                     0, None)
    n, ne = U32(), U64()
    dp = _ptr(d) if d.shape[0] else None
    R, V, E = int(g.num_rels), int(g.num_vertices), int(ro[-1])
    a = {k: np.zeros(max(E, 1), np.uint32) for k in ("src", "rel", "dst", "wout", "win")}  # bounds: one call
    group = np.zeros(V, np.uint32)
    wnode = np.zeros(max(2 * R * V, 1), np.uint32)
    _check(lib().gs_compress_host(ctypes.byref(desc), d.shape[0], dp, ctypes.byref(n), ctypes.byref(ne), _ptr(group),
                                  _ptr(a["src"]), _ptr(a["rel"]), _ptr(a["dst"]), _ptr(a["wout"]), _ptr(a["win"]),
                                  _ptr(wnode)))
    out = {k: v[: ne.value] for k, v in a.items()}
    out["group"] = group
    out["nodes"] = n.value
    out["wnode"] = wnode[: 2 * R * n.value].reshape(2, R, n.value)
    return out


class CompressedGraph:
    """A data graph and its multi-level compression (Section 3.4), both
    device-resident; queries matched through it give the data graph's
    embeddings (Section 3.5)."""

    def __init__(self, g, deltas):
        d = np.ascontiguousarray(np.asarray(list(deltas), np.float64))
        ro = np.ascontiguousarray(np.asarray(g.row_offsets, dtype=np.uint64))
        keep = (ro, _u32(g.col_targets), _u32(g.edge_rel), _u32(g.vertex_type))
        desc = GraphDesc(int(g.num_vertices), int(ro[-1]), *[_ptr(x) for x in keep], int(g.num_types),
                         int(g.num_rels), 0, None)
        self._h = P()
        self.num_vertices, self.num_rels = int(g.num_vertices), int(g.num_rels)
        _check(lib().gs_cgraph_build(ctypes.byref(desc), d.shape[0], _ptr(d) if d.shape[0] else None,
                                     ctypes.byref(self._h)))
        del keep

    def info(self) -> dict:
        i = CGraphInfo()
        _check(lib().gs_cgraph_get_info(self._h, ctypes.byref(i)))
        return {"levels": i.levels, "vertices": i.vertices, "edges": i.edges, "nodes": i.nodes,
                "weighted_edges": i.weighted_edges, "inner_edges": i.inner_edges, "ratio": i.ratio}

    def export(self) -> dict:
        """The compression: node of each vertex, weighted edges and weights."""
        i = self.info()
        V, n, ne, R = i["vertices"], i["nodes"], i["weighted_edges"], self.num_rels
        a = {k: np.zeros(max(ne, 1), np.uint32) for k in ("src", "rel", "dst", "wout", "win")}
        group = np.zeros(V, np.uint32)
        wnode = np.zeros(max(2 * R * n, 1), np.uint32)
        _check(lib().gs_cgraph_export(self._h, _ptr(group), _ptr(a["src"]), _ptr(a["rel"]), _ptr(a["dst"]),
                                      _ptr(a["wout"]), _ptr(a["win"]), _ptr(wnode)))
        out = {k: v[:ne] for k, v in a.items()}
        out["group"] = group
        out["wnode"] = wnode[: 2 * R * n].reshape(2, R, n)
        return out

    def candidates(self, q) -> list[np.ndarray]:
        """Weighted-graph candidate sets of q after refinement to the fixpoint."""
        pack = _QueryPack([q])
        k = len(q.vtype)
        off = np.zeros(k + 1, np.uint64)
        n = U64()
        _check(lib().gs_cgraph_candidates(self._h, pack.arr, _ptr(off), None, 0, ctypes.byref(n)))
        ids = np.zeros(max(n.value, 1), np.uint32)
        _check(lib().gs_cgraph_candidates(self._h, pack.arr, _ptr(off), _ptr(ids), ids.shape[0], ctypes.byref(n)))
        return [ids[int(off[u]):int(off[u + 1])].copy() for u in range(k)]

    def match_batch(self, queries, cap=1 << 20, mode=GS_ENUMERATE, max_refine_rounds=0, project=None,
                    refine=0) -> list[MatchResult]:
        pack = _QueryPack(queries)
        o = _opts(cap, mode, max_refine_rounds, 0, project=project, refine=refine)
        res = (ResultDesc * max(len(queries), 1))()
        _check(lib().gs_match_batch_compressed(self._h, pack.arr, len(queries), ctypes.byref(o), res))
        return _take_all(res, len(queries))

    def free(self):
        if self._h:
            lib().gs_cgraph_free(self._h)
            self._h = P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def run_all(batches, stream=None) -> None:
    """Run several prepared batches at once, each on its own stream, after
    the work queued on `stream`; `stream` then waits for all of them."""
    hs = (P * len(batches))(*[b._h for b in batches])
    _check(lib().gs_batch_run_all(hs, len(batches), stream))


def stats_busy(batches) -> dict:
    """Per kernel kind, the milliseconds during which at least one launch of
    it was running, over the batches' timed runs since their stats resets
    (overlapping launches of batches run together count once)."""
    hs = (P * len(batches))(*[b._h for b in batches])
    busy = (ctypes.c_double * NUM_KERNEL_KINDS)()
    _check(lib().gs_stats_busy(hs, len(batches), busy))
    names = batches[0].stats().keys() if batches else []
    return {name: float(busy[i]) for i, name in enumerate(names)}


def debug_fail_alloc(after: int) -> None:
    """Make the library's device allocation after `after` more succeed
    fail as out-of-memory (one-shot; negative disarms)."""
    lib().gs_debug_fail_alloc(after)


def debug_fail_serve_wait(n: int) -> None:
    """Make the serving worker's next n completion checks report a CUDA error."""
    lib().gs_debug_fail_serve_wait(n)


class Server:
    """Continuous-batching request loop over a device-resident graph
    (gs_serve_*): submit queries, poll results by ticket."""

    def __init__(self, dg: DeviceGraph, budget_bytes=0, slots=0, max_batch=0, queue_depth=0):
        self.dg = dg
        o = ServeOpts(budget_bytes, slots, max_batch, queue_depth, 0)
        self._h = P()
        _check(lib().gs_serve_create(dg._h, ctypes.byref(o), ctypes.byref(self._h)))

    def submit(self, q, cap=1 << 20, mode=GS_ENUMERATE, max_refine_rounds=0, project=None) -> int:
        pack = _QueryPack([q])
        o = _opts(cap, mode, max_refine_rounds, 0, project=project)
        t = U64()
        _check(lib().gs_serve_submit(self._h, pack.arr, ctypes.byref(o), ctypes.byref(t)))
        return t.value

    def submit_packed(self, pack: "_QueryPack", i: int, cap=1 << 20, mode=GS_ENUMERATE) -> int:
        """Submit query i of a pre-built _QueryPack (no per-call packing)."""
        o = _opts(cap, mode, 0, 0)
        t = U64()
        _check(lib().gs_serve_submit(self._h, ctypes.byref(pack.arr[i]), ctypes.byref(o), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """(MatchResult, latency_s) when done, else None."""
        r = ResultDesc()
        lat = ctypes.c_double()
        st = lib().gs_serve_poll(self._h, ticket, ctypes.byref(r), ctypes.byref(lat))
        if st == GS_ERR_NOT_READY:
            return None
        _check(st)
        return _take(r), lat.value

    def close(self):
        if self._h:
            lib().gs_serve_destroy(self._h)
            self._h = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
