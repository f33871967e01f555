"""Small graph/query builders shared by the tests (input construction only)."""
from __future__ import annotations

import itertools
import os

import numpy as np

from paper_1807_08804_gb300.inputs import ANY, UNBOUND, Graph, Query

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def graph_from_triples(V: int, triples, vtype=None, T: int = 1, R: int = 1) -> Graph:
    """Out-CSR from (src, rel, dst) triples (kept in the given order)."""
    triples = list(triples)
    ro = np.zeros(V + 1, np.uint64)
    by = [[] for _ in range(V)]
    for s, r, d in triples:
        by[s].append((r, d))
    col, rel = [], []
    for s in range(V):
        ro[s + 1] = ro[s] + len(by[s])
        for r, d in by[s]:
            rel.append(r)
            col.append(d)
    vt = np.zeros(V, np.uint32) if vtype is None else np.asarray(vtype, np.uint32)
    return Graph(V, ro, np.asarray(col, np.uint32), np.asarray(rel, np.uint32), vt, T, R)


def query(k, edges, vtype=None, vbind=None) -> Query:
    """edges: (src, dst, rel) triples over query vertices 0..k-1."""
    vt = np.full(k, ANY, np.uint32) if vtype is None else np.asarray(vtype, np.uint32)
    vb = np.full(k, UNBOUND, np.uint32) if vbind is None else np.asarray(vbind, np.uint32)
    e = np.asarray(list(edges), np.uint32).reshape(-1, 3)
    return Query(vt, vb, e[:, 0].copy(), e[:, 1].copy(), e[:, 2].copy())


def random_tiny(rng: np.random.Generator, n_max=7, k_max=5, p_any=0.0):
    """A tiny random instance: dense multi-relation digraph + random query;
    each query edge becomes a variable edge (relation ANY) with p_any."""
    V = int(rng.integers(2, n_max + 1))
    T = int(rng.integers(1, 4))
    R = int(rng.integers(1, 4))
    p = float(rng.uniform(0.2, 0.9))
    triples = [(s, r, d) for s in range(V) for d in range(V) for r in range(R) if s != d and rng.random() < p]
    if rng.random() < 0.3 and triples:  # repeated triples must not change results
        triples = triples + [triples[int(rng.integers(len(triples)))]]
    vt = rng.integers(0, T, V)
    g = graph_from_triples(V, triples, vt, T, R)
    k = int(rng.integers(1, min(k_max, V) + 1))
    edges = []
    for i in range(1, k):  # connected: each vertex attaches to an earlier one
        j = int(rng.integers(0, i))
        edges.append((j, i, int(rng.integers(R))) if rng.random() < 0.5 else (i, j, int(rng.integers(R))))
    for _ in range(int(rng.integers(0, 3))):
        if k >= 2:
            a, b = rng.choice(k, 2, replace=False)
            edges.append((int(a), int(b), int(rng.integers(R))))
    qt = [int(rng.integers(T)) if rng.random() < 0.6 else ANY for _ in range(k)]
    qb = [int(rng.integers(V)) if rng.random() < 0.15 else UNBOUND for _ in range(k)]
    if p_any > 0:
        edges = [(a, b, ANY if rng.random() < p_any else r) for a, b, r in edges]
    return g, query(k, edges, qt, qb)


def connected_random_query(rng, k, R=1, extra=0):
    edges = []
    for i in range(1, k):
        j = int(rng.integers(0, i))
        edges.append((j, i, int(rng.integers(R))) if rng.random() < 0.5 else (i, j, int(rng.integers(R))))
    for _ in range(extra):
        a, b = rng.choice(k, 2, replace=False)
        edges.append((int(a), int(b), int(rng.integers(R))))
    return edges


def edge_sets(g: Graph):
    """(triples, pairs): the set of (src, rel, dst) data triples and the set
    of (src, dst) pairs joined by an edge of any relation."""
    E = set()
    for s in range(g.num_vertices):
        for e in range(int(g.row_offsets[s]), int(g.row_offsets[s + 1])):
            E.add((s, int(g.edge_rel[e]), int(g.col_targets[e])))
    return E, {(a, b) for a, _, b in E}


def _keeps(g, q, E, P, f):
    """Does the vertex map f keep bindings, types and every query edge (a
    variable edge, relation ANY, needs an edge of any relation)?"""
    ok = all((q.vbind[u] == UNBOUND or f[u] == q.vbind[u]) and (q.vtype[u] == ANY or g.vertex_type[f[u]] == q.vtype[u])
             for u in range(q.k))
    return ok and all(((f[a], f[b]) in P) if r == ANY else ((f[a], int(r), f[b]) in E)
                      for a, b, r in zip(q.esrc, q.edst, q.erel))


def python_brute(g: Graph, q: Query):
    """Every embedding (injective map keeping bindings, types and edges) in
    lexicographic order, found by trying every injective map in Python."""
    E, P = edge_sets(g)
    return [f for f in itertools.permutations(range(g.num_vertices), q.k) if _keeps(g, q, E, P, f)]


def homomorphism_projections(g: Graph, q: Query):
    """Sets {f(u)} over every map f (injective or not) that keeps bindings,
    types and all query edges: computed by trying every map."""
    V, k = g.num_vertices, q.k
    E, P = edge_sets(g)
    out = np.zeros((k, V), bool)
    for f in itertools.product(range(V), repeat=k):
        if _keeps(g, q, E, P, f):
            for u in range(k):
                out[u, f[u]] = True
    return out


def parse_worked_example(path=None):
    path = path or os.path.join(GOLDEN, "worked_example.txt")
    lab = {"A": 0, "B": 1, "C": 2, "D": 3, "E": 4}
    d = {"expect_candidates": {}}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, *toks = line.split()
        if key in ("query_labels", "data_labels"):
            d[key] = {t.split("=")[0]: lab[t.split("=")[1]] for t in toks}
        elif key in ("query_edges", "data_edges"):
            d[key] = [tuple(t.split("-")) for t in toks]
        elif key == "expect_candidates":
            u, vs = toks[0].split("=")
            d[key][u] = sorted(vs.split(","))
        elif key == "expect_match":
            d[key] = dict(t.split("=") for t in toks)
        elif key == "expect_count":
            d[key] = int(toks[0])
    return d


def complete_digraph_triples(n, rel=0):
    return [(s, rel, d) for s in range(n) for d in range(n) if s != d]
