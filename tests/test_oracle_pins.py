"""Pins for the CPU oracle: each check comes from somewhere other than the
oracle's own code (brute force, closed-form counts, homomorphism projections,
the thesis's worked example, planted mistakes)."""
import os
from math import comb, perm

import numpy as np
import pytest

import oracle as O
from paper_1807_08804_gb300.inputs import ANY, UNBOUND
from tests.helpers import (connected_random_query, edge_sets, graph_from_triples, homomorphism_projections,
                           parse_worked_example, python_brute, query, random_tiny)


def og(g):
    return O.OracleGraph.from_graph(g)


# ----------------------------------------------------------- brute force
def test_backtracking_equals_brute_force_2000_cases():
    """Definition 3.2 (injective, edges and labels kept) read for directed,
    relation-labelled graphs: backtracking == every injective map tried."""
    rng = np.random.default_rng(12345)
    nonzero = 0
    for case in range(2000):
        g, q = random_tiny(rng)
        o = og(g)
        a = O.match(o, q, cap=1 << 16)
        b = O.brute(o, q, cap=1 << 16)
        assert a.status == 0 and b.status == 0
        assert a.count == b.count, case
        assert a.fingerprint == b.fingerprint, case
        np.testing.assert_array_equal(a.rows, b.rows)
        nonzero += a.count > 0
    assert nonzero > 300  # the cases are not all trivially empty


def test_cap_keeps_lexicographically_smallest_rows():
    rng = np.random.default_rng(7)
    for _ in range(200):
        g, q = random_tiny(rng)
        o = og(g)
        full = O.brute(o, q, cap=1 << 16)
        for cap in (1, 2, 5):
            t = O.match(o, q, cap=cap)
            assert t.count == full.count and t.fingerprint == full.fingerprint
            np.testing.assert_array_equal(t.rows, full.rows[:cap])


# ----------------------------------------------------------- closed forms
def complete_digraph(n, T=1, types=None):
    return graph_from_triples(n, [(s, 0, d) for s in range(n) for d in range(n) if s != d], types, T, 1)


@pytest.mark.parametrize("n,k", [(6, 1), (6, 3), (7, 4), (8, 5), (9, 4)])
def test_complete_digraph_counts(n, k):
    """K_n (every ordered pair, one relation): any connected k-vertex query
    has n!/(n-k)! embeddings; with one bound vertex (n-1)!/(n-k)!."""
    rng = np.random.default_rng(n * 100 + k)
    o = og(complete_digraph(n))
    for extra in (0, 2):
        edges = connected_random_query(rng, k, 1, extra if k > 1 else 0)
        assert O.match(o, query(k, edges), cap=0).count == perm(n, k)
        vb = [UNBOUND] * k
        vb[int(rng.integers(k))] = int(rng.integers(n))
        assert O.match(o, query(k, edges, vbind=vb), cap=0).count == perm(n - 1, k - 1)


def test_typed_complete_digraph_counts():
    """Typed K_n: types of sizes n_t, query with c_t vertices of type t:
    prod_t n_t!/(n_t-c_t)!."""
    sizes = [3, 4, 2]
    types = sum([[t] * s for t, s in enumerate(sizes)], [])
    o = og(complete_digraph(sum(sizes), T=3, types=types))
    rng = np.random.default_rng(3)
    for _ in range(20):
        k = int(rng.integers(2, 6))
        qt = [int(x) for x in rng.integers(0, 3, k)]
        want = 1
        for t, s in enumerate(sizes):
            want *= perm(s, qt.count(t)) if qt.count(t) <= s else 0
        edges = connected_random_query(rng, k, 1, 1)
        assert O.match(o, query(k, edges, vtype=qt), cap=0).count == want


def transitive_tournament(n):
    return graph_from_triples(n, [(i, 0, j) for i in range(n) for j in range(n) if i < j])


@pytest.mark.parametrize("n,k", [(7, 3), (9, 4), (10, 5)])
def test_transitive_tournament_direction(n, k):
    """Edges i->j iff i<j: a directed k-path and a transitive k-clique both
    give C(n,k); a directed k-cycle gives 0 (ignoring direction would give
    n!/(n-k)! for each)."""
    o = og(transitive_tournament(n))
    path = [(i, i + 1, 0) for i in range(k - 1)]
    clique = [(i, j, 0) for i in range(k) for j in range(i + 1, k)]
    cycle = [(i, (i + 1) % k, 0) for i in range(k)]
    assert O.match(o, query(k, path), cap=0).count == comb(n, k)
    assert O.match(o, query(k, clique), cap=0).count == comb(n, k)
    assert O.match(o, query(k, cycle), cap=0).count == 0
    reversed_path = [(i + 1, i, 0) for i in range(k - 1)]
    assert O.match(o, query(k, reversed_path), cap=0).count == comb(n, k)


@pytest.mark.parametrize("c,m", [(3, 4), (2, 5), (4, 3)])
def test_disjoint_cycles(c, m):
    """c disjoint directed m-cycles: a directed k-path (k<=m) gives c*m
    embeddings; a directed m-cycle c*m; a k-cycle with k != m gives 0."""
    tr = [(b * m + i, 0, b * m + (i + 1) % m) for b in range(c) for i in range(m)]
    o = og(graph_from_triples(c * m, tr))
    for k in range(1, m + 1):
        assert O.match(o, query(k, [(i, i + 1, 0) for i in range(k - 1)]), cap=0).count == c * m
    assert O.match(o, query(m, [(i, (i + 1) % m, 0) for i in range(m)]), cap=0).count == c * m
    for k in range(2, m + 3):
        if k != m:
            assert O.match(o, query(k, [(i, (i + 1) % k, 0) for i in range(k)]), cap=0).count == 0


@pytest.mark.parametrize("d,s", [(5, 2), (6, 4), (7, 7), (4, 5)])
def test_out_star(d, s):
    """Hub with d out-leaves: an out-star query with s leaves gives
    d!/(d-s)! (0 when s > d); its in-star mirror gives 0."""
    o = og(graph_from_triples(d + 1, [(0, 0, i) for i in range(1, d + 1)]))
    want = perm(d, s) if s <= d else 0
    assert O.match(o, query(s + 1, [(0, i, 0) for i in range(1, s + 1)]), cap=0).count == want
    assert O.match(o, query(s + 1, [(i, 0, 0) for i in range(1, s + 1)]), cap=0).count == 0


def test_relation_labels_matter():
    """Two relations on the same pairs: a query on relation 1 only sees
    relation-1 edges."""
    tr = [(0, 0, 1), (1, 1, 2), (2, 0, 0), (0, 1, 2)]
    o = og(graph_from_triples(3, tr, R=2))
    assert O.match(o, query(2, [(0, 1, 1)]), cap=0).count == 2   # (1,2), (0,2)
    assert O.match(o, query(2, [(0, 1, 0)]), cap=0).count == 2   # (0,1), (2,0)
    assert O.match(o, query(3, [(0, 1, 0), (1, 2, 1)]), cap=0).count == 1  # 0->1->2


# ------------------------------------------------- variable edges (ANY)
def test_variable_edges_equal_python_brute_force():
    """A query edge with relation ANY (a variable edge) maps onto a data edge
    of any relation; embeddings stay vertex maps, so a pair joined under
    several relations counts once.  The oracle equals a Python enumeration
    of every injective map that uses its own triple and pair sets."""
    rng = np.random.default_rng(808)
    nonzero = wild = 0
    for case in range(400):
        g, q = random_tiny(rng, n_max=6, k_max=4, p_any=0.5)
        o = og(g)
        want = python_brute(g, q)
        r = O.match(o, q, cap=1 << 16)
        assert r.status == 0 and r.count == len(want), case
        np.testing.assert_array_equal(r.rows, np.asarray(want, np.uint32).reshape(-1, q.k))
        assert r.fingerprint == O.fingerprint(r.rows)
        b = O.brute(o, q, cap=1 << 16)
        assert (b.count, b.fingerprint) == (r.count, r.fingerprint)
        nonzero += r.count > 0
        wild += int((q.erel == ANY).any())
    assert nonzero > 100 and wild > 200


def test_variable_edges_on_multi_relation_complete_digraph():
    """K_n where every ordered pair carries a random non-empty set of the
    R relations: any connected query whose edges are all variable gives
    n!/(n-k)! (counting a pair once per relation would give more); with one
    edge fixed to relation r the count drops to what the r-pairs allow."""
    rng = np.random.default_rng(17)
    n, R = 7, 3
    tr = []
    for s_ in range(n):
        for d in range(n):
            if s_ != d:
                rels = [r for r in range(R) if rng.random() < 0.5] or [int(rng.integers(R))]
                tr += [(s_, r, d) for r in rels]
    g = graph_from_triples(n, tr, R=R)
    o = og(g)
    for k in (2, 3, 4, 5):
        for extra in (0, 2):
            edges = [(a, b, ANY) for a, b, _ in connected_random_query(rng, k, 1, extra)]
            assert O.match(o, query(k, edges), cap=0).count == perm(n, k)
    r0 = sum(1 for s_, r, d in tr if r == 0)
    assert O.match(o, query(2, [(0, 1, 0)]), cap=0).count == r0 < perm(n, 2)
    assert O.match(o, query(2, [(0, 1, ANY)]), cap=0).count == perm(n, 2)


def test_variable_edge_is_the_union_over_relations():
    """When every ordered pair carries at most one relation, the embeddings
    with edge e variable are the disjoint union over r of those with e set
    to r, so the counts add up; with pairs that carry two relations the
    variable count is strictly smaller than the sum."""
    rng = np.random.default_rng(23)
    for case in range(60):
        n, R = int(rng.integers(4, 7)), int(rng.integers(2, 4))
        tr = [(a, int(rng.integers(R)), b) for a in range(n) for b in range(n) if a != b and rng.random() < 0.6]
        g = graph_from_triples(n, tr, R=R)
        o = og(g)
        k = int(rng.integers(2, 5))
        edges = connected_random_query(rng, k, R, int(rng.integers(0, 2)))
        j = int(rng.integers(len(edges)))
        with_any = [(a, b, ANY) if i == j else (a, b, r) for i, (a, b, r) in enumerate(edges)]
        total = sum(O.match(o, query(k, [(a, b, rr) if i == j else (a, b, r) for i, (a, b, r) in enumerate(edges)]),
                            cap=0).count for rr in range(R))
        assert O.match(o, query(k, with_any), cap=0).count == total, case
    g = graph_from_triples(3, [(0, 0, 1), (0, 1, 1), (1, 0, 2)], R=2)
    o = og(g)
    assert O.match(o, query(2, [(0, 1, ANY)]), cap=0).count == 2       # (0,1), (1,2)
    assert sum(O.match(o, query(2, [(0, 1, r)]), cap=0).count for r in range(2)) == 3


def test_variable_edge_degree_test_counts_distinct_neighbours():
    """The degree test of a variable edge counts v's distinct neighbours over
    all relations in that direction (counted here from the pair set)."""
    rng = np.random.default_rng(29)
    for _ in range(50):
        g, _ = random_tiny(rng, n_max=7)
        s_ = int(rng.integers(1, 4))
        q = query(s_ + 1, [(0, i, ANY) for i in range(1, s_ + 1)])
        c0 = O.candidates(og(g), q, True)
        _, P = edge_sets(g)
        outs = [sum(1 for a, b in P if a == v) for v in range(g.num_vertices)]
        ins = [sum(1 for a, b in P if b == v) for v in range(g.num_vertices)]
        assert [bool(x) for x in c0[0]] == [outs[v] >= s_ for v in range(g.num_vertices)]
        assert [bool(x) for x in c0[1]] == [ins[v] >= 1 for v in range(g.num_vertices)]


# ------------------------------------------------------------ projection
def test_projection_is_the_distinct_projected_embeddings():
    """Projection (only some query vertices' matches are wanted): the rows
    are the distinct tuples of the projected columns of the embeddings,
    ascending (here from a Python enumeration and numpy's unique), cut at
    cap with `truncated` when more exist; count and fingerprint still cover
    every embedding."""
    rng = np.random.default_rng(606)
    dup = 0
    for case in range(400):
        g, q = random_tiny(rng, n_max=6, k_max=4, p_any=0.2)
        o = og(g)
        full = np.asarray(python_brute(g, q), np.uint32).reshape(-1, q.k)
        cols = [u for u in range(q.k) if rng.random() < 0.5] or [int(rng.integers(q.k))]
        want = np.unique(full[:, cols], axis=0) if len(full) else np.zeros((0, len(cols)), np.uint32)
        dup += len(want) < len(full)
        r = O.match(o, q, cap=1 << 16, project=cols)
        assert (r.count, r.fingerprint) == (len(full), O.fingerprint(full))
        np.testing.assert_array_equal(r.rows, want)
        assert r.truncated is False
        for cap in (1, 2, 3):
            t = O.match(o, q, cap=cap, project=cols)
            np.testing.assert_array_equal(t.rows, want[:cap])
            assert t.truncated == (len(want) > cap) and t.count == len(full)
        a = O.match(o, q, cap=1 << 16, project=list(range(q.k)))
        np.testing.assert_array_equal(a.rows, full)
    assert dup > 40


@pytest.mark.parametrize("n,k", [(7, 3), (8, 4), (9, 5)])
def test_projection_closed_forms(n, k):
    """Complete digraph K_n, directed k-path: the endpoints take every
    ordered pair of distinct vertices (n(n-1) rows), the start every vertex
    (n rows).  Transitive tournament (i->j iff i<j), directed k-path: the
    start takes 0..n-k and the end k-1..n-1 (n-k+1 rows each)."""
    path = query(k, [(i, i + 1, 0) for i in range(k - 1)])
    o = og(complete_digraph(n))
    r = O.match(o, path, cap=1 << 16, project=[0, k - 1])
    assert r.count == perm(n, k) and len(r.rows) == perm(n, 2)
    assert {tuple(x) for x in r.rows} == {(a, b) for a in range(n) for b in range(n) if a != b}
    assert O.match(o, path, cap=1 << 16, project=[0]).rows[:, 0].tolist() == list(range(n))
    t = og(transitive_tournament(n))
    assert O.match(t, path, cap=1 << 16, project=[0]).rows[:, 0].tolist() == list(range(n - k + 1))
    assert O.match(t, path, cap=1 << 16, project=[k - 1]).rows[:, 0].tolist() == list(range(k - 1, n))
    assert O.match(t, path, cap=1 << 16, project=1 << k).status == 1   # vertex out of range


# ----------------------------------------------- domain-graph exploration
def min_plus_distances(g, dirs, rels=None):
    """All-pairs hop distances by repeated min-plus products of the one-hop
    matrix (edges kept by direction and relation), independent of any
    queue-based search."""
    V = g.num_vertices
    INF = 10 ** 6
    A = np.full((V, V), INF, np.int64)
    np.fill_diagonal(A, 0)
    for s_ in range(V):
        for e in range(int(g.row_offsets[s_]), int(g.row_offsets[s_ + 1])):
            r, d = int(g.edge_rel[e]), int(g.col_targets[e])
            if rels is not None and r not in rels:
                continue
            if dirs & 1:
                A[s_, d] = min(A[s_, d], 1)
            if dirs & 2:
                A[d, s_] = min(A[d, s_], 1)
    D = A.copy()
    for _ in range(V):
        D2 = np.minimum(D, (D[:, :, None] + A[None, :, :]).min(axis=1))
        if (D2 == D).all():
            break
        D = D2
    return D


def test_khop_equals_min_plus_distances():
    """Domain-graph exploration (Ch. 5): the level of v is its hop distance
    from the nearest seed when within `levels`, for out-, in- and both
    directions and relation subsets."""
    rng = np.random.default_rng(4040)
    for case in range(150):
        g, _ = random_tiny(rng, n_max=9)
        V = g.num_vertices
        dirs = int(rng.integers(1, 4))
        rels = None if rng.random() < 0.5 else [r for r in range(g.num_rels) if rng.random() < 0.6]
        seeds = [int(x) for x in rng.choice(V, int(rng.integers(1, 3)), replace=True)]
        L = int(rng.integers(0, 5))
        st, lv, cnt = O.khop(og(g), seeds, L, dirs, rels)
        D = min_plus_distances(g, dirs, rels)[seeds].min(axis=0)
        want = np.where(D <= L, D, 255).astype(np.uint8)
        assert st == 0
        np.testing.assert_array_equal(lv, want, err_msg=str(case))
        np.testing.assert_array_equal(cnt, [(want == l).sum() for l in range(L + 1)])


def test_khop_closed_forms():
    """Directed path 0->1->...->9: out from 0 reaches level i at vertex i;
    in from 9 mirrors it; both directions from 5 give |v - 5|.  A directed
    6-cycle out from 0 gives v.  An out-star from its hub reaches every leaf
    at level 1 and nothing in reverse."""
    n = 10
    p = og(graph_from_triples(n, [(i, 0, i + 1) for i in range(n - 1)]))
    assert O.khop(p, [0], 20, 1)[1].tolist() == list(range(n))
    assert O.khop(p, [9], 20, 2)[1].tolist() == list(range(n))[::-1]
    assert O.khop(p, [5], 3, 3)[1].tolist() == [abs(v - 5) if abs(v - 5) <= 3 else 255 for v in range(n)]
    assert O.khop(p, [0], 3, 2)[1].tolist() == [0] + [255] * (n - 1)
    c = og(graph_from_triples(6, [(i, 0, (i + 1) % 6) for i in range(6)]))
    assert O.khop(c, [0], 10, 1)[1].tolist() == list(range(6))
    star = og(graph_from_triples(8, [(0, 0, i) for i in range(1, 8)]))
    assert O.khop(star, [0], 2, 1)[1].tolist() == [0] + [1] * 7
    assert O.khop(star, [0], 2, 2)[1].tolist() == [0] + [255] * 7
    assert O.khop(star, [3], 2, 3)[1].tolist() == [1, 2, 2, 0, 2, 2, 2, 2]
    assert O.khop(star, [8], 2, 3)[0] == 1  # seed out of range


# --------------------------------------------------------- worked example
def test_worked_example():
    """Facts printed for the thesis's sample query/data graph (Section 3.3):
    Definition 3.3 candidates C(u3), C(u1) and the stated match."""
    d = parse_worked_example()
    qn = sorted(d["query_labels"], key=lambda s: int(s[1:]))
    dn = sorted(d["data_labels"], key=lambda s: int(s[1:]))
    qi = {u: i for i, u in enumerate(qn)}
    di = {v: i for i, v in enumerate(dn)}
    tr = []
    for a, b in d["data_edges"]:
        tr += [(di[a], 0, di[b]), (di[b], 0, di[a])]
    g = graph_from_triples(len(dn), tr, [d["data_labels"][v] for v in dn], 5, 1)
    qe = []
    for a, b in d["query_edges"]:
        qe += [(qi[a], qi[b], 0), (qi[b], qi[a], 0)]
    q = query(len(qn), qe, vtype=[d["query_labels"][u] for u in qn])
    o = og(g)
    c0 = O.candidates(o, q, signature=True)
    for u, vs in d["expect_candidates"].items():
        got = sorted(dn[v] for v in np.flatnonzero(c0[qi[u]]))
        assert got == sorted(vs, key=lambda s: int(s[1:])), u
    r = O.match(o, q, cap=16)
    assert r.count == d["expect_count"]
    want = [di[d["expect_match"][u]] for u in qn]
    assert [list(x) for x in r.rows] == [want]


# ------------------------------------------------ filter and refinement
def test_refinement_on_trees_equals_homomorphism_projection():
    """Arc consistency is exact on tree-shaped queries: starting from the
    binding/type sets, the refinement fixpoint equals {f(u)} over all
    (not necessarily injective) edge-preserving maps."""
    rng = np.random.default_rng(99)
    checked = 0
    for case in range(300):
        g, _ = random_tiny(rng, n_max=5, k_max=4)
        k = int(rng.integers(1, 5))
        edges = connected_random_query(rng, k, g.num_rels, 0)  # a tree
        if case >= 150:  # variable edges
            edges = [(a, b, ANY if rng.random() < 0.5 else r) for a, b, r in edges]
        qt = [int(rng.integers(g.num_types)) if rng.random() < 0.5 else ANY for _ in range(k)]
        qb = [int(rng.integers(g.num_vertices)) if rng.random() < 0.15 else UNBOUND for _ in range(k)]
        q = query(k, edges, qt, qb)
        o = og(g)
        start = O.candidates(o, q, signature=False)
        fix, _ = O.refine(o, q, start)
        want = homomorphism_projections(g, q)
        if not want.any():
            # with no homomorphism at all, every set empties (tree case)
            assert not fix.any()
        else:
            np.testing.assert_array_equal(fix, want)
        checked += 1
    assert checked == 300


def test_filter_and_fixpoint_are_sound():
    """Every vertex used by an embedding survives C0 (with the degree test)
    and the refinement fixpoint, on cyclic queries too."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        g, q = random_tiny(rng)
        o = og(g)
        emb = O.brute(o, q, cap=1 << 16)
        c0 = O.candidates(o, q, True)
        fix, _ = O.refine(o, q, c0)
        assert not (fix & ~c0).any()
        for row in emb.rows:
            for u, v in enumerate(row):
                assert c0[u, v] and fix[u, v]


def test_degree_test_is_per_direction_and_relation():
    """Definition 3.3 read per (direction, relation): a query vertex with s
    out-neighbours over relation r admits exactly the data vertices with at
    least s distinct r-out-neighbours (counted here from the triple list)."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        g, _ = random_tiny(rng, n_max=7)
        R = g.num_rels
        s = int(rng.integers(1, 4))
        r = int(rng.integers(R))
        q = query(s + 1, [(0, i, r) for i in range(1, s + 1)])
        c0 = O.candidates(og(g), q, True)
        outs = {}
        for v in range(g.num_vertices):
            a, b = int(g.row_offsets[v]), int(g.row_offsets[v + 1])
            outs[v] = len({int(g.col_targets[e]) for e in range(a, b) if g.edge_rel[e] == r})
        assert [bool(x) for x in c0[0]] == [outs[v] >= s for v in range(g.num_vertices)]
        ins = {v: 0 for v in range(g.num_vertices)}
        seen = set()
        for v in range(g.num_vertices):
            for e in range(int(g.row_offsets[v]), int(g.row_offsets[v + 1])):
                t = (v, int(g.col_targets[e]))
                if g.edge_rel[e] == r and t not in seen:
                    seen.add(t)
                    ins[t[1]] += 1
        assert [bool(x) for x in c0[1]] == [ins[v] >= 1 for v in range(g.num_vertices)]


def test_edge_tables_against_single_edge_matches():
    """Section 3.3.4's candidate edges: for a one-edge query the total table
    size equals the number of embeddings, in both orientations, and every
    embedding's (f(a), f(b)) pair is in the table of any query edge."""
    rng = np.random.default_rng(21)
    for case in range(300):
        g, q = random_tiny(rng, p_any=0.0 if case < 200 else 0.5)
        o = og(g)
        if q.m == 0:
            continue
        fix = O.fixpoint(o, q)
        emb = O.brute(o, q, cap=1 << 16)
        for e in range(q.m):
            a, b = int(q.esrc[e]), int(q.edst[e])
            for from_src in (True, False):
                keys, off, vals = O.edge_table(o, q, fix, e, from_src)
                pairs = set()
                for i, key in enumerate(keys):
                    for v in vals[int(off[i]):int(off[i + 1])]:
                        pairs.add((int(key), int(v)) if from_src else (int(v), int(key)))
                    lst = [int(x) for x in vals[int(off[i]):int(off[i + 1])]]
                    assert lst == sorted(set(lst))  # ascending, each vertex once
                for row in emb.rows:
                    assert (int(row[a]), int(row[b])) in pairs
        # one-edge query: table size == embeddings
        e = 0
        q1 = query(2, [(0, 1, int(q.erel[e]))],
                   vtype=[q.vtype[q.esrc[e]], q.vtype[q.edst[e]]], vbind=[q.vbind[q.esrc[e]], q.vbind[q.edst[e]]])
        f1 = O.fixpoint(o, q1)
        n1 = O.brute(o, q1, cap=0).count
        for from_src in (True, False):
            _, off, _ = O.edge_table(o, q1, f1, 0, from_src)
            assert int(off[-1]) == n1


# ----------------------------------------------------- verifier, fingerprint
def test_verifier_catches_planted_mistakes():
    rng = np.random.default_rng(31)
    caught = 0
    for _ in range(300):
        g, q = random_tiny(rng)
        o = og(g)
        emb = O.brute(o, q, cap=1 << 16)
        assert O.verify(o, q, emb.rows) == -1
        if emb.count == 0:
            continue
        valid = {tuple(r) for r in emb.rows}
        bad = emb.rows[0].copy()
        i = int(rng.integers(q.k))
        bad[i] = (bad[i] + 1 + int(rng.integers(g.num_vertices - 1))) % g.num_vertices
        rows = np.vstack([emb.rows, bad[None]])
        if tuple(bad) in valid:
            assert O.verify(o, q, rows) == -1
        else:
            assert O.verify(o, q, rows) == len(emb.rows)
            caught += 1
    assert caught > 50


def test_fingerprint_is_order_free_sum():
    rng = np.random.default_rng(41)
    for _ in range(100):
        g, q = random_tiny(rng)
        o = og(g)
        r = O.match(o, q, cap=1 << 16)
        perm_rows = r.rows[rng.permutation(len(r.rows))] if len(r.rows) else r.rows
        assert O.fingerprint(perm_rows) == r.fingerprint
        if len(r.rows) >= 2:
            # a changed row changes the fingerprint
            alt = r.rows.copy()
            alt[0, 0] ^= 1
            assert O.fingerprint(alt) != r.fingerprint


def test_invalid_queries_rejected():
    o = og(complete_digraph(4))
    assert O.match(o, query(2, [(0, 0, 0)]), cap=0).status == 1      # self-loop
    assert O.match(o, query(2, [(0, 2, 0)]), cap=0).status == 1      # endpoint out of range
    assert O.match(o, query(2, [(0, 1, 3)]), cap=0).status == 1      # relation out of range
    assert O.match(o, query(2, [(0, 1, 0)], vbind=[9, UNBOUND]), cap=0).status == 1


def test_duplicate_query_edges_and_shared_binding():
    o = og(complete_digraph(5))
    a = O.match(o, query(3, [(0, 1, 0), (1, 2, 0)]), cap=0).count
    b = O.match(o, query(3, [(0, 1, 0), (1, 2, 0), (0, 1, 0)]), cap=0).count
    assert a == b == perm(5, 3)
    assert O.match(o, query(2, [(0, 1, 0)], vbind=[2, 2]), cap=0).count == 0  # injectivity


# ----------------------------------------------------------- fingerprint
GOLDEN_RATIO_64 = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def _splitmix64_golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
    seed, outs = None, []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("seed"):
            seed = int(line.split()[1])
        else:
            outs.append(int(line))
    return seed, outs


def test_mix64_equals_published_splitmix64_outputs():
    """The finaliser under the fingerprint is splitmix64's output function:
    its values at seed + n * golden ratio are the generator's published first
    outputs.  A wrong shift or multiplier constant fails here."""
    seed, outs = _splitmix64_golden()
    assert len(outs) == 5
    for n, want in enumerate(outs, start=1):
        assert O.mix64((seed + n * GOLDEN_RATIO_64) & M64) == want


def test_row_hash_is_the_stated_fold_of_the_pinned_finaliser():
    """h(f) starts at k and folds f(0..k-1) in column order, each step
    h <- mix64(h xor (f(i) + (i+1) * golden ratio)), with mix64 the finaliser
    pinned above."""
    rng = np.random.default_rng(77)
    for _ in range(200):
        k = int(rng.integers(1, 13))
        row = rng.integers(0, 1 << 32, size=k, dtype=np.uint64).astype(np.uint32)
        h = k
        for i, v in enumerate(row.tolist()):
            h = O.mix64(h ^ ((v + (i + 1) * GOLDEN_RATIO_64) & M64))
        assert O.row_hash(row) == h


def test_row_hash_depends_on_column_position_and_width():
    """Swapping two different columns, or appending a column, changes the
    hash: an embedding is a map of query vertices, not a set of data ids."""
    rng = np.random.default_rng(78)
    for _ in range(500):
        k = int(rng.integers(2, 13))
        row = rng.choice(1 << 24, size=k, replace=False).astype(np.uint32)
        i, j = rng.choice(k, size=2, replace=False)
        sw = row.copy()
        sw[[i, j]] = sw[[j, i]]
        assert O.row_hash(sw) != O.row_hash(row)
        assert O.row_hash(np.append(row, np.uint32(0))) != O.row_hash(row)
        assert O.row_hash(row[:-1]) != O.row_hash(row)


def test_fingerprint_sums_row_hashes_mod_2_64():
    rng = np.random.default_rng(79)
    for _ in range(50):
        n, k = int(rng.integers(1, 200)), int(rng.integers(1, 9))
        rows = rng.integers(0, 1 << 32, size=(n, k), dtype=np.uint64).astype(np.uint32)
        assert O.fingerprint(rows) == sum(O.row_hash(r) for r in rows) & M64


@pytest.mark.parametrize("threads", [1, 0])
def test_match_many_equals_match_per_query(threads):
    """The batched oracle entry (used by the large parity tests and the CPU
    baseline) gives per query exactly what orc_match gives: same status,
    count and fingerprint, on one thread and on every host thread."""
    from paper_1807_08804_gb300 import inputs as I
    g = I.make_graph(10_000, 60_000, seed=0x6753001)
    qs = I.make_walk_queries(g, 120, 3, 6, p_bind=0.2, seed=5) + I.make_walk_queries(g, 80, 3, 8, p_bind=0.0,
                                                                                      seed=6)
    o = og(g)
    cnt, fp, st, used = O.match_many(o, qs, threads=threads)
    assert used >= 1 and (threads == 0 or used == threads)
    assert sum(int(c) > 0 for c in cnt) == len(qs)  # every walked query matches itself
    for i, q in enumerate(qs):
        r = O.match(o, q, cap=0)
        assert (int(st[i]), int(cnt[i]), int(fp[i])) == (r.status, r.count, r.fingerprint), i
