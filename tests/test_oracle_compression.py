"""Pins for the oracle's multi-level graph compression (Section 3.4) and its
matching through the weighted graph and the mapping lists (Section 3.5),
each from somewhere other than the oracle's own code: brute force over every
injective map, weights recounted from the triple list, the greedy pairing's
maximality, Theorems 3.1 and 3.2 checked on every embedding, and closed forms
on complete bipartite digraphs."""
import itertools
from math import ceil

import numpy as np
import pytest

import oracle as O
from paper_1807_08804_gb300.inputs import ANY, UNBOUND
from tests.helpers import edge_sets, graph_from_triples, python_brute, query, random_tiny


def twin_tiny(rng):
    """A tiny random graph in which some vertices get twins (a new vertex of
    the same type with the same out- and in-edges), plus a random query:
    graphs where compression has something to merge."""
    V0 = int(rng.integers(2, 6))
    T, R = int(rng.integers(1, 3)), int(rng.integers(1, 3))
    p = float(rng.uniform(0.2, 0.7))
    tr = {(s, r, d) for s in range(V0) for d in range(V0) for r in range(R) if s != d and rng.random() < p}
    vt = list(rng.integers(0, T, V0))
    V = V0
    for v in range(V0):
        if rng.random() < 0.6 and V < 8:
            w = V
            V += 1
            vt.append(vt[v])
            tr |= {(w, r, d) for (s, r, d) in tr if s == v} | {(s, r, w) for (s, r, d) in tr if d == v}
    tr = sorted(tr)
    g = graph_from_triples(V, tr, vt, T, R)
    k = int(rng.integers(1, min(4, V) + 1))
    edges = []
    for i in range(1, k):
        j = int(rng.integers(0, i))
        edges.append((j, i, int(rng.integers(R))) if rng.random() < 0.5 else (i, j, int(rng.integers(R))))
    if k >= 3 and rng.random() < 0.5:
        a, b = rng.choice(k, 2, replace=False)
        edges.append((int(a), int(b), int(rng.integers(R))))
    qt = [int(rng.integers(T)) if rng.random() < 0.5 else ANY for _ in range(k)]
    qb = [int(rng.integers(V)) if rng.random() < 0.1 else UNBOUND for _ in range(k)]
    return g, query(k, edges, qt, qb)


def deltas(rng):
    return [float(rng.choice([1.0, 0.8, 0.5, 0.3])) for _ in range(int(rng.integers(1, 4)))]


def triples_of(g):
    E, _ = edge_sets(g)
    return E


# ------------------------------------------------------------ end to end
@pytest.mark.parametrize("maker", [random_tiny, twin_tiny])
def test_matching_through_weighted_graph_equals_brute_force(maker):
    """Section 3.5: matching on the weighted graph and expanding every
    solution through the mapping lists yields exactly the embeddings of the
    query in the data graph (every injective map tried in Python)."""
    rng = np.random.default_rng(301 if maker is random_tiny else 302)
    merged = 0
    for case in range(1200):
        g, q = maker(rng)
        o = O.OracleGraph.from_graph(g)
        w = O.WeightedGraph(o, deltas(rng))
        merged += w.n < g.num_vertices
        want = python_brute(g, q)
        got, homs = O.match_compressed(o, w, q, cap=1 << 16)
        assert got.status == 0
        assert got.count == len(want), case
        assert [tuple(r) for r in got.rows.tolist()] == want, case
        assert got.fingerprint == (O.fingerprint(np.array(want, np.uint32)) if want else 0)
        assert homs >= (1 if want else 0)
    assert merged > 300  # the cases do compress


def test_no_level_is_the_graph_itself():
    rng = np.random.default_rng(303)
    for _ in range(50):
        g, q = random_tiny(rng)
        o = O.OracleGraph.from_graph(g)
        w = O.WeightedGraph(o, [])
        E = {t for t in triples_of(g) if t[0] != t[2]}
        assert w.n == g.num_vertices and list(w.group) == list(range(g.num_vertices))
        assert set(zip(w.src.tolist(), w.rel.tolist(), w.dst.tolist())) == E
        assert (w.wout == 1).all() and (w.win == 1).all()


# ------------------------------------------------------------ structure
def check_structure(g, w):
    V = g.num_vertices
    E = triples_of(g)
    grp = w.group.tolist()
    # mapping lists partition V, ascending, numbered by smallest member
    lists = [w.mem[w.moff[x]:w.moff[x + 1]].tolist() for x in range(w.n)]
    assert sorted(v for L in lists for v in L) == list(range(V))
    assert all(L == sorted(L) and L for L in lists)
    assert [L[0] for L in lists] == sorted(L[0] for L in lists)
    assert all(grp[v] == x for x, L in enumerate(lists) for v in L)
    # one type per node
    assert all(g.vertex_type[v] == w.type[grp[v]] for v in range(V))
    # edges: the quotient of E between different nodes
    want = {(grp[a], r, grp[b]) for a, r, b in E if grp[a] != grp[b]}
    got = list(zip(w.src.tolist(), w.rel.tolist(), w.dst.tolist()))
    assert set(got) == want and len(got) == len(want) and got == sorted(got)
    # weights bound the neighbour counts they stand for, recounted from E
    for (x, r, y), wo, wi in zip(got, w.wout.tolist(), w.win.tolist()):
        out_max = max(sum((a, r, b) in E for b in lists[y]) for a in lists[x])
        in_max = max(sum((a, r, b) in E for a in lists[x]) for b in lists[y])
        assert 1 <= out_max <= wo and 1 <= in_max <= wi
    # node weights: the largest number of neighbours a member has in its own node
    for d in range(2):
        for r in range(g.num_rels):
            for x, L in enumerate(lists):
                m = max(sum(((a, r, b) if d == 0 else (b, r, a)) in E for b in L) for a in L)
                assert w.wnode[d, r, x] == m


@pytest.mark.parametrize("maker", [random_tiny, twin_tiny])
def test_mapping_lists_edges_and_weights(maker):
    rng = np.random.default_rng(304 if maker is random_tiny else 305)
    for _ in range(400):
        g, _ = maker(rng)
        o = O.OracleGraph.from_graph(g)
        check_structure(g, O.WeightedGraph(o, deltas(rng)))


def adjacency(g, grp, n):
    """(direction, relation, other node) triples of each node's edges to other nodes."""
    adj = [set() for _ in range(n)]
    for a, r, b in triples_of(g):
        x, y = grp[a], grp[b]
        if x != y:
            adj[x].add((0, r, y))
            adj[y].add((1, r, x))
    return adj


def similar(adj, types, x, y, delta):
    if types[x] != types[y]:
        return False
    a, b = len(adj[x]), len(adj[y])
    if a == 0 or b == 0:
        return a == 0 and b == 0
    c = len(adj[x] & adj[y])
    return c >= delta * a and c >= delta * b


def test_one_level_pairs_similar_nodes_greedily():
    """One level: every merged pair is similar (reading of the garbled test:
    common edges make up at least delta of both adjacency lists; with
    delta = 1 the lists are equal), and no two nodes left alone are similar
    to each other (the greedy pass would have paired them)."""
    rng = np.random.default_rng(306)
    for _ in range(400):
        g, _ = twin_tiny(rng)
        delta = float(rng.choice([1.0, 0.5]))
        o = O.OracleGraph.from_graph(g)
        w = O.WeightedGraph(o, [delta])
        V = g.num_vertices
        adj0 = adjacency(g, list(range(V)), V)
        types = [int(t) for t in g.vertex_type]
        lists = [w.mem[w.moff[x]:w.moff[x + 1]].tolist() for x in range(w.n)]
        assert all(len(L) <= 2 for L in lists)
        for L in lists:
            if len(L) == 2:
                assert similar(adj0, types, L[0], L[1], delta)
                if delta == 1.0:
                    assert adj0[L[0]] == adj0[L[1]]
        alone = [L[0] for L in lists if len(L) == 1]
        for a, b in itertools.combinations(alone, 2):
            assert not similar(adj0, types, a, b, delta)


def test_one_level_weights_from_unit_weights():
    """From unit weights, one level gives wout(U, r, V) = the number of
    members of V with an r-in-neighbour in U (the recursion's sum of maxima
    over single-vertex parts), and win(U, r, V) = the members of U with an
    r-out-neighbour in V."""
    rng = np.random.default_rng(307)
    for _ in range(300):
        g, _ = twin_tiny(rng)
        o = O.OracleGraph.from_graph(g)
        w = O.WeightedGraph(o, [float(rng.choice([1.0, 0.5]))])
        E = triples_of(g)
        lists = [w.mem[w.moff[x]:w.moff[x + 1]].tolist() for x in range(w.n)]
        for x, r, y, wo, wi in zip(w.src.tolist(), w.rel.tolist(), w.dst.tolist(), w.wout.tolist(),
                                   w.win.tolist()):
            assert wo == sum(any((a, r, b) in E for a in lists[x]) for b in lists[y])
            assert wi == sum(any((a, r, b) in E for b in lists[y]) for a in lists[x])


# ------------------------------------------------------------ Theorems 3.1, 3.2
def test_theorem_3_1_candidates_survive_compression():
    """A candidate v of u in the data graph (Definition 3.3) lies in a node
    that is a candidate of u in the weighted graph (Definition 3.5)."""
    rng = np.random.default_rng(308)
    for _ in range(600):
        g, q = twin_tiny(rng) if rng.random() < 0.5 else random_tiny(rng)
        o = O.OracleGraph.from_graph(g)
        w = O.WeightedGraph(o, deltas(rng))
        c0 = O.candidates(o, q, True)
        cw = O.wcandidates(w, q)
        for u in range(q.k):
            for v in np.flatnonzero(c0[u]):
                assert cw[u, w.group[v]], (u, v)


def test_theorem_3_2_embeddings_map_to_weighted_solutions():
    """Every embedding f of the query in the data graph maps, through the
    nodes holding its vertices, onto a solution in the weighted graph (query
    edges on weighted edges, or inside one node), and each f(u)'s node
    survives the refinement there."""
    rng = np.random.default_rng(309)
    seen = 0
    for _ in range(600):
        g, q = twin_tiny(rng) if rng.random() < 0.5 else random_tiny(rng)
        o = O.OracleGraph.from_graph(g)
        w = O.WeightedGraph(o, deltas(rng))
        S = O.wrefine(w, q, O.wcandidates(w, q))
        wedges = set(zip(w.src.tolist(), w.rel.tolist(), w.dst.tolist()))
        inner = {(x, r) for r in range(g.num_rels) for x in range(w.n) if w.wnode[0, r, x] > 0}
        for f in python_brute(g, q):
            h = [int(w.group[v]) for v in f]
            for u in range(q.k):
                assert S[u, h[u]]
            for a, b, r in zip(q.esrc.tolist(), q.edst.tolist(), q.erel.tolist()):
                if h[a] == h[b]:
                    assert any((h[a], rr) in inner for rr in range(g.num_rels) if r == ANY or rr == r)
                else:
                    assert any((h[a], rr, h[b]) in wedges for rr in range(g.num_rels) if r == ANY or rr == r)
            seen += 1
    assert seen > 200


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("a,b,levels", [(4, 4, 1), (5, 3, 2), (8, 6, 3), (7, 7, 2)])
def test_complete_bipartite_compresses_to_power_of_two_groups(a, b, levels):
    """K_{a,b} directed from A to B, one relation, one type: with delta = 1
    all of A (all of B) share one adjacency list at every level, so each
    level pairs consecutive nodes: ceil(a / 2^L) + ceil(b / 2^L) nodes, every
    edge weight exact (wout = |M(V)|, win = |M(U)|), no internal edges, and
    a k-vertex out-star query still has perm(b, k-1) * a embeddings."""
    tr = [(s, 0, a + d) for s in range(a) for d in range(b)]
    g = graph_from_triples(a + b, tr)
    o = O.OracleGraph.from_graph(g)
    w = O.WeightedGraph(o, [1.0] * levels)
    assert w.n == ceil(a / 2 ** levels) + ceil(b / 2 ** levels)
    sizes = np.diff(w.moff)
    for x, r, y, wo, wi in zip(w.src, w.rel, w.dst, w.wout, w.win):
        assert wo == sizes[y] and wi == sizes[x]
    assert w.ne == ceil(a / 2 ** levels) * ceil(b / 2 ** levels)
    assert (w.wnode == 0).all()
    assert w.ratio() == pytest.approx((w.n + w.ne) / (a + b + a * b))
    for k in (2, 3):
        q = query(k, [(0, i, 0) for i in range(1, k)])
        got, homs = O.match_compressed(o, w, q, cap=0)
        want = a
        for i in range(k - 1):
            want *= b - i
        assert got.count == want == O.match(o, q, cap=0).count
