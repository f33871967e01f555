"""The seeded generators: determinism and the stated structure."""
import numpy as np

import oracle as O
from paper_1807_08804_gb300 import inputs as I


def test_graph_structure_and_determinism():
    g = I.make_graph(5000, 40000, seed=3)
    h = I.make_graph(5000, 40000, seed=3)
    np.testing.assert_array_equal(g.col_targets, h.col_targets)
    np.testing.assert_array_equal(g.vertex_type, h.vertex_type)
    deg = np.diff(g.row_offsets.astype(np.int64))
    assert deg.sum() == 40000 and deg.min() >= 1 and deg.max() <= 1000
    src = np.repeat(np.arange(5000, dtype=np.uint64), deg)
    assert not (src == g.col_targets).any()                       # no self-loops
    key = (src << np.uint64(32)) | (g.edge_rel.astype(np.uint64) << np.uint64(24)) | g.col_targets
    assert np.unique(key).size == key.size                        # no repeated triples
    tf = np.bincount(g.vertex_type, minlength=64) / 5000
    rf = np.bincount(g.edge_rel, minlength=34) / 40000
    assert 0.17 < tf[0] < 0.25 and 0.24 < rf[0] < 0.32            # Zipf heads (21.1%, 28.0%)
    assert I.make_graph(5000, 40000, seed=4).col_targets.tolist() != g.col_targets.tolist()


def test_walk_queries_contain_their_walk():
    g = I.make_graph(3000, 18000, seed=9)
    og = O.OracleGraph.from_graph(g)
    qs = I.make_walk_queries(g, 60, 3, 8, p_bind=0.3, seed=2)
    for q in qs:
        assert 3 <= q.k <= 8 and q.m >= q.k - 1
        assert O.verify(og, q, q.walked[None, :]) == -1            # the walked map is a match
        b = q.vbind != I.UNBOUND
        assert (q.vtype[b] == I.ANY).all() and (q.vbind[b] == q.walked[b]).all()
        assert (q.vtype[~b] == g.vertex_type[q.walked[~b]]).all()
    qc = I.make_walk_queries(g, 40, 3, 12, p_bind=0.1, cyclic_half=True, seed=5)
    assert all(q.m == q.k - 1 for q in qc[1::2])                  # odd: trees
    assert sum(q.m > q.k - 1 for q in qc[0::2]) >= 15             # even: mostly cyclic


def test_shape_queries_and_arrivals():
    g = I.make_graph(3000, 18000, seed=9)
    qs = I.make_shape_queries(g, 8, seed=1)
    assert [q.k for q in qs] == [4, 4, 5, 5, 4, 4, 6, 6]
    assert [q.m for q in qs] == [4, 4, 5, 5, 6, 6, 5, 5]
    assert all((q.vbind == I.UNBOUND).all() for q in qs)
    t = I.make_arrivals(20000, 1000.0, seed=1)
    assert (np.diff(t) > 0).all() and abs(t[-1] - 20.0) < 1.0


def test_variable_edge_queries():
    """single-10k-var: the single-10k queries with about 30% of edges made
    variable, the rest unchanged, deterministic, the walked map still a
    match."""
    w, wv = I.WORKLOADS["single-10k"], I.WORKLOADS["single-10k-var"]
    g = wv.graph()
    og = O.OracleGraph.from_graph(g)
    base, qs, again = w.queries(g), wv.queries(g), wv.queries(g)
    var = tot = 0
    for b, q, a in zip(base, qs, again):
        np.testing.assert_array_equal(q.erel, a.erel)
        np.testing.assert_array_equal(q.esrc, b.esrc)
        fixed = q.erel != I.ANY
        np.testing.assert_array_equal(q.erel[fixed], b.erel[fixed])
        assert O.verify(og, q, q.walked[None, :]) == -1
        var += int((~fixed).sum())
        tot += q.m
    assert 0.22 < var / tot < 0.38


def test_anchored_untyped_queries():
    """ablation-1m's recipe on a small graph: one concept node (the walk
    start, bound), untyped variables elsewhere; the walked map matches."""
    g = I.make_graph(3000, 18000, seed=9)
    og = O.OracleGraph.from_graph(g)
    qs = I.anchor_untyped(I.make_walk_queries(g, 30, 4, 8, p_bind=0.0, cyclic_half=True, seed=3))
    for q in qs:
        assert q.vbind[0] == q.walked[0] and (q.vbind[1:] == I.UNBOUND).all() and (q.vtype == I.ANY).all()
        assert O.verify(og, q, q.walked[None, :]) == -1
