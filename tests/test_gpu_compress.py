"""Matching through a multi-level compression (Sections 3.4-3.5) on the GPU,
through the C ABI: the compression loaded on the device equals the oracle's,
the weighted-graph candidate sets after refinement equal the oracle's
fixpoint of Definition 3.5's sets, and the embeddings found through the
compressed graph equal the oracle's embeddings in the data graph (counts,
fingerprints, sorted rows) on tiny graphs, the 10,000-vertex concept-family
graph and a sample of the 1M-vertex one."""
import numpy as np
import pytest

import oracle as O
import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I
from tests.test_oracle_compression import deltas, twin_tiny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fam10k():
    import torch
    torch.cuda.set_device(0)
    w = I.WORKLOADS["compress-10k"]
    g = w.graph()
    qs = w.queries(g)
    cg = gs.CompressedGraph(g, w.deltas)
    og = O.OracleGraph.from_graph(g)
    ow = O.WeightedGraph(og, w.deltas)
    return w, g, qs, cg, og, ow


def test_device_compression_equals_oracle(fam10k):
    w, g, qs, cg, og, ow = fam10k
    ex = cg.export()
    info = cg.info()
    assert info["nodes"] == ow.n and info["weighted_edges"] == ow.ne
    np.testing.assert_array_equal(ex["group"], ow.group)
    for k in ("src", "rel", "dst", "wout", "win"):
        np.testing.assert_array_equal(ex[k], getattr(ow, k), err_msg=k)
    np.testing.assert_array_equal(ex["wnode"], ow.wnode)
    assert info["ratio"] == pytest.approx(ow.ratio())
    assert info["ratio"] < 0.8


def test_weighted_candidates_equal_oracle_fixpoint(fam10k):
    """The weighted-graph stage (Definition 3.5 filter, exploration,
    refinement to the fixpoint) gives the oracle's unique fixpoint."""
    w, g, qs, cg, og, ow = fam10k
    for q in qs[:60]:
        want = O.wrefine(ow, q, O.wcandidates(ow, q))
        got = cg.candidates(q)
        for u in range(q.k):
            np.testing.assert_array_equal(got[u], np.flatnonzero(want[u]).astype(np.uint32))


def assert_same(res, want):
    assert res.status == 0, res.status
    assert (res.count, res.fingerprint) == (want.count, want.fingerprint)
    np.testing.assert_array_equal(res.rows, want.rows)


def test_compressed_matching_equals_oracle_10k(fam10k):
    w, g, qs, cg, og, ow = fam10k
    res = cg.match_batch(qs, cap=1 << 16)
    for q, r in zip(qs, res):
        assert_same(r, O.match(og, q, cap=1 << 16))
    assert sum(r.count for r in res) > len(qs)
    # and again: the stages' buffers were left clean for the next call
    res2 = cg.match_batch(qs[::-1], cap=1 << 16)
    for a, b in zip(res2, res[::-1]):
        assert (a.count, a.fingerprint) == (b.count, b.fingerprint)


def test_compressed_matching_variable_edges_and_projection(fam10k):
    w, g, qs, cg, og, ow = fam10k
    vq = I.with_variable_edges(qs[:40], 0.4, seed=9)
    for q, r in zip(vq, cg.match_batch(vq, cap=1 << 16, project=[0, 1])):
        o = O.match(og, q, cap=1 << 16, project=[0, 1])
        assert r.status == 0 and (r.count, r.fingerprint) == (o.count, o.fingerprint)
        np.testing.assert_array_equal(r.rows, o.rows)


def test_compressed_matching_tiny_graphs():
    rng = np.random.default_rng(501)
    for case in range(80):
        g, q = twin_tiny(rng)
        ds = deltas(rng)
        cg = gs.CompressedGraph(g, ds)
        og = O.OracleGraph.from_graph(g)
        r = cg.match_batch([q], cap=1 << 12)[0]
        assert_same(r, O.match(og, q, cap=1 << 12))
        cg.free()


def test_compressed_matching_1m_sample():
    """The 1M-vertex concept-family graph compressed at the thesis's
    thresholds: a seeded sample of 100 queries equals the oracle."""
    w = I.WORKLOADS["compress-1m"]
    g = w.graph()
    qs = w.queries(g)
    cg = gs.CompressedGraph(g, w.deltas)
    assert cg.info()["ratio"] < 0.7
    og = O.OracleGraph.from_graph(g)
    idx = np.random.default_rng(7).choice(len(qs), 100, replace=False)
    sample = [qs[i] for i in sorted(idx)]
    res = cg.match_batch(sample, cap=1 << 14)
    for q, r in zip(sample, res):
        o = O.match(og, q, cap=1 << 14, time_limit_s=10.0)
        if o.status == 2:
            continue
        assert_same(r, o)
    dg = gs.DeviceGraph(g)
    for a, b in zip(res, gs.match_batch(dg, sample, cap=1 << 14)):
        assert (a.count, a.fingerprint) == (b.count, b.fingerprint)
        np.testing.assert_array_equal(a.rows, b.rows)
    cg.free()
    dg.free()
