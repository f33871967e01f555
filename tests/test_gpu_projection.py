"""Projection (Section 3.5: only the matches of some query vertices are
wanted) on the CUDA engine against the oracle: the distinct tuples of the
projected vertices, ascending, cut at cap with `truncated` when more exist;
count and fingerprint over every embedding.  Exact comparisons."""
import numpy as np
import pytest

import oracle as O
import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I
from tests.helpers import complete_digraph_triples, graph_from_triples, query, random_tiny

pytestmark = pytest.mark.gpu


def assert_proj(r, o, ctx=""):
    assert r.status == 0, (ctx, r.status)
    assert (r.count, r.fingerprint) == (o.count, o.fingerprint), ctx
    np.testing.assert_array_equal(r.rows, o.rows, err_msg=str(ctx))
    assert r.truncated == o.truncated, (ctx, r.truncated, o.truncated)


def test_tiny_random_instances_with_projection():
    """Small outputs: duplicates dropped inside the one-block sort."""
    rng = np.random.default_rng(5150)
    for case in range(100):
        g, q = random_tiny(rng, p_any=0.2)
        cols = [u for u in range(q.k) if rng.random() < 0.5] or [int(rng.integers(q.k))]
        o = O.OracleGraph.from_graph(g)
        dg = gs.DeviceGraph(g)
        for cap in (1 << 16, 2):
            want = O.match(o, q, cap=cap, project=cols)
            for r in gs.match_batch(dg, [q, q], cap=cap, project=cols):
                assert_proj(r, want, (case, cap))
        dg.free()


@pytest.fixture(scope="module")
def k12():
    n = 12
    g = graph_from_triples(n, complete_digraph_triples(n))
    return g, O.OracleGraph.from_graph(g), gs.DeviceGraph(g)


@pytest.mark.parametrize("cols,cap", [
    ([0, 5], 1 << 20),          # 132 tuples of 665,280 rows: device merge sort, then per-tile dedupe
    ([2], 1 << 20),             # 12 tuples
    ([0, 1, 2, 3], 1 << 20),    # 11,880 tuples across many tiles
    ([0, 1, 2, 3, 4], 50_000),  # 95,040 tuples, cut at cap on the device (truncated)
    ([0, 5], 50),               # more rows than 16 x cap: the chunked path's running top-cap
    ([0, 1, 2, 3], 5000),       # chunked path, more tuples than cap (truncated)
])
def test_large_projected_outputs(k12, cols, cap):
    g, og, dg = k12
    path6 = query(6, [(i, i + 1, 0) for i in range(5)])
    want = O.match(og, path6, cap=cap, project=cols)
    assert_proj(gs.match(dg, path6, cap=cap, project=cols), want, (cols, cap))
    # mixed with unprojected-shape queries in one batch: per-query outputs stay independent
    star = query(4, [(0, 1, 0), (0, 2, 0), (0, 3, 0)])
    pc = [c for c in cols if c < 4][:2]  # vertices both queries have
    res = gs.match_batch(dg, [path6, star], cap=cap, project=pc)
    assert_proj(res[0], O.match(og, path6, cap=cap, project=pc), ("batch", cols, cap))
    assert_proj(res[1], O.match(og, star, cap=cap, project=pc), ("star", cols, cap))


def test_workload_batch_with_projection():
    w = I.WORKLOADS["single-10k-var"]
    g = w.graph()
    og = O.OracleGraph.from_graph(g)
    dg = gs.DeviceGraph(g)
    qs = w.queries(g)
    for cols in ([0], [0, 2], [1, 2]):
        for i, r in enumerate(gs.match_batch(dg, qs, cap=1 << 20, project=cols)):
            assert_proj(r, O.match(og, qs[i], cap=1 << 20, project=cols), (cols, i))


def test_projection_errors_and_identity(k12):
    g, og, dg = k12
    path3 = query(3, [(0, 1, 0), (1, 2, 0)])
    r = gs.match_batch(dg, [path3], cap=10, project=1 << 3)  # vertex 3 does not exist
    assert r[0].status == 1
    with pytest.raises(gs.GSError):
        gs.match(dg, path3, mode=gs.GS_CHUNKED, on_chunk=lambda rows, q: None, project=[0])
    full = gs.match(dg, path3, cap=1 << 12)
    allv = gs.match(dg, path3, cap=1 << 12, project=[0, 1, 2])
    np.testing.assert_array_equal(full.rows, allv.rows)
    assert full.truncated == allv.truncated


def test_serving_with_projection(k12):
    g, og, dg = k12
    qs = [query(3, [(0, 1, 0), (1, 2, 0)]), query(4, [(0, 1, 0), (1, 2, 0), (2, 3, 0)])]
    srv = gs.Server(dg)
    try:
        tickets = [(srv.submit(q, cap=100, project=[0, q.k - 1]), q) for q in qs for _ in range(3)]
        for t, q in tickets:
            got = None
            for _ in range(20000):
                got = srv.poll(t)
                if got is not None:
                    break
                import time
                time.sleep(0.001)
            assert got is not None
            assert_proj(got[0], O.match(og, q, cap=100, project=[0, q.k - 1]))
    finally:
        srv.close()
