"""Parity of the CUDA engine with the CPU oracle, through the C ABI.

Integer work: every comparison is exact (counts, fingerprints, the sorted
embedding rows, candidate sets, candidate-edge tables)."""
import numpy as np
import pytest

import oracle as O
import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I
from tests.helpers import complete_digraph_triples, graph_from_triples, query, random_tiny

pytestmark = pytest.mark.gpu


def assert_same(r, o, ctx=""):
    assert r.status == 0, (ctx, r.status)
    assert r.count == o.count, (ctx, r.count, o.count)
    assert r.fingerprint == o.fingerprint, (ctx, r.fingerprint, o.fingerprint)
    np.testing.assert_array_equal(r.rows, o.rows, err_msg=str(ctx))


@pytest.fixture(scope="module")
def small():
    w = I.WORKLOADS["single-10k"]
    g = w.graph()
    qs = w.queries(g)
    return g, qs, O.OracleGraph.from_graph(g), gs.DeviceGraph(g)


def test_graph_canonicalisation_counts_distinct_triples(small):
    g, _, og, dg = small
    assert dg.num_edges == og.E


def test_small_workload_batch_bit_exact(small):
    g, qs, og, dg = small
    res = gs.match_batch(dg, qs, cap=1 << 20)
    for i, (q, r) in enumerate(zip(qs, res)):
        assert_same(r, O.match(og, q, cap=1 << 20), i)


def test_small_workload_one_at_a_time(small):
    g, qs, og, dg = small
    for i, q in enumerate(qs[:25]):
        assert_same(gs.match(dg, q, cap=1 << 20), O.match(og, q, cap=1 << 20), i)


def test_filter_kernel_candidates(small):
    g, qs, og, dg = small
    for q in qs[:30]:
        got = gs.inspect_candidates(dg, q, gs.GS_STAGE_FILTER)
        want = O.candidates(og, q, signature=True)
        for u in range(q.k):
            np.testing.assert_array_equal(got[u], np.flatnonzero(want[u]).astype(np.uint32))


def test_refinement_fixpoint(small):
    g, qs, og, dg = small
    for q in qs[:30]:
        got = gs.inspect_candidates(dg, q, gs.GS_STAGE_FIXPOINT)
        want = O.fixpoint(og, q)
        for u in range(q.k):
            np.testing.assert_array_equal(got[u], np.flatnonzero(want[u]).astype(np.uint32))


def test_edge_tables(small):
    g, qs, og, dg = small
    for q in qs[:20]:
        fix = O.fixpoint(og, q)
        for e in range(q.m):
            for from_src in (True, False):
                k1, o1, v1 = gs.inspect_edge_table(dg, q, e, from_src)
                k2, o2, v2 = O.edge_table(og, q, fix, e, from_src)
                np.testing.assert_array_equal(k1, k2)
                np.testing.assert_array_equal(o1, o2)
                np.testing.assert_array_equal(v1, v2)


def test_tiny_random_instances_against_brute_force():
    rng = np.random.default_rng(2024)
    for case in range(120):
        g, q = random_tiny(rng)
        o = O.OracleGraph.from_graph(g)
        dg = gs.DeviceGraph(g)
        want = O.brute(o, q, cap=1 << 16)
        got = gs.match_batch(dg, [q, q], cap=1 << 16)
        for r in got:
            assert_same(r, want, case)
        dg.free()


def test_closed_forms():
    from math import comb, perm
    n = 9
    dg = gs.DeviceGraph(graph_from_triples(n, complete_digraph_triples(n)))
    for k in (2, 3, 4, 5):
        path = query(k, [(i, i + 1, 0) for i in range(k - 1)])
        cyc = query(k, [(i, (i + 1) % k, 0) for i in range(k)]) if k > 2 else path
        for r in gs.match_batch(dg, [path, cyc], cap=0, mode=gs.GS_COUNT_ONLY):
            assert r.count == perm(n, k)
    tt = gs.DeviceGraph(graph_from_triples(10, [(i, 0, j) for i in range(10) for j in range(10) if i < j]))
    for k in (3, 4, 5):
        path = query(k, [(i, i + 1, 0) for i in range(k - 1)])
        cyc = query(k, [(i, (i + 1) % k, 0) for i in range(k)])
        clique = query(k, [(i, j, 0) for i in range(k) for j in range(i + 1, k)])
        r = gs.match_batch(tt, [path, cyc, clique], cap=0, mode=gs.GS_COUNT_ONLY)
        assert [x.count for x in r] == [comb(10, k), 0, comb(10, k)]
    star = gs.DeviceGraph(graph_from_triples(8, [(0, 0, i) for i in range(1, 8)]))
    for s in (1, 3, 5, 7, 8):
        r = gs.match(star, query(s + 1, [(0, i, 0) for i in range(1, s + 1)]), cap=0, mode=gs.GS_COUNT_ONLY)
        assert r.count == (perm(7, s) if s <= 7 else 0)


def test_large_outputs_take_the_radix_path():
    """Outputs above the one-block sort limit (2,048 rows) are sorted by the
    global radix path; a batch mixes both kinds."""
    n = 9
    g = graph_from_triples(n, complete_digraph_triples(n))
    og = O.OracleGraph.from_graph(g)
    dg = gs.DeviceGraph(g)
    qs = [query(k, [(i, i + 1, 0) for i in range(k - 1)]) for k in (2, 4, 5, 3)]
    qs.append(query(4, [(0, 1, 0), (0, 2, 0), (0, 3, 0)], vbind=[I.UNBOUND, 3, I.UNBOUND, I.UNBOUND]))
    res = gs.match_batch(dg, qs, cap=1 << 20)
    for i, (q, r) in enumerate(zip(qs, res)):
        assert_same(r, O.match(og, q, cap=1 << 20), i)
    assert res[2].count == 15120
    r = gs.match(dg, qs[2], cap=1 << 20)
    assert_same(r, O.match(og, qs[2], cap=1 << 20))


def test_more_embeddings_than_cap_returns_the_smallest_rows():
    """count > cap: the exact count and fingerprint, and the cap
    lexicographically smallest embeddings (the chunked path's running top-cap)."""
    n = 9
    g = graph_from_triples(n, complete_digraph_triples(n))
    og = O.OracleGraph.from_graph(g)
    dg = gs.DeviceGraph(g)
    qs = [query(5, [(i, i + 1, 0) for i in range(4)]), query(4, [(i, (i + 1) % 4, 0) for i in range(4)]),
          query(1, [], vtype=[0]), query(3, [(0, 1, 0), (2, 1, 0)])]
    for cap in (1, 100, 5000):
        res = gs.match_batch(dg, qs, cap=cap)
        for i, (q, r) in enumerate(zip(qs, res)):
            o = O.match(og, q, cap=cap)
            assert_same(r, o, (cap, i))
            assert r.truncated == (o.count > cap)


def test_outputs_cut_at_cap_before_sorting():
    """More than 2,048 rows and more than cap, within 16 x cap: the rows stay
    on the device, a radix select on the sort keys keeps about cap of them
    and the sorted first cap equal the oracle's, also when every key shares
    its top bits (a bound first vertex)."""
    n = 16
    g = graph_from_triples(n, complete_digraph_triples(n))
    og = O.OracleGraph.from_graph(g)
    dg = gs.DeviceGraph(g)
    path4 = query(4, [(i, i + 1, 0) for i in range(3)])                       # 43,680 rows
    bound = query(4, [(i, i + 1, 0) for i in range(3)], vbind=[3, I.UNBOUND, I.UNBOUND, I.UNBOUND])  # 2,730 rows
    star = query(4, [(1, 0, 0), (2, 0, 0), (3, 0, 0)])                        # 43,680 rows, centre last in keys
    for q, cap in ((path4, 3000), (path4, 2731), (bound, 300), (bound, 2729), (star, 4096)):
        r = gs.match_batch(dg, [q], cap=cap)[0]
        o = O.match(og, q, cap=cap)
        assert o.count > 2048 and cap < o.count <= 16 * cap
        assert_same(r, o, cap)


def test_chunked_mode_streams_every_embedding():
    """GS_CHUNKED: every embedding reaches the callback exactly once (rows in
    query-vertex order, chunks in any order), with the exact count and
    fingerprint; small chunk budgets force many chunks."""
    n = 12
    g = graph_from_triples(n, complete_digraph_triples(n))
    og = O.OracleGraph.from_graph(g)
    dg = gs.DeviceGraph(g)
    path6 = query(6, [(i, i + 1, 0) for i in range(5)])                        # 665,280 embeddings
    star = query(4, [(0, 1, 0), (0, 2, 0), (0, 3, 0)], vbind=[5, I.UNBOUND, I.UNBOUND, I.UNBOUND])
    single = query(1, [], vtype=[0])
    none = query(2, [(0, 1, 0)], vbind=[3, 3])                                 # injectivity: no embedding
    qs = [path6, star, single, none]
    for chunk_bytes in (1 << 16, 1 << 22):
        got = {i: [] for i in range(len(qs))}
        res = gs.match_batch(dg, qs, cap=0, mode=gs.GS_CHUNKED, chunk_bytes=chunk_bytes,
                             on_chunk=lambda rows, q: got[q].append(rows))
        for i, q in enumerate(qs):
            o = O.match(og, q, cap=1 << 21)
            rows = np.concatenate(got[i]) if got[i] else np.zeros((0, len(q.vtype)), np.uint32)
            order = np.lexsort(rows.T[::-1]) if rows.shape[0] else np.zeros(0, int)
            np.testing.assert_array_equal(rows[order], o.rows)
            assert (res[i].count, res[i].fingerprint) == (o.count, o.fingerprint) == (rows.shape[0], o.fingerprint)
            assert res[i].rows.shape[0] == 0 and not res[i].truncated
        if chunk_bytes == 1 << 16:
            assert len(got[0]) > 10
    with pytest.raises(gs.GSError):
        gs.match(dg, path6, mode=gs.GS_CHUNKED)  # no callback


def test_chunked_join_with_small_level_buffers(monkeypatch):
    """Partial embeddings that overflow the level budget finish on the
    chunked depth-first path; tiny buffers force many chunks."""
    from math import perm
    monkeypatch.setenv("GS_FALLBACK_DEPTH_WORDS", "32768")
    monkeypatch.setenv("GS_FALLBACK_DEPTH_ROWS", "8192")
    n = 12
    g = graph_from_triples(n, complete_digraph_triples(n))
    og = O.OracleGraph.from_graph(g)
    dg = gs.DeviceGraph(g)  # fresh graph: fresh chunked-join context with the small buffers
    path6 = query(6, [(i, i + 1, 0) for i in range(5)])
    star = query(5, [(0, i, 0) for i in range(1, 5)])
    res = gs.match_batch(dg, [path6, star], cap=1 << 20, chunk_bytes=1 << 16)
    assert res[0].count == perm(12, 6)
    for q, r in zip([path6, star], res):
        assert_same(r, O.match(og, q, cap=1 << 20))
    cnt = gs.match_batch(dg, [path6, star], cap=0, mode=gs.GS_COUNT_ONLY, chunk_bytes=1 << 16)
    assert [(c.count, c.fingerprint) for c in cnt] == [(r.count, r.fingerprint) for r in res]
    top = gs.match(dg, path6, cap=777, chunk_bytes=1 << 16)
    assert_same(top, O.match(og, path6, cap=777))


def test_results_invariant_to_schedule(small):
    g, qs, og, dg = small
    sub = qs[:40]
    base = gs.match_batch(dg, sub, cap=1 << 20)
    for group in (4, 8, 16, 32):
        for use_graph in (True, False):
            for rounds in (0, 1, 3, gs.GS_ROUNDS_NONE):
                b = gs.Batch(dg, sub, cap=1 << 20)
                b.configure(use_graph=use_graph, group=group, refine_rounds=rounds)
                b.run()
                b.finish()
                for i, (x, y) in enumerate(zip(b.fetch(), base)):
                    assert (x.count, x.fingerprint) == (y.count, y.fingerprint), (group, use_graph, rounds, i)
                    np.testing.assert_array_equal(x.rows, y.rows)
                b.close()
    b = gs.Batch(dg, sub, cap=1 << 20, wave_queries=1)
    for rep in range(2):  # a replayed batch gives the same results
        b.run()
        b.finish()
        for x, y in zip(b.fetch(), base):
            assert (x.count, x.fingerprint) == (y.count, y.fingerprint)
            np.testing.assert_array_equal(x.rows, y.rows)
    b.close()


def test_count_only_mode(small):
    g, qs, og, dg = small
    a = gs.match_batch(dg, qs[:50], cap=1 << 20)
    b = gs.match_batch(dg, qs[:50], cap=0, mode=gs.GS_COUNT_ONLY)
    for x, y in zip(a, b):
        assert (x.count, x.fingerprint) == (y.count, y.fingerprint)
        assert y.rows.shape[0] == 0


def test_edge_cases(small):
    g, qs, og, dg = small
    V = g.num_vertices
    single = query(1, [], vtype=[3])
    bound_wrong = query(2, [(0, 1, 0)], vtype=[I.ANY, I.ANY], vbind=[0, 0])  # same id twice: 0 embeddings
    self_loop = query(2, [(0, 0, 0)])
    disconnected = query(3, [(0, 1, 0)])
    out_of_range = query(2, [(0, 1, 0)], vbind=[V, I.UNBOUND])
    res = gs.match_batch(dg, [single, bound_wrong, self_loop, disconnected, out_of_range, qs[0]], cap=1 << 20)
    assert_same(res[0], O.match(og, single, cap=1 << 20))
    assert res[1].status == 0 and res[1].count == 0 and res[1].rows.shape[0] == 0
    assert res[2].status == gs.GS_ERR_INVALID
    assert res[3].status == gs.GS_ERR_UNSUPPORTED
    assert res[4].status == gs.GS_ERR_INVALID
    assert_same(res[5], O.match(og, qs[0], cap=1 << 20))
    with pytest.raises(gs.GSError):
        gs.match(dg, self_loop)
    assert gs.match_batch(dg, [], cap=1) == []


@pytest.fixture(scope="module")
def scale_1m():
    w = I.WORKLOADS["single-1m"]
    g = w.graph()
    qs = w.queries(g)
    return g, qs, O.OracleGraph.from_graph(g), gs.DeviceGraph(g)


def test_scale_1m_batch_against_oracle(scale_1m):
    """The 1M-vertex / 8M-edge workload at full size, in the batched launch
    configuration the benchmark times: all 1,000 queries' counts and
    fingerprints, rows for a sample."""
    g, qs, og, dg = scale_1m
    res = gs.match_batch(dg, qs, cap=1 << 22)
    cnt, fp, st, _ = O.match_many(og, qs, threads=0, time_limit_s=60.0)
    assert (st == 0).all()
    for i, r in enumerate(res):
        assert r.status == 0
        assert (r.count, r.fingerprint) == (int(cnt[i]), int(fp[i])), i
    rng = np.random.default_rng(1)
    for i in rng.choice(len(qs), 60, replace=False):
        assert_same(res[i], O.match(og, qs[i], cap=1 << 22), i)


def test_scale_1m_one_at_a_time_waves(scale_1m):
    g, qs, og, dg = scale_1m
    sub = qs[:100]
    b = gs.Batch(dg, sub, cap=1 << 22, wave_queries=1)
    b.run()
    b.finish()
    for i, r in enumerate(b.fetch()):
        assert_same(r, O.match(og, sub[i], cap=1 << 22), i)
    b.close()


def test_autotuner_choice_is_cached_and_results_unchanged(small, tmp_path):
    g, qs, og, dg = small
    sub = qs[:60]
    base = gs.match_batch(dg, sub, cap=1 << 20)
    cache = str(tmp_path / "tune.txt")
    t1 = gs.tune(dg, sub, cap=1 << 20, cache_path=cache)
    assert t1["group"] in (4, 8, 16, 32) and t1["refine_rounds"] in (gs.GS_ROUNDS_NONE, 1, 2, 4) and not t1["from_cache"]
    assert t1["configs_tried"] == 22 and t1["join_group"] in (4, 8, 16, 32)
    t2 = gs.tune(dg, sub, cap=1 << 20, cache_path=cache)
    assert t2["from_cache"] and (t2["group"], t2["refine_rounds"], t2["join_group"]) == (
        t1["group"], t1["refine_rounds"], t1["join_group"])
    b = gs.Batch(dg, sub, cap=1 << 20)  # built with the tuned settings
    b.run()
    b.finish()
    for x, y in zip(b.fetch(), base):
        assert (x.count, x.fingerprint) == (y.count, y.fingerprint)
        np.testing.assert_array_equal(x.rows, y.rows)
    b.close()
    gs.lib().gs_tune_set(dg._h, 0, 0)


def test_large_call_as_concurrent_sub_batches(small):
    """gs_match_batch with 4,096 queries or more runs as four sub-batches at
    once on their own streams, their rows in four page-locked buffers: the
    results equal one batch's, query by query, and the buffers come back to
    the pool when the results go."""
    import torch
    g, qs, og, dg = small
    many = I.make_walk_queries(g, 5000, 3, 7, p_bind=0.2, seed=31)
    b = gs.Batch(dg, many, cap=1 << 12)
    b.run()
    b.finish()
    want = b.fetch()
    b.close()
    for rep in range(3):  # pooled buffers are reused call after call
        got = gs.match_batch(dg, many, cap=1 << 12)
        assert len(got) == len(want)
        for i, (x, y) in enumerate(zip(got, want)):
            assert (x.count, x.fingerprint, x.status) == (y.count, y.fingerprint, y.status), i
            np.testing.assert_array_equal(x.rows, y.rows)
        del got
    # prepared batches run together give the same results too
    streams = [torch.cuda.Stream() for _ in range(3)]
    parts = [gs.Batch(dg, many[i * 1700:(i + 1) * 1700], cap=1 << 12, stream=streams[i].cuda_stream) for i in range(3)]
    for p in parts:
        p.stats_enable(True)
    gs.run_all(parts, None)  # timed: each batch's events are read after all are queued
    for p in parts:
        p.finish()
        p.stats_reset()
    gs.run_all(parts, None)
    res = []
    for p in parts:
        p.finish()
        res += p.fetch()
    for x, y in zip(res, want):
        assert (x.count, x.fingerprint) == (y.count, y.fingerprint)
        np.testing.assert_array_equal(x.rows, y.rows)
    # the time some launch of a kind ran lies between the longest one batch
    # spent in that kind (its launches run one after another on its stream)
    # and the sum over the batches
    busy = gs.stats_busy(parts)
    per = [p.stats() for p in parts]
    for kind in busy:
        ms = [st[kind]["ms"] for st in per]
        if sum(st[kind]["launches"] for st in per) == 0:
            assert busy[kind] == 0.0
            continue
        assert max(ms) * 0.999 - 1e-3 <= busy[kind] <= sum(ms) * 1.001 + 1e-3, (kind, busy[kind], ms)
    assert sum(busy.values()) > 0
    for p in parts:
        p.close()


@pytest.fixture(scope="module")
def wide_ids():
    """A 12-vertex complete digraph placed at the top of 4.2M vertex ids
    (ids need 23 bits, so a sort key holds four columns and rows of five or
    more vertices tie on their keys), the other vertices isolated."""
    V, n = 4_200_000, 12
    hub = np.arange(V - n, V, dtype=np.uint32)
    ro = np.zeros(V + 1, np.uint64)
    ro[V - n + 1:] = np.cumsum(np.full(n, n - 1, np.uint64))
    col = np.array([d for s in hub for d in hub if d != s], np.uint32)
    g = I.Graph(V, ro, col, np.zeros(col.shape[0], np.uint32), np.zeros(V, np.uint32), 1, 1)
    return g, O.OracleGraph.from_graph(g), gs.DeviceGraph(g), hub


def test_sample_sort_and_merge_path_agree_with_the_oracle(wide_ids):
    """Large outputs (above 2,048 rows) through the sample sort and through
    the tile sort and merge passes give the oracle's rows: paths of 4-7
    vertices (keys holding the whole row, and rows tying on their keys) with
    a 3-vertex path of 1,320 rows beside them (one-block sort), a
    path with more rows than cap (selection first), twelve outputs of 7,920
    rows each (one per bound start vertex) and projected rows with repeats."""
    g, og, dg, hub = wide_ids
    cap = 1 << 20
    paths = [query(k, [(i, i + 1, 0) for i in range(k - 1)]) for k in (3, 4, 5, 6, 7)]
    bound = [query(5, [(i, i + 1, 0) for i in range(4)], vbind=[int(h)] + [I.UNBOUND] * 4) for h in hub]
    qs = paths + bound
    want = [O.match(og, q, cap=cap) for q in qs]
    assert want[4].count > cap and all(w.count > 2048 for w in want[1:])  # the 3-path: one-block sort
    for merge_only in (False, True):
        b = gs.Batch(dg, qs, cap=cap)
        b.set_sort(merge_only=merge_only)
        for _ in range(2):  # the second run reuses every buffer
            b.run()
            b.finish()
            for i, (r, o) in enumerate(zip(b.fetch(), want)):
                assert_same(r, o, (merge_only, i))
        b.close()
    proj = [query(5, [(i, i + 1, 0) for i in range(4)])]
    pw = O.match(og, proj[0], cap=cap, project=[0, 3])
    for merge_only in (False, True):
        b = gs.Batch(dg, proj, cap=cap, project=[0, 3])
        b.set_sort(merge_only=merge_only)
        b.run()
        b.finish()
        assert_same(b.fetch()[0], pw, ("projected", merge_only))
        b.close()
