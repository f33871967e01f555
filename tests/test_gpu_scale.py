"""Parity at the full sizes of the batched (4M vertices / 32M edges, 10,000
queries) and stress (16M / 200M, 200 unbound shape queries) workloads, in
the launch configuration the benchmark uses.  Where the oracle cannot finish
(up to ~1e9 embeddings per query), properties that hold at any size are
checked instead: count-only == enumerated count and fingerprint, and every
returned row verified edge by edge against the input graph."""
import numpy as np
import pytest

import oracle as O
import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def triple_keys(g, sources=None):
    """Sorted (src, rel, dst) keys of the data edges leaving `sources` (all
    vertices when None)."""
    ro = g.row_offsets.astype(np.int64)
    if sources is None:
        src = np.repeat(np.arange(g.num_vertices, dtype=np.uint64), np.diff(ro))
        rel, dst = g.edge_rel, g.col_targets
    else:
        sources = np.unique(np.asarray(sources, np.int64))
        lens = ro[sources + 1] - ro[sources]
        idx = np.repeat(ro[sources] - np.cumsum(np.concatenate([[0], lens[:-1]])), lens) + np.arange(lens.sum())
        src = np.repeat(sources.astype(np.uint64), lens)
        rel, dst = g.edge_rel[idx], g.col_targets[idx]
    k = (src << np.uint64(32)) | (rel.astype(np.uint64) << np.uint64(24)) | dst.astype(np.uint64)
    return np.unique(k)


def verify_rows(keys, g, q, rows):
    """Every row is injective, keeps bindings/types, and maps every query
    edge onto a data triple (binary search in the sorted triple keys)."""
    if rows.shape[0] == 0:
        return
    r = rows.astype(np.uint64)
    srt = np.sort(rows, axis=1)
    assert (np.diff(srt, axis=1) != 0).all()
    for u in range(q.k):
        if q.vbind[u] != I.UNBOUND:
            assert (rows[:, u] == q.vbind[u]).all()
        if q.vtype[u] != I.ANY:
            assert (g.vertex_type[rows[:, u]] == q.vtype[u]).all()
    for a, b, rel in zip(q.esrc, q.edst, q.erel):
        k = (r[:, a] << np.uint64(32)) | (np.uint64(rel) << np.uint64(24)) | r[:, b]
        pos = np.searchsorted(keys, k)
        assert (pos < keys.size).all() and (keys[np.minimum(pos, keys.size - 1)] == k).all()
    # rows ascend lexicographically
    for i in range(1, min(rows.shape[0], 5000)):
        assert tuple(rows[i - 1]) < tuple(rows[i])


@pytest.fixture(scope="module")
def batch4m():
    w = I.WORKLOADS["batch-4m"]
    g = w.graph()
    qs = w.queries(g)
    return w, g, qs, gs.DeviceGraph(g)


def test_batch_4m_against_oracle_sample(batch4m):
    w, g, qs, dg = batch4m
    b = gs.Batch(dg, qs, cap=w.cap)
    b.run()
    b.finish()
    res = b.fetch()
    b.close()
    assert all(r.status == 0 for r in res)
    og = O.OracleGraph.from_graph(g)
    rng = np.random.default_rng(4)
    sample = sorted(rng.choice(len(qs), 300, replace=False).tolist())
    cnt, fp, st, _ = O.match_many(og, [qs[i] for i in sample], threads=0, time_limit_s=20.0)
    checked = 0
    for j, i in enumerate(sample):
        if st[j] != 0:
            continue
        assert (res[i].count, res[i].fingerprint) == (int(cnt[j]), int(fp[j])), i
        checked += 1
    assert checked >= 250
    for i in sample[:40]:
        o = O.match(og, qs[i], cap=w.cap, time_limit_s=20.0)
        if o.status == 0:
            np.testing.assert_array_equal(res[i].rows, o.rows)


def test_batch_4m_one_at_a_time_equals_batched(batch4m):
    w, g, qs, dg = batch4m
    sub = qs[:200]
    a = gs.match_batch(dg, sub, cap=w.cap)
    b = gs.Batch(dg, sub, cap=w.cap, wave_queries=1)
    b.run()
    b.finish()
    for x, y in zip(a, b.fetch()):
        assert (x.count, x.fingerprint) == (y.count, y.fingerprint)
        np.testing.assert_array_equal(x.rows, y.rows)
    b.close()


def test_stress_shapes_reduced_scale_against_oracle():
    """The stress workload's query shapes and label recipe on a 200k-vertex
    graph with the same average degree (12.5), where the oracle finishes."""
    g = I.make_graph(200_000, 2_500_000, seed=0x6753005)
    qs = I.make_shape_queries(g, 40, seed=0x6753005)
    og = O.OracleGraph.from_graph(g)
    dg = gs.DeviceGraph(g)
    cnt_only = gs.match_batch(dg, qs, cap=0, mode=gs.GS_COUNT_ONLY)
    enum = gs.match_batch(dg, qs, cap=1 << 12)
    cnt, fp, st, _ = O.match_many(og, qs, threads=0, time_limit_s=60.0)
    for i, q in enumerate(qs):
        assert (cnt_only[i].count, cnt_only[i].fingerprint) == (enum[i].count, enum[i].fingerprint)
        if st[i] == 0:
            assert (enum[i].count, enum[i].fingerprint) == (int(cnt[i]), int(fp[i])), i
    for i in range(0, 40, 5):
        o = O.match(og, qs[i], cap=1 << 12, time_limit_s=60.0)
        if o.status == 0:
            np.testing.assert_array_equal(enum[i].rows, o.rows)


def test_stress_16m_count_only_vs_chunked_enumeration():
    w = I.WORKLOADS["stress-16m"]
    g = w.graph()
    qs = w.queries(g)
    dg = gs.DeviceGraph(g)
    sub = qs[::4]  # 50 queries, every shape
    c = gs.match_batch(dg, sub, cap=0, mode=gs.GS_COUNT_ONLY)
    e = gs.match_batch(dg, sub, cap=1 << 16)
    assert sum(x.count for x in c) > 0
    for x, y, q in zip(c, e, sub):
        assert x.status == 0 and y.status == 0
        assert (x.count, x.fingerprint) == (y.count, y.fingerprint)
        assert y.rows.shape[0] == min(y.count, 1 << 16)
        if y.rows.shape[0]:
            keys = triple_keys(g, y.rows[:, np.unique(q.esrc)].ravel())
            verify_rows(keys, g, q, y.rows)
    # GS_CHUNKED on all 200 queries with 64 MB chunks: the number and
    # fingerprint of the streamed rows equal the count-only result of every
    # query, and a sample of every chunk is verified edge by edge.
    call = gs.match_batch(dg, qs, cap=0, mode=gs.GS_COUNT_ONLY)
    n_rows = [0] * len(qs)
    fps = [0] * len(qs)
    rng = np.random.default_rng(5)
    samples = {i: [] for i in range(len(qs))}

    def on_chunk(rows, qi):
        n_rows[qi] += rows.shape[0]
        fps[qi] = (fps[qi] + O.fingerprint(rows)) & 0xFFFFFFFFFFFFFFFF
        pick = rng.choice(rows.shape[0], min(rows.shape[0], 128), replace=False)
        samples[qi].append(rows[pick])

    ch = gs.match_batch(dg, qs, cap=0, mode=gs.GS_CHUNKED, chunk_bytes=64 << 20, on_chunk=on_chunk)
    for i in range(0, len(qs), 3):
        if samples[i]:
            rows = np.concatenate(samples[i])
            rows = rows[np.lexsort(rows.T[::-1])]
            verify_rows(triple_keys(g, rows[:, np.unique(qs[i].esrc)].ravel()), g, qs[i], rows)
    assert sum(x.count for x in call) > 10 ** 7
    for i, (x, z) in enumerate(zip(call, ch)):
        assert x.status == 0 and z.status == 0 and (z.count, z.fingerprint) == (x.count, x.fingerprint)
        assert (n_rows[i], fps[i]) == (x.count, x.fingerprint), i
