"""The library's multi-level compression (host code, no device needed)
equals the oracle's: the node of every vertex, every weighted edge with both
weights, and every node weight, on tiny random graphs, graphs with twins and
the seeded 10,000-vertex graph."""
import numpy as np
import pytest

import oracle as O
import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I
from tests.helpers import random_tiny
from tests.test_oracle_compression import deltas, twin_tiny


def same_compression(g, ds):
    lib = gs.compress_host(g, ds)
    w = O.WeightedGraph(O.OracleGraph.from_graph(g), ds)
    assert lib["nodes"] == w.n
    np.testing.assert_array_equal(lib["group"], w.group)
    for k in ("src", "rel", "dst", "wout", "win"):
        np.testing.assert_array_equal(lib[k], getattr(w, k), err_msg=k)
    np.testing.assert_array_equal(lib["wnode"], w.wnode)
    return w


@pytest.mark.parametrize("maker", [random_tiny, twin_tiny])
def test_library_compression_equals_oracle_on_tiny_graphs(maker):
    rng = np.random.default_rng(401 if maker is random_tiny else 402)
    for _ in range(500):
        g, _ = maker(rng)
        same_compression(g, deltas(rng))


@pytest.mark.parametrize("ds", [[1.0], [0.5], [1.0, 0.5, 0.3], [0.3, 0.3]])
def test_library_compression_equals_oracle_on_10k_graph(ds):
    same_compression(I.WORKLOADS["single-10k"].graph(), ds)


def test_library_compression_equals_oracle_on_concept_families():
    """The compression workload's 10,000-vertex graph at the thesis's
    thresholds: every level merges, as on SenticNet."""
    w = I.WORKLOADS["compress-10k"]
    g = w.graph()
    prev = g.num_vertices
    for levels in (1, 2, 3):
        ow = same_compression(g, w.deltas[:levels])
        assert ow.n < prev
        prev = ow.n
    assert ow.ratio() < 0.8


def test_invalid_compression_arguments_are_rejected():
    g = I.make_graph(100, 400, seed=3)
    for ds in ([0.0], [1.5], [float("nan")]):
        with pytest.raises(gs.GSError) as e:
            gs.compress_host(g, ds)
        assert e.value.status == gs.GS_ERR_INVALID
    bad = I.Graph(g.num_vertices, g.row_offsets, g.col_targets.copy(), g.edge_rel, g.vertex_type, g.num_types,
                  g.num_rels)
    bad.col_targets[5] = 100
    with pytest.raises(gs.GSError):
        gs.compress_host(bad, [1.0])
