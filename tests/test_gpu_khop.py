"""Domain-graph exploration (Ch. 5) on the CUDA engine against the oracle's
breadth-first search: the level array and the per-level counts, exact."""
import numpy as np
import pytest

import oracle as O
import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I
from tests.helpers import random_tiny

pytestmark = pytest.mark.gpu


def check(dg, og, seeds, levels, dirs, rels, ctx=""):
    st, want, wc = O.khop(og, seeds, levels, dirs, rels)
    assert st == 0
    lv, cnt, edges = gs.khop(dg, seeds, levels, dirs, rels)
    np.testing.assert_array_equal(lv, want, err_msg=str(ctx))
    np.testing.assert_array_equal(cnt, wc, err_msg=str(ctx))
    return edges


def test_tiny_instances():
    rng = np.random.default_rng(1234)
    for case in range(80):
        g, _ = random_tiny(rng, n_max=9)
        og, dg = O.OracleGraph.from_graph(g), gs.DeviceGraph(g)
        dirs = int(rng.integers(1, 4))
        rels = None if rng.random() < 0.5 else [r for r in range(g.num_rels) if rng.random() < 0.6]
        seeds = [int(x) for x in rng.choice(g.num_vertices, int(rng.integers(0, 4)), replace=True)]
        check(dg, og, seeds, int(rng.integers(0, 5)), dirs, rels, case)
        dg.free()


@pytest.mark.parametrize("name", ["single-10k", "single-1m"])
def test_workload_graphs(name):
    w = I.WORKLOADS[name]
    g = w.graph()
    og, dg = O.OracleGraph.from_graph(g), gs.DeviceGraph(g)
    rng = np.random.default_rng(9)
    for levels in (0, 1, 3, 4):
        for dirs in (1, 2, 3):
            seeds = rng.choice(g.num_vertices, 16, replace=False)
            check(dg, og, seeds, levels, dirs, None, (name, levels, dirs))
    check(dg, og, rng.choice(g.num_vertices, 64), 4, 3, [0, 1, 2, 3], (name, "rels"))


def test_edge_cases():
    g = I.WORKLOADS["single-10k"].graph()
    og, dg = O.OracleGraph.from_graph(g), gs.DeviceGraph(g)
    lv, cnt, _ = gs.khop(dg, [], 3)
    assert (lv == 255).all() and cnt.tolist() == [0, 0, 0, 0]
    check(dg, og, [5, 5, 5, 7], 2, 3, None, "repeated seeds")
    check(dg, og, [5], 0, 3, None, "no hops")
    with pytest.raises(gs.GSError):
        gs.khop(dg, [g.num_vertices], 2)
    with pytest.raises(gs.GSError):
        gs.khop(dg, [1], 2, rels=[g.num_rels])
    with pytest.raises(gs.GSError):
        gs.khop(dg, [1], 2, directions=4)


def test_device_pointers_match_host_path():
    import torch
    g = I.WORKLOADS["single-10k"].graph()
    dg = gs.DeviceGraph(g)
    seeds = np.array([3, 99, 4321], np.uint32)
    lv, cnt, edges = gs.khop(dg, seeds, 3)
    ts = torch.tensor(seeds.astype(np.int32), device="cuda")
    tl = torch.zeros(g.num_vertices, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    _, cnt2, edges2 = gs.khop(dg, None, 3, device=(ts.data_ptr(), 3, tl.data_ptr()))
    np.testing.assert_array_equal(tl.cpu().numpy(), lv)
    assert cnt2.tolist() == cnt.tolist() and edges2 == edges
    bad = torch.tensor([g.num_vertices], dtype=torch.int32, device="cuda")
    with pytest.raises(gs.GSError):
        gs.khop(dg, None, 3, device=(bad.data_ptr(), 1, tl.data_ptr()))


def test_stress_graph_properties():
    """16M vertices / 200M edges, 4 levels both ways from 16 seeds: every
    vertex at level l + 1 has a neighbour at level l, every neighbour of a
    vertex below the last level is at most one level deeper, and counts
    match the level array (checked on samples of the CSR)."""
    w = I.WORKLOADS["stress-16m"]
    g = w.graph()
    dg = gs.DeviceGraph(g)
    rng = np.random.default_rng(3)
    seeds = rng.choice(g.num_vertices, 16, replace=False)
    lv, cnt, edges = gs.khop(dg, seeds, 4)
    assert cnt.tolist() == [int((lv == l).sum()) for l in range(5)]
    assert (lv[seeds] == 0).all() and cnt[0] == 16
    ro = g.row_offsets.astype(np.int64)
    src = np.repeat(np.arange(g.num_vertices, dtype=np.int64), np.diff(ro))
    dst = g.col_targets.astype(np.int64)
    a, b = lv[src].astype(np.int64), lv[dst].astype(np.int64)
    both = (a != 255) & (b != 255)
    assert (np.abs(a[both] - b[both]) <= 1).all()          # an edge joins levels at most one apart
    assert not ((a < 4) & (b == 255)).any() and not ((b < 4) & (a == 255)).any()  # nothing left unexplored
    parent = np.zeros(g.num_vertices, bool)                 # every non-seed reached vertex has a parent one level up
    m = (a != 255) & (b == a + 1)
    parent[dst[m]] = True
    m = (b != 255) & (a == b + 1)
    parent[src[m]] = True
    reached = (lv != 255) & (lv > 0)
    assert parent[reached].all()
