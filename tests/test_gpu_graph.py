"""Graph canonicalisation on the device (Section 3.3.1's node and edge
arrays, in both directions as Section 3.5 asks), element by element against
a construction in numpy: every CSR plane (out and in rows sorted by
(relation, neighbour) with repeated triples dropped; out and in rows of
distinct neighbours over all relations) and every 4-bit degree signature."""
import numpy as np
import pytest

import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I
from tests.helpers import graph_from_triples

pytestmark = pytest.mark.gpu


def host_planes(g):
    V, R = g.num_vertices, g.num_rels
    src = np.repeat(np.arange(V, dtype=np.uint64), np.diff(g.row_offsets.astype(np.int64)))
    t = np.unique(np.stack([src, g.edge_rel.astype(np.uint64), g.col_targets.astype(np.uint64)], 1), axis=0)
    s, r, d = t[:, 0], t[:, 1], t[:, 2]

    def csr(row, key):
        order = np.lexsort((key, row))
        off = np.zeros(V + 1, np.uint64)
        np.add.at(off, row.astype(np.int64) + 1, 1)
        return np.cumsum(off).astype(np.uint64), key[order].astype(np.uint32)

    planes = [csr(s, (r << 24) | d), csr(d, (r << 24) | s)]
    for row, nb in ((s, d), (d, s)):
        pairs = np.unique(np.stack([row, nb], 1), axis=0) if len(row) else np.zeros((0, 2), np.uint64)
        planes.append(csr(pairs[:, 0], pairs[:, 1]))
    sig = np.zeros((2 * R + 2, V), np.int64)
    np.add.at(sig, (r.astype(np.int64), s.astype(np.int64)), 1)
    np.add.at(sig, (R + r.astype(np.int64), d.astype(np.int64)), 1)
    sig[2 * R] = np.diff(planes[2][0].astype(np.int64))
    sig[2 * R + 1] = np.diff(planes[3][0].astype(np.int64))
    return planes, np.minimum(sig, 15).astype(np.uint8)


@pytest.mark.parametrize("name", ["tiny", "single-10k", "compress-10k"])
def test_device_canonical_graph_equals_host_construction(name):
    if name == "tiny":  # repeated triples, a self-loop, several relations between one pair
        tr = [(0, 1, 2), (0, 1, 2), (0, 0, 2), (2, 2, 2), (3, 1, 0), (1, 0, 3), (1, 2, 3), (3, 1, 0), (2, 0, 1)]
        g = graph_from_triples(4, [(a, r, b) for a, r, b in tr], [0, 1, 0, 1], 2, 3)
    else:
        g = I.WORKLOADS[name].graph()
    planes, sig = host_planes(g)
    dg = gs.DeviceGraph(g)
    for p in range(4):
        off, adj = dg.export(p)
        np.testing.assert_array_equal(off, planes[p][0], err_msg=f"plane {p} offsets")
        np.testing.assert_array_equal(adj, planes[p][1], err_msg=f"plane {p} rows")
    _, _, dsig = dg.export(0, signatures=True)
    np.testing.assert_array_equal(dsig, sig)
    assert dg.num_edges == len(planes[0][1])
    dg.free()
