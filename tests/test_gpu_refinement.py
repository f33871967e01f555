"""Refinement variants (Section 3.3.3 and the refinement experiments of
Section 3.6): no refinement, one query vertex at a time in reversed order,
skipping low-connectivity vertices and the thesis's comparison baseline
(outgoing graph only, spanning-tree exploration) only prune candidates, so every
result equals the oracle's; refined to convergence in either order the
candidate sets are the unique fixpoint, so even the join's partial-embedding
sizes agree."""
import numpy as np
import pytest

import oracle as O
import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I
from tests.helpers import random_tiny

pytestmark = pytest.mark.gpu

VARIANTS = [(0, 64), (gs.GS_REFINE_REVERSED, 64), (gs.GS_REFINE_REVERSED, 1), (gs.GS_REFINE_OFF, 1),
            (gs.GS_REFINE_REVERSED | gs.GS_REFINE_LOW(1), 1), (gs.GS_REFINE_LOW(2), 3), (gs.GS_REFINE_BASELINE, 1)]


def test_variants_on_tiny_instances():
    rng = np.random.default_rng(77)
    for case in range(60):
        g, q = random_tiny(rng, p_any=0.2)
        o = O.OracleGraph.from_graph(g)
        dg = gs.DeviceGraph(g)
        want = O.match(o, q, cap=1 << 16)
        for refine, rounds in VARIANTS:
            r = gs.match_batch(dg, [q], cap=1 << 16, refine=refine, max_refine_rounds=rounds)[0]
            assert r.status == 0 and (r.count, r.fingerprint) == (want.count, want.fingerprint), (case, refine)
            np.testing.assert_array_equal(r.rows, want.rows)
        dg.free()


@pytest.fixture(scope="module")
def small():
    w = I.WORKLOADS["single-10k"]
    g = w.graph()
    return g, w.queries(g), O.OracleGraph.from_graph(g), gs.DeviceGraph(g)


def test_variants_on_workload(small):
    g, qs, og, dg = small
    want = [O.match(og, q, cap=1 << 20) for q in qs]
    sizes = {}
    for refine, rounds in VARIANTS:
        b = gs.Batch(dg, qs, cap=1 << 20, refine=refine, max_refine_rounds=rounds)
        b.run()
        b.finish()
        for i, r in enumerate(b.fetch()):
            assert (r.count, r.fingerprint) == (want[i].count, want[i].fingerprint), (refine, i)
            np.testing.assert_array_equal(r.rows, want[i].rows)
        sizes[(refine, rounds)] = b.join_sizes()
        b.close()
    # the converged sets are the unique fixpoint whatever the order: same join, same sizes
    conv, rev = sizes[(0, 64)], sizes[(gs.GS_REFINE_REVERSED, 64)]
    np.testing.assert_array_equal(conv[0], rev[0])
    np.testing.assert_array_equal(conv[1], rev[1])
    assert (conv[1] <= conv[0]).all() and conv[0].sum() > 0
    # the baseline (outgoing graph only, spanning-tree exploration) never has
    # smaller intermediate results than the converged sets
    base = sizes[(gs.GS_REFINE_BASELINE, 1)]
    assert (base[0] >= conv[0]).all() and base[0].sum() > conv[0].sum()


def test_unknown_refine_flags_rejected(small):
    g, qs, og, dg = small
    r = gs.match_batch(dg, qs[:2], cap=8, refine=1 << 20)
    assert all(x.status == gs.GS_ERR_INVALID for x in r)
