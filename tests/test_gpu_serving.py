"""The serving loop (continuous batching): every result is identical alone
and in the mix, including requests that arrive while others run."""
import time

import numpy as np
import pytest

import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def drain(srv, tickets, timeout_s=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        assert time.time() - t0 < timeout_s, "serving did not finish in time"
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        time.sleep(0.0005)
    return out


@pytest.fixture(scope="module")
def setup():
    w = I.WORKLOADS["single-10k"]
    g = w.graph()
    qs = I.make_walk_queries(g, 300, 3, 8, p_bind=0.2, seed=11)
    dg = gs.DeviceGraph(g)
    alone = gs.match_batch(dg, qs, cap=1 << 16)
    return g, qs, dg, alone


def test_served_results_equal_alone(setup):
    g, qs, dg, alone = setup
    srv = gs.Server(dg, slots=3, max_batch=32)
    rng = np.random.default_rng(3)
    order = rng.permutation(len(qs))
    tickets = {}
    for j, i in enumerate(order):  # arrivals spread out so batches overlap
        tickets[srv.submit(qs[i], cap=1 << 16)] = i
        if j % 17 == 0:
            time.sleep(0.001)
    res = drain(srv, list(tickets))
    for t, (r, lat) in res.items():
        a = alone[tickets[t]]
        assert r.status == 0 and lat > 0
        assert (r.count, r.fingerprint) == (a.count, a.fingerprint)
        np.testing.assert_array_equal(r.rows, a.rows)
    srv.close()


def test_serving_small_budget_still_progresses(setup):
    g, qs, dg, alone = setup
    srv = gs.Server(dg, budget_bytes=1 << 20, slots=2, max_batch=8)  # admits little at a time
    tickets = {srv.submit(q, cap=1 << 16): i for i, q in enumerate(qs[:60])}
    res = drain(srv, list(tickets))
    for t, (r, _) in res.items():
        a = alone[tickets[t]]
        assert (r.count, r.fingerprint) == (a.count, a.fingerprint)
    srv.close()


def test_serving_rejects_bad_queries_and_unknown_tickets(setup):
    g, qs, dg, alone = setup
    srv = gs.Server(dg)
    bad = I.Query(np.array([I.ANY, I.ANY], np.uint32), np.array([I.UNBOUND] * 2, np.uint32),
                  np.array([0], np.uint32), np.array([0], np.uint32), np.array([0], np.uint32))
    with pytest.raises(gs.GSError):
        srv.submit(bad)
    with pytest.raises(gs.GSError):
        srv.poll(10 ** 9)
    t = srv.submit(qs[0], cap=1 << 16)
    r, _ = drain(srv, [t])[t]
    assert (r.count, r.fingerprint) == (alone[0].count, alone[0].fingerprint)
    srv.close()
