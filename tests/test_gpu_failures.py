"""Failure paths, provoked on the host side only (no kernel is made to fault):

- the prefix scans' bounded look-back wait runs out (the first tile of every
  multi-tile scan withholds its state, a flag nothing else sets) and the run
  reports GS_ERR_TIMEOUT, while the scans stay exact and the batch stays
  usable;
- a device allocation fails (a simulated out-of-memory at every allocation of
  a graph load, a batch and a serving slot in turn): GS_ERR_OOM, nothing left
  allocated, and the library still works afterwards;
- the serving worker's completion check reports a CUDA error: the affected
  requests complete with GS_ERR_CUDA, the others are exact, and destroy
  returns; a ticket already collected is rejected.
"""
import time

import numpy as np
import pytest

import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LEAK_SLACK = 4 << 20  # bytes of free-memory drift tolerated (driver bookkeeping)


@pytest.fixture(scope="module")
def setup():
    import torch
    torch.cuda.set_device(0)
    w = I.WORKLOADS["single-10k"]
    g = w.graph()
    qs = I.make_walk_queries(g, 64, 3, 6, p_bind=0.0, seed=21)
    dg = gs.DeviceGraph(g)
    want = gs.match_batch(dg, qs, cap=1 << 12)
    return g, qs, dg, want


@pytest.fixture(scope="module")
def wide(setup):
    """Three-vertex paths of untyped, unbound vertices: every candidate set
    holds thousands of vertices, so the scans over edge-table keys and join
    rows span many 2,048-count tiles."""
    g, qs, dg, want = setup
    paths = []
    for q in I.make_walk_queries(g, 8, 3, 3, p_close=0.0, p_bind=0.0, seed=22):
        paths.append(I.Query(np.full(q.k, I.ANY, np.uint32), np.full(q.k, I.UNBOUND, np.uint32), q.esrc, q.edst,
                             q.erel))
    return paths, gs.match_batch(dg, paths, cap=1 << 12)


def same(a, b):
    return all((x.count, x.fingerprint) == (y.count, y.fingerprint) and np.array_equal(x.rows, y.rows)
               for x, y in zip(a, b))


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_scan_wait_bound_reports_timeout_and_stays_exact(setup, wide):
    g, _, dg, _ = setup
    qs, want = wide
    assert sum(r.count for r in want) > 10_000
    for use_graph in (True, False):
        b = gs.Batch(dg, qs, cap=1 << 12)
        b.configure(use_graph=use_graph, group=32, refine_rounds=2)
        b.run()
        b.finish()
        assert same(b.fetch(), want)
        b.set_wait(64, withhold_first_tile=True)
        b.run()
        with pytest.raises(gs.GSError) as e:
            b.finish()
        assert e.value.status == gs.GS_ERR_TIMEOUT
        # the record is cleared by the finish that reported it, and the
        # scans were exact throughout: the next normal run is clean
        b.set_wait(0, withhold_first_tile=False)
        b.run()
        b.finish()
        assert same(b.fetch(), want)
        b.close()


def test_scan_wait_bound_without_withholding_is_not_hit(setup):
    g, qs, dg, want = setup
    b = gs.Batch(dg, qs, cap=1 << 12)
    b.set_wait(1 << 20)
    for _ in range(3):
        b.run()
        b.finish()
        assert same(b.fetch(), want)
    b.close()


def test_allocation_failure_in_batch_creation(setup):
    g, qs, dg, want = setup
    gs.Batch(dg, qs, cap=1 << 12).close()  # warm: library-lifetime state exists
    free0 = free_bytes()
    failures = 0
    for after in range(200):
        gs.debug_fail_alloc(after)
        try:
            b = gs.Batch(dg, qs, cap=1 << 12)
        except gs.GSError as e:
            assert e.status == gs.GS_ERR_OOM, (after, e)
            failures += 1
            continue
        gs.debug_fail_alloc(-1)
        b.run()
        b.finish()
        assert same(b.fetch(), want)
        b.close()
        break
    else:
        pytest.fail("batch creation never succeeded")
    gs.debug_fail_alloc(-1)
    assert failures >= 5  # every allocation of a batch was made to fail in turn
    assert abs(free_bytes() - free0) <= LEAK_SLACK


def test_allocation_failure_in_graph_load(setup):
    g, qs, dg, want = setup
    free0 = free_bytes()
    failures = 0
    for after in range(200):
        gs.debug_fail_alloc(after)
        try:
            d2 = gs.DeviceGraph(g)
        except gs.GSError as e:
            assert e.status == gs.GS_ERR_OOM, (after, e)
            failures += 1
            continue
        gs.debug_fail_alloc(-1)
        assert same(gs.match_batch(d2, qs, cap=1 << 12), want)
        d2.free()
        break
    else:
        pytest.fail("graph load never succeeded")
    gs.debug_fail_alloc(-1)
    assert failures >= 10
    assert abs(free_bytes() - free0) <= LEAK_SLACK


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


def test_serving_completion_error_fails_only_its_micro_batch(setup):
    g, qs, dg, want = setup
    srv = gs.Server(dg, slots=2, max_batch=8)
    gs.debug_fail_serve_wait(1)
    tickets = {srv.submit(q, cap=1 << 12): i for i, q in enumerate(qs)}
    res = drain(srv, list(tickets))
    gs.debug_fail_serve_wait(0)
    failed = 0
    for t, (r, lat) in res.items():
        if r.status == gs.GS_ERR_CUDA:
            failed += 1
            continue
        a = want[tickets[t]]
        assert r.status == 0 and (r.count, r.fingerprint) == (a.count, a.fingerprint)
        np.testing.assert_array_equal(r.rows, a.rows)
    assert 1 <= failed <= 8  # one micro-batch of at most max_batch requests
    # the server keeps serving after the failure
    t2 = srv.submit(qs[0], cap=1 << 12)
    r, _ = drain(srv, [t2])[t2]
    assert r.status == 0 and r.count == want[0].count
    # a ticket already collected is rejected instead of staying "not ready"
    with pytest.raises(gs.GSError) as e:
        srv.poll(t2)
    assert e.value.status == gs.GS_ERR_INVALID
    srv.close()  # returns: no slot is left busy


def test_serving_allocation_failure_completes_requests_with_oom(setup):
    g, qs, dg, want = setup
    srv = gs.Server(dg, slots=1, max_batch=8)
    gs.debug_fail_alloc(0)  # the slot's first batch cannot allocate
    tickets = {srv.submit(q, cap=1 << 12): i for i, q in enumerate(qs[:16])}
    res = drain(srv, list(tickets))
    gs.debug_fail_alloc(-1)
    st = [r.status for r, _ in res.values()]
    assert st.count(gs.GS_ERR_OOM) >= 1
    for t, (r, _) in res.items():
        if r.status == 0:
            assert r.count == want[tickets[t]].count
    srv.close()
