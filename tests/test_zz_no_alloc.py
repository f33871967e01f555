"""gs_filter_candidates_static: the candidate filter for callers that must
not let the library allocate device memory (its scratch is a fixed array
inside the library).  Its output must equal the allocating inspection entry
point's, call after call; this file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import paper_1807_08804_gb300 as gs
from paper_1807_08804_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_static_filter_equals_allocating_filter_twice():
    import torch

    w = I.WORKLOADS["single-10k"]
    g = w.graph()
    qs = w.queries(g, 12)
    dg = gs.DeviceGraph(g)
    cap = g.num_vertices
    ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    count = torch.empty(1, dtype=torch.int64, device="cuda")
    L = gs.lib()
    checked = 0
    wants = [gs.inspect_candidates(dg, q, gs.GS_STAGE_FILTER) for q in qs]  # allocating reference, first
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for q, want in zip(qs, wants):
        pack = gs._QueryPack([q])
        for u in range(q.k):
            for call in range(2):  # two calls in a row share the scratch
                ids.fill_(-1)
                count.fill_(-1)
                st = L.gs_filter_candidates_static(dg._h, pack.arr, u, ctypes.c_void_p(ids.data_ptr()), cap,
                                                   ctypes.c_void_p(count.data_ptr()), None)
                assert st == gs.GS_OK, L.gs_last_error()
                torch.cuda.synchronize()
                n = int(count.item())
                got = ids[:n].cpu().numpy().astype(np.uint32)
                assert n == want[u].shape[0], (u, call)
                np.testing.assert_array_equal(got, want[u])
                checked += 1
    assert checked >= 2 * 12 * 3
    # the calls allocated nothing: the device's free memory did not move
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # a short output buffer: the count stays exact, only cap_ids ids are written
    q = qs[0]
    u = int(np.argmax([x.shape[0] for x in gs.inspect_candidates(dg, q, gs.GS_STAGE_FILTER)]))
    want = gs.inspect_candidates(dg, q, gs.GS_STAGE_FILTER)[u]
    ids.fill_(-1)
    pack = gs._QueryPack([q])
    st = L.gs_filter_candidates_static(dg._h, pack.arr, u, ctypes.c_void_p(ids.data_ptr()), 3,
                                       ctypes.c_void_p(count.data_ptr()), None)
    assert st == gs.GS_OK
    torch.cuda.synchronize()
    assert int(count.item()) == want.shape[0]
    np.testing.assert_array_equal(ids[:min(3, want.shape[0])].cpu().numpy().astype(np.uint32), want[:3])
    if want.shape[0] > 3:
        assert int(ids[3].item()) == -1
    # invalid arguments are rejected before any work
    assert L.gs_filter_candidates_static(dg._h, pack.arr, q.k, ctypes.c_void_p(ids.data_ptr()), cap,
                                         ctypes.c_void_p(count.data_ptr()), None) == gs.GS_ERR_INVALID
    dg.free()
