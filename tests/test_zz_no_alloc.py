"""tc_count_plain_static: the allocation-free plain count, for callers that
cannot call cudaMalloc/cudaFree where they need a count (the allocator calls
can synchronize the device, and some applications own or budget all device
memory up front).

The entry point is called through the C ABI on device buffers the test
allocates, twice in a row (its static scratch keeps the previous call's
contents), and must give the same count as the existing tc_count entry
point.  Counts are exact integers, so the tolerance is zero, as in every
other parity test.  This file is collected last on purpose.
"""
import ctypes

import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


def test_static_plain_count_matches_tc_count():
    import torch
    import paper_2210_00389_gb300 as tc

    lib = tc._lib
    stream = torch.cuda.current_stream()
    graphs = [gg.rmat(14, 16, seed=11, relabel_seed=12),
              gg.disjoint_union(gg.complete(40), gg.empty(3), gg.wheel(9))]
    for g in graphs:
        with tc.Graph(g.offsets, g.cols) as G:
            want = G.count(tc.TC_MODE_PLAIN)
            assert want == G.count(tc.TC_MODE_COVER)
        off = torch.from_numpy(g.offsets).cuda()
        cols = torch.from_numpy(g.cols).cuda()
        out = torch.empty(1, dtype=torch.int64, device="cuda")
        for _ in range(2):
            out.fill_(-1)
            st = lib.tc_count_plain_static(off.data_ptr(), cols.data_ptr(), g.n, g.nnz,
                                           out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert st == tc.TC_OK, tc.tc_last_error()
            torch.cuda.synchronize()
            assert int(out.item()) == want


def test_static_plain_count_rejects_oversized_graphs():
    import torch
    import paper_2210_00389_gb300 as tc

    out = torch.empty(1, dtype=torch.int64, device="cuda")
    dummy = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = tc._lib.tc_count_plain_static(dummy.data_ptr(), None, (1 << 22) + 1, 0,
                                       out.data_ptr(), None)
    assert st == tc.TC_ERR_CAPACITY
    assert "static scratch limit" in tc.tc_last_error()
    # binding wrapper raises the same error
    with pytest.raises(tc.TCError):
        tc.tc_count_plain_static(torch.zeros((1 << 22) + 2, dtype=torch.int64, device="cuda"),
                                 torch.zeros(0, dtype=torch.uint32, device="cuda"), out)
