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

import numpy as np
import pytest

import graphgen as gg
import oracle

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


def _spread(g, n, seed):
    """g's edges with its vertices placed at random distinct ids of [0, n),
    the last id included, so a graph of n vertices with few edges."""
    rng = np.random.default_rng(seed)
    ids = np.sort(rng.choice(n - 1, size=g.n - 1, replace=False)).astype(np.uint32)
    ids = np.append(ids, np.uint32(n - 1))
    rng.shuffle(ids)
    u, v = gg.to_edge_list(g)
    return gg.from_edges(n, ids[u], ids[v], name=f"{g.name}-in-{n}")


def test_static_plain_count_at_capacity_vs_oracle():
    """n = 4,194,304, the scratch's exact capacity (every upper-start slot of
    the static array in use), and a small graph: the count against the
    CPU oracle's plain edge iterator and Alg. 1 count, two calls in a row."""
    import torch
    import paper_2210_00389_gb300 as tc

    stream = torch.cuda.current_stream()
    for g in (_spread(gg.rmat(14, 16, seed=21), 1 << 22, 5), gg.rmat(9, 8, seed=3)):
        want = oracle.plain_count(g)
        assert want == oracle.cetc(g)["T"]
        off = torch.from_numpy(g.offsets).cuda()
        cols = torch.from_numpy(g.cols).cuda()
        out = torch.empty(1, dtype=torch.int64, device="cuda")
        for _ in range(2):
            out.fill_(-1)
            st = tc._lib.tc_count_plain_static(off.data_ptr(), cols.data_ptr(), g.n, g.nnz,
                                               out.data_ptr(),
                                               ctypes.c_void_p(stream.cuda_stream))
            assert st == tc.TC_OK, tc.tc_last_error()
            torch.cuda.synchronize()
            assert int(out.item()) == want, g.name


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
