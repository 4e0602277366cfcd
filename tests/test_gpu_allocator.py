"""tc_set_allocator with real callbacks: every device allocation of the
library goes through PyTorch's caching allocator (raw blocks on the stream
the library asks for), counted here; the counts stay exact against the
oracle, every block handed out is given back, and the default allocator
works again after the hook is removed."""
import ctypes

import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def test_allocations_through_torch_caching_allocator():
    import torch
    import paper_2210_00389_gb300 as tc

    torch.cuda.init()
    live, stats = {}, {"alloc": 0, "free": 0, "bytes": 0}

    @ALLOC
    def alloc(nbytes, stream, ctx):
        p = torch.cuda.caching_allocator_alloc(max(int(nbytes), 1), stream=int(stream or 0))
        live[p] = int(nbytes)
        stats["alloc"] += 1
        stats["bytes"] += int(nbytes)
        return p

    @FREE
    def free(ptr, stream, ctx):
        assert ptr in live, "freed a block the hook did not hand out"
        del live[ptr]
        torch.cuda.caching_allocator_delete(ptr)
        stats["free"] += 1

    g = gg.rmat(14, 16, seed=5, relabel_seed=6)
    want = oracle.cetc(g)["T"]
    tc.tc_set_allocator(alloc, free)
    try:
        with tc.Graph(g.offsets, g.cols, flags=tc.TC_GRAPH_VALIDATE) as G:
            assert G.count(tc.TC_MODE_COVER) == want
            assert G.count(tc.TC_MODE_PLAIN) == want
            assert int(G.cover_edge_counts().sum()) == want
        torch.cuda.synchronize()
        counts, status = tc.tc_count_batch([(g.offsets, g.cols), (gg.complete(9).offsets,
                                                                  gg.complete(9).cols)],
                                           tc.TC_MODE_COVER)
        assert counts.tolist() == [want, 84] and (status == tc.TC_OK).all()
    finally:
        tc.tc_set_allocator(None, None)
    torch.cuda.synchronize()
    assert stats["alloc"] > 10 and stats["bytes"] >= g.nnz * 4
    assert stats["free"] == stats["alloc"] and not live
    # the default allocator again
    with tc.Graph(g.offsets, g.cols) as G:
        assert G.count(tc.TC_MODE_COVER) == want
    assert stats["alloc"] == stats["free"]
