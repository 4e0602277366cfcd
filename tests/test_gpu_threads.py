"""Calls on one tc_graph from several host threads at once: the graph's
lock runs them one after another, and every result is the oracle's."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def test_one_graph_many_threads():
    import torch
    import paper_2210_00389_gb300 as tc

    torch.cuda.init()
    g = gg.rmat(15, 16, seed=8, relabel_seed=9)
    ref = oracle.cetc(g)
    want_c = oracle.cetc_edge_counts(g, ref["levels"], ref["H"])
    with tc.Graph(g.offsets, g.cols) as G:
        def work(i):
            if i % 4 == 0:
                return ("T", G.count(tc.TC_MODE_COVER))
            if i % 4 == 1:
                return ("P", G.count(tc.TC_MODE_PLAIN))
            if i % 4 == 2:
                return ("C", G.cover_edge_counts())
            G.invalidate()  # drops the cached levels and H mid-stream
            return ("T", G.count(tc.TC_MODE_COVER))
        with ThreadPoolExecutor(8) as ex:
            out = list(ex.map(work, range(32)))
    for kind, v in out:
        if kind == "C":
            assert np.array_equal(v, want_c)
        else:
            assert v == ref["T"]
