"""Triangle finding with the cover edges (Alg. 1 / Thm. 2): per-vertex
counts against the oracle's enumerated triangles and closed forms; the list
of triangles equals the oracle's set, each triangle once, each at the cover
edge and apex the count-once rule assigns it to."""
from math import comb

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    torch.cuda.init()
    import paper_2210_00389_gb300 as tc
    return tc


def per_vertex_from(tri, n):
    t = np.zeros(n, dtype=np.uint64)
    for col in range(3):
        np.add.at(t, tri[:, col].astype(np.int64), 1)
    return t


def check(tc, g):
    tri = oracle.triangles(g)
    L, _ = oracle.bfs_levels(g, None)
    with tc.Graph(g.offsets, g.cols, n=g.n) as G:
        pv = G.vertex_counts()
        lst = G.list_triangles()
    assert np.array_equal(pv, per_vertex_from(tri, g.n)), g.name
    assert len(lst) == len(tri), g.name
    if len(lst):
        u, v, w = (lst[:, k].astype(np.int64) for k in range(3))
        # (u, v) a cover edge, w an apex the count-once rule accepts
        assert np.all(u < v) and np.all(L[u] == L[v])
        assert np.all((L[w] != L[u]) | (w > v))
        # the same triangles as the oracle's, each once
        got = np.sort(lst, axis=1)
        got = got[np.lexsort(got.T[::-1])]
        want = tri[np.lexsort(tri.T[::-1])]
        assert np.array_equal(got, want), g.name
    return pv


def test_closed_forms(tc):
    pv = check(tc, gg.complete(12))
    assert (pv == comb(11, 2)).all()
    pv = check(tc, gg.wheel(40))
    assert int(pv.max()) == 40 and (np.sort(pv)[:-1] == 2).all()
    pv = check(tc, gg.friendship(9))
    assert int(pv.max()) == 9 and int((pv == 1).sum()) == 18
    assert not check(tc, gg.star(30)).any()
    assert not check(tc, gg.grid(7, 9)).any()


def test_random_and_generated(tc):
    for g in pins.random_small_graphs()[:20]:
        check(tc, g)
    check(tc, gg.rmat(10, 16, seed=1))
    check(tc, gg.rmat(12, 16, seed=77, relabel_seed=5))
    check(tc, gg.chung_lu_islands(1 << 13, mean_degree=10, cap=512, seed=4))
    check(tc, gg.disjoint_union(gg.complete(200), gg.wheel(2049), gg.star(1500), gg.empty(7)))


def test_capacity_and_device_output(tc):
    import torch
    g = gg.complete(10)
    with tc.Graph(g.offsets, g.cols, n=g.n) as G:
        out = np.zeros((5, 3), dtype=np.uint32)
        cnt = tc.ctypes.c_int64(0)
        st = tc._lib.tc_list_triangles(G.handle, out.ctypes.data, 5, tc.ctypes.byref(cnt))
        assert st == tc.TC_ERR_CAPACITY and cnt.value == comb(10, 3)
        assert not out.any()  # nothing written
        dev = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        G.vertex_counts(dev)
        assert (dev.cpu().numpy() == comb(9, 2)).all()
