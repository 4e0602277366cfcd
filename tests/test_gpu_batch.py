"""tc_count_batch against the CPU oracle: every graph's count exact, alone or
in a mix, for every block shape; invalid graphs flagged; graphs too large
for the batch kernel take the single-graph path."""
import os

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


def mixed_graphs():
    gs = [c[0] for c in pins.closed_form_cases()]
    gs += pins.random_small_graphs()
    gs += [gg.rmat(s, ef, seed=500 + s + ef, relabel_seed=(600 + s) if s % 2 else None)
           for s, ef in ((6, 8), (8, 16), (10, 32), (11, 8), (12, 16))]
    gs += [gg.erdos_renyi(300, 10 / 299, 71), gg.complete(25), gg.complete(120)]
    gs += [gg.chung_lu_islands(1 << 12, mean_degree=8, cap=256, seed=9)]
    return gs


def expected(g):
    return oracle.cetc(g)["T"]


def test_batch_mixed_host_views(tc):
    gs = mixed_graphs()
    want = [expected(g) for g in gs]
    for mode in (tc.TC_MODE_COVER, tc.TC_MODE_PLAIN):
        counts, status = tc.tc_count_batch([(g.offsets, g.cols) for g in gs], mode)
        assert (status == tc.TC_OK).all()
        assert counts.tolist() == want


@pytest.mark.parametrize("threads,per_sm", [(128, 8), (256, 4), (512, 2), (256, 1)])
def test_batch_block_shapes(tc, threads, per_sm):
    gs = mixed_graphs()
    want = [expected(g) for g in gs]
    opt = tc.Options(threads, per_sm, 0)
    counts, status = tc.tc_count_batch([(g.offsets, g.cols) for g in gs], tc.TC_MODE_COVER, opt)
    assert (status == tc.TC_OK).all()
    assert counts.tolist() == want


def test_batch_device_views_and_alone_vs_mix(tc):
    import torch
    gs = mixed_graphs()
    dev = [(torch.from_numpy(g.offsets).cuda(), torch.from_numpy(g.cols).cuda()) for g in gs]
    mix, st = tc.tc_count_batch(dev, tc.TC_MODE_COVER)
    assert (st == tc.TC_OK).all()
    for i in (0, 5, len(gs) - 1):
        alone, st1 = tc.tc_count_batch([dev[i]], tc.TC_MODE_COVER)
        assert st1[0] == tc.TC_OK and alone[0] == mix[i] == expected(gs[i])


def test_batch_invalid_and_large(tc):
    good = gg.complete(6)
    bad_cols = good.cols.copy()
    bad_cols[3] = 77                      # column out of range
    unsorted = good.cols.copy()
    unsorted[0], unsorted[1] = unsorted[1], unsorted[0]
    bad_off = good.offsets.copy()
    bad_off[2] = bad_off[3] + 1           # offsets not monotone
    large = gg.rmat(17, 4, seed=3)        # n = 131072 > the batch kernel's limit
    items = [(good.offsets, good.cols), (good.offsets, bad_cols), (good.offsets, unsorted),
             (bad_off, good.cols), (large.offsets, large.cols), (good.offsets, good.cols)]
    counts, status = tc.tc_count_batch(items, tc.TC_MODE_COVER)
    assert status.tolist() == [tc.TC_OK, tc.TC_ERR_INVALID_GRAPH, tc.TC_ERR_INVALID_GRAPH,
                               tc.TC_ERR_INVALID_GRAPH, tc.TC_OK, tc.TC_OK]
    assert counts[0] == counts[5] == 20
    assert counts[4] == oracle.plain_count(large)


@pytest.mark.slow
def test_batch_mixed_recipe_full(tc):
    """The whole 4,096-graph mixed recipe (R-MAT scale 6-14, Erdos-Renyi,
    complete graphs, seed 3) in one call, with the autotuned setting the
    benchmark uses: every count against the oracle (the oracle runs one
    graph per host thread), cover and plain."""
    from concurrent.futures import ThreadPoolExecutor
    specs = gg.mixed_graph_specs(4096, seed=3)
    with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        gs = list(ex.map(gg.graph_from_spec, specs))
        want = list(ex.map(expected, gs))
    items = [(g.offsets, g.cols) for g in gs]
    for mode in (tc.TC_MODE_COVER, tc.TC_MODE_PLAIN):
        counts, status = tc.tc_count_batch(items, mode)
        assert (status == tc.TC_OK).all()
        bad = [i for i, (a, b) in enumerate(zip(counts.tolist(), want)) if a != b]
        assert not bad, f"{len(bad)} graphs differ, first {bad[:5]}"


def test_batch_union_path(tc):
    """Members above the batch kernel's limits are packed into one disjoint
    union and counted together; each count comes from its own range of
    per-edge counts.  Mixed with tiny members, an invalid large member, and an
    edgeless member with many vertices, for both modes and both view kinds."""
    import torch
    big = [gg.rmat(13, 8, seed=41), gg.rmat(14, 16, seed=42, relabel_seed=7),
           gg.chung_lu_islands(1 << 14, mean_degree=12, cap=1024, seed=5),
           gg.complete(200), gg.erdos_renyi(5000, 12 / 4999, 13)]
    assert all(g.nnz > (1 << 15) for g in big)
    bad = big[0].cols.copy()
    bad[100] = big[0].n + 5                               # column out of range
    empty = gg.CSR(70000, np.zeros(70001, dtype=np.int64), np.zeros(0, dtype=np.uint32))
    tiny = [gg.complete(6), gg.wheel(9), gg.rmat(8, 8, seed=4)]
    gs = [big[0], tiny[0], big[1], big[2], tiny[1], big[3], big[4], tiny[2]]
    items = [(g.offsets, g.cols) for g in gs]
    items.insert(3, (big[0].offsets, bad))
    items.append((empty.offsets, empty.cols))
    want = [expected(g) for g in gs]
    want.insert(3, 0)
    want.append(0)
    want_st = [tc.TC_OK] * len(items)
    want_st[3] = tc.TC_ERR_INVALID_GRAPH
    for mode in (tc.TC_MODE_COVER, tc.TC_MODE_PLAIN):
        counts, status = tc.tc_count_batch(items, mode)
        assert status.tolist() == want_st
        assert counts.tolist() == want
        dev = [(torch.from_numpy(o).cuda(), torch.from_numpy(c).cuda()) for o, c in items]
        counts, status = tc.tc_count_batch(dev, mode)
        assert status.tolist() == want_st
        assert counts.tolist() == want


@pytest.mark.parametrize("tiny", [1, 1 << 11, 1 << 17, 1 << 22])
def test_batch_split_threshold(tc, tiny):
    """Any split between the per-graph kernel and the union path gives the
    same exact counts (tiny = 1: nearly everything in the union)."""
    gs = mixed_graphs()
    want = [expected(g) for g in gs]
    for mode in (tc.TC_MODE_COVER, tc.TC_MODE_PLAIN):
        counts, status = tc.tc_count_batch([(g.offsets, g.cols) for g in gs], mode,
                                           tc.Options(256, 2, 0, tiny))
        assert (status == tc.TC_OK).all()
        assert counts.tolist() == want
