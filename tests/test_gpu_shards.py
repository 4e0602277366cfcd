"""Virtual shards on one GPU: the slices of tc_shard_bounds, counted by
tc_count_range, add up to the oracle's T; each cover slice equals the sum
of the oracle's per-edge counts over the same cover edges."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    torch.cuda.init()
    import paper_2210_00389_gb300 as tc
    return tc


GRAPHS = [
    lambda: gg.complete(40),
    lambda: gg.wheel(300),
    lambda: gg.rmat(14, 16, seed=21, relabel_seed=22),
    lambda: gg.chung_lu_islands(1 << 15, mean_degree=12, cap=1024, seed=3),
    lambda: gg.disjoint_union(gg.star(1500), gg.complete(60), gg.empty(10)),
]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_virtual_shards(tc, gi):
    g = GRAPHS[gi]()
    L, _ = oracle.bfs_levels(g, None)
    H = oracle.cover_edges(g, L)
    T = oracle.cetc_count(g, L)
    per = oracle.cetc_edge_counts(g, L, H) if len(H) else np.zeros(0, np.int64)
    with tc.Graph(g.offsets, g.cols, n=g.n) as G:
        for P in (1, 2, 3, 7, 64):
            for mode, m in ((tc.TC_MODE_COVER, len(H)), (tc.TC_MODE_PLAIN, g.nnz)):
                b = G.shard_bounds(mode, P)
                assert len(b) == P + 1 and b[0] == 0 and b[-1] == m
                assert np.all(np.diff(b) >= 0)
                assert all(x % 4096 == 0 or x == m for x in b[1:-1])
                parts = [G.count_range(mode, int(b[k]), int(b[k + 1])) for k in range(P)]
                assert sum(parts) == T, (mode, P)
                if mode == tc.TC_MODE_COVER:
                    assert parts == [int(per[b[k]:b[k + 1]].sum()) for k in range(P)]


def test_ranges_and_errors(tc):
    g = gg.rmat(11, 16, seed=9, relabel_seed=10)
    L, _ = oracle.bfs_levels(g, None)
    H = oracle.cover_edges(g, L)
    per = oracle.cetc_edge_counts(g, L, H)
    with tc.Graph(g.offsets, g.cols, n=g.n) as G:
        # arbitrary, unaligned cover ranges against the oracle's per-edge sums
        rng = np.random.default_rng(5)
        for _ in range(10):
            a, c = sorted(rng.integers(0, len(H) + 1, size=2))
            assert G.count_range(tc.TC_MODE_COVER, int(a), int(c)) == int(per[a:c].sum())
        assert G.count_range(tc.TC_MODE_COVER, 7, 7) == 0
        # plain ranges split anywhere add up to the total
        cuts = [0, 1, 333, 4097, g.nnz // 2, g.nnz]
        assert sum(G.count_range(tc.TC_MODE_PLAIN, cuts[k], cuts[k + 1])
                   for k in range(len(cuts) - 1)) == oracle.plain_count(g)
        for bad in ((-1, 5), (5, 4), (0, len(H) + 1)):
            with pytest.raises(tc.TCError):
                G.count_range(tc.TC_MODE_COVER, *bad)
        with pytest.raises(tc.TCError):
            G.shard_bounds(tc.TC_MODE_COVER, 0)
        with pytest.raises(tc.TCError):
            G.count_range(7, 0, 1)


def test_count_sharded_single_process(tc):
    """The multi-GPU driver with world size P emulated by P calls in one
    process (the all-reduce sums the P partial counts)."""
    from paper_2210_00389_gb300.shard import count_sharded
    g = gg.rmat(12, 16, seed=31, relabel_seed=32)
    T = oracle.plain_count(g)
    with tc.Graph(g.offsets, g.cols, n=g.n) as G:
        for mode in (tc.TC_MODE_COVER, tc.TC_MODE_PLAIN):
            P = 4
            locals_ = [count_sharded(G, mode, r, P, lambda x: x)[0] for r in range(P)]
            assert sum(locals_) == T


@pytest.mark.parametrize("mode_name", ["cover", "plain"])
def test_shard_balance_rmat18(tc, mode_name):
    """Slices of tc_shard_bounds balance the intersection's real work: on
    R-MAT scale 18 (relabelled) with 8 virtual shards, the list elements each
    slice's count handles (counted by the kernels) stay within 1.35x of the
    mean, and the slices add up to the oracle's T."""
    g = gg.rmat(18, 16, seed=2, relabel_seed=2 + 2**32)
    T = oracle.cetc_count_mt(g, oracle.bfs_levels(g)[0])
    mode = tc.TC_MODE_COVER if mode_name == "cover" else tc.TC_MODE_PLAIN
    P = 8
    with tc.Graph(g.offsets, g.cols, n=g.n) as G:
        b = G.shard_bounds(mode, P)
        parts, elems = [], []
        for k in range(P):
            parts.append(G.count_range(mode, int(b[k]), int(b[k + 1])))
            elems.append(G.stats()["list_elems"])
    assert sum(parts) == T
    assert max(elems) <= 1.35 * (sum(elems) / P), elems
