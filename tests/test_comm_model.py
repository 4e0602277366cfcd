"""Comm-CETC communication model (Sec. III-B) and the size fits (Sec. IV-A),
pinned to the values the paper prints in its communication table and text:
RMAT-36 (p = 128, k = 0.311, 2.73e16 wedges): previous 218 PB, this paper
192 TB, reduction 1156; RMAT-42 (p = 256, k = 0.260, 5.79e18 wedges): 52.8 EB,
22.8 PB, 2368; k = 0.260 at scale 42 from the fit; triangles 1.20e14 and
1.30e16 from the fit.  The paper's own rounding (and its k = 0.311 at scale
36, where the fit gives 0.322) leaves differences below 1%."""
import math

import pytest

from paper_2210_00389_gb300 import comm


def rel(a, b):
    return abs(a - b) / abs(b)


def test_rmat36_row():
    r = comm.rmat_row(36, 0.311, 128, 2.73e16)
    assert rel(r["previous_bytes"] / comm.PB, 218) < 0.01
    assert rel(r["this_bytes"] / comm.TB, 192) < 0.01
    assert rel(r["reduction"], 1156) < 0.01


def test_rmat42_row():
    r = comm.rmat_row(42, 0.260, 256, 5.79e18)
    assert rel(r["previous_bytes"] / comm.EB, 52.8) < 0.01
    assert rel(r["this_bytes"] / comm.PB, 22.8) < 0.01
    assert rel(r["reduction"], 2368) < 0.01


def test_fits():
    assert round(comm.k_fit(42), 3) == 0.260
    assert rel(comm.k_fit(36), 0.311) < 0.04      # the table's 0.311 vs the fit's 0.322
    assert rel(comm.triangles_fit(2 ** 36), 1.20e14) < 0.01
    assert rel(comm.triangles_fit(2 ** 42), 1.30e16) < 0.01


def test_formula_terms():
    # p = 1, k = 0: only the BFS term and no reduction
    n, m = 1 << 20, 1 << 24
    assert comm.comm_cetc_bits(n, m, 0.0, 1, 3) == m * (3 + 3 * 20)
    # each processor more adds k m ceil(log n) + ceil(log n) bits
    d = comm.comm_cetc_bits(n, m, 0.5, 9, 3) - comm.comm_cetc_bits(n, m, 0.5, 8, 3)
    assert d == pytest.approx(0.5 * m * 20 + 20)
    assert comm.wedges_exact([0, 1, 2, 3, 4]) == 0 + 0 + 1 + 3 + 6
    assert comm.clog2(1) == 0 and comm.clog2(2 ** 36) == 36 and comm.clog2(2 ** 36 + 1) == 37


def _cut_brute(g, bounds):
    part = {}
    for i in range(len(bounds) - 1):
        for v in range(bounds[i], bounds[i + 1]):
            part[v] = i
    c = 0
    for u in range(g.n):
        for v in g.cols[g.offsets[u]:g.offsets[u + 1]]:
            c += part[u] != part[int(v)]
    return c


@pytest.mark.parametrize("p", [2, 4, 8])
def test_measured_volume_small(p):
    """The counted volumes of Comm-CETC on p virtual processors (Alg. 2,
    Sec. III-B) on R-MAT scale 10 and 11, against a brute-force count of the
    cut edge traversals and the model's terms: the exchange term is the
    model's times (p - 1) / p exactly (the model charges p transfers per
    cover edge, Alg. 2 makes p - 1); the BFS term is 2 x (cut fraction) x
    the model's (the model charges every one of the m edges as one remote
    traversal), so measured / model stays within [0.5, 1.5] for p >= 2 on
    these graphs (stated tolerance)."""
    import graphgen as gg
    import oracle
    for scale in (10, 11):
        g = gg.rmat(scale, 16, seed=scale, relabel_seed=scale + 2 ** 32)
        L, nl = oracle.bfs_levels(g)
        h = oracle.num_cover(g, L)
        r = comm.measured_volume(g.offsets, g.cols, h, nl, p)
        b = comm.vertex_partition(g.offsets, p)
        assert b[0] == 0 and b[-1] == g.n and all(b[i] <= b[i + 1] for i in range(p))
        # each part holds about 2m/p endpoints (within one vertex's degree)
        ends = [int(g.offsets[b[i + 1]] - g.offsets[b[i]]) for i in range(p)]
        assert max(ends) - min(ends) <= 2 * int(g.degrees().max()) + 2
        assert r["cut_directed_traversals"] == _cut_brute(g, b)
        assert r["exchange_bits"] == pytest.approx(r["model_exchange_bits"] * (p - 1) / p)
        frac = r["cut_directed_traversals"] / g.nnz
        assert r["bfs_bits"] == pytest.approx(2 * frac * r["model_bfs_bits"])
        assert 0.5 <= r["measured_bits"] / r["model_bits"] <= 1.5
