"""Independent checks ("pins") for the CPU oracle.

None of these computes its expected value with the oracle: they use brute
force over vertex triples, the matrix identity trace(A^3) = 6T, scipy's
breadth-first shortest paths, closed forms, and the paper's Lemma 1 /
Lemma 2 / Thm. 2 restated as properties of the oracle's outputs.  The
functions take an oracle object so a deliberately broken oracle build can be
run through the same checks (tests/test_oracle_mutants.py).
"""
from __future__ import annotations

from math import comb

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components, shortest_path

import graphgen as gg


def dense(g) -> np.ndarray:
    A = np.zeros((g.n, g.n), dtype=np.int64)
    rows = np.repeat(np.arange(g.n), np.diff(g.offsets))
    A[rows, g.cols.astype(np.int64)] = 1
    return A


def brute_force_triangles(g) -> list[tuple[int, int, int]]:
    """Every triple a < b < c with all three edges present (Omega(n^3))."""
    A = dense(g).astype(bool)
    out = []
    for a in range(g.n):
        for b in range(a + 1, g.n):
            if not A[a, b]:
                continue
            for c in range(b + 1, g.n):
                if A[a, c] and A[b, c]:
                    out.append((a, b, c))
    return out


def trace_count(g) -> int:
    """T = trace(A^3) / 6 (the matrix formulation, Sec. V-A)."""
    A = dense(g)
    t = int(np.trace(A @ A @ A))
    assert t % 6 == 0
    return t // 6


def scipy_graph(g):
    data = np.ones(g.nnz, dtype=np.int8)
    return sp.csr_matrix((data, g.cols.astype(np.int64), g.offsets), shape=(g.n, g.n))


def root_rule_roots(g) -> list[int]:
    """Max-degree vertex (lowest id on ties), then the lowest id of every
    other connected component (components from scipy)."""
    if g.n == 0:
        return []
    deg = g.degrees()
    r0 = int(np.argmax(deg))  # argmax returns the first (lowest) index
    _, lab = connected_components(scipy_graph(g), directed=False)
    roots = [r0]
    seen = {lab[r0]}
    for v in range(g.n):
        if lab[v] not in seen:
            seen.add(lab[v])
            roots.append(v)
    return roots


def scipy_levels(g, roots) -> np.ndarray:
    """Shortest-path distance from each vertex's component root."""
    if g.n == 0:
        return np.zeros(0, dtype=np.int64)
    D = shortest_path(scipy_graph(g), unweighted=True, directed=False, indices=roots)
    D = np.atleast_2d(D)
    L = np.full(g.n, -1, dtype=np.int64)
    for i in range(D.shape[0]):
        fin = np.isfinite(D[i]) & (L < 0)
        L[fin] = D[i][fin].astype(np.int64)
    assert (L >= 0).all()
    return L


def effective_roots(g, roots) -> list[int]:
    """Given explicit roots in order: keep the first root of each component,
    then the lowest id of every component left without one."""
    _, lab = connected_components(scipy_graph(g), directed=False)
    out, seen = [], set()
    for r in roots:
        if lab[r] not in seen:
            seen.add(lab[r])
            out.append(int(r))
    for v in range(g.n):
        if lab[v] not in seen:
            seen.add(lab[v])
            out.append(v)
    return out


def is_bfs_labelling(g, L, roots) -> bool:
    """Characterisation of BFS distances: roots at 0, |L(u)-L(v)| <= 1 on
    every edge, and every non-root vertex has a neighbour one level lower."""
    L = np.asarray(L, dtype=np.int64)
    rs = set(int(r) for r in roots)
    if any(L[r] != 0 for r in rs):
        return False
    rows = np.repeat(np.arange(g.n), np.diff(g.offsets))
    c = g.cols.astype(np.int64)
    if np.any(np.abs(L[rows] - L[c]) > 1):
        return False
    for v in range(g.n):
        if v in rs:
            continue
        nb = g.neighbors(v).astype(np.int64)
        if not np.any(L[nb] == L[v] - 1):
            return False
    return True


def assigned_edge_counts(tris, L, H) -> np.ndarray:
    """Thm. 2's accounting: a triangle with exactly one horizontal edge is
    charged to that edge; one with three is charged to its (min, mid) edge.
    Returns the charge per cover edge in H's order."""
    idx = {(int(u), int(v)): i for i, (u, v) in enumerate(H)}
    out = np.zeros(len(H), dtype=np.int64)
    for a, b, c in tris:
        horiz = [(x, y) for x, y in ((a, b), (a, c), (b, c)) if L[x] == L[y]]
        if len(horiz) == 3:
            out[idx[(a, b)]] += 1
        elif len(horiz) == 1:
            out[idx[horiz[0]]] += 1
        else:
            raise AssertionError(f"triangle {a,b,c} has {len(horiz)} horizontal edges")
    return out


# ---------------------------------------------------------------------------
# graph families with closed forms

def closed_form_cases():
    """(graph, expected T, expected levels or None, expected H or None)."""
    cases = []
    for k in (1, 2, 3, 4, 5, 9, 17):
        g = gg.complete(k)
        L = np.array([0] + [1] * (k - 1)) if k > 0 else np.zeros(0)
        H = [(i, j) for i in range(1, k) for j in range(i + 1, k)]
        cases.append((g, comb(k, 3), L, H))
    for rim in (3, 4, 5, 8, 13):
        g = gg.wheel(rim)
        T = 4 if rim == 3 else rim
        if rim >= 4:
            L = np.array([0] + [1] * rim)
            H = sorted(tuple(sorted((i, i % rim + 1))) for i in range(1, rim + 1))
        else:
            L, H = None, None
        cases.append((g, T, L, H))
    for k in (3, 4, 5, 10):
        g = gg.cycle(k)
        cases.append((g, 1 if k == 3 else 0, None, None))
    for k in (1, 2, 5, 12):
        g = gg.path(k)
        # max degree 2 first reached at vertex 1 (k >= 3); else vertex 0
        if k >= 3:
            L = np.array([1] + list(range(k - 1)))
        else:
            L = np.arange(k)
        cases.append((g, 0, L, []))
    for r, c in ((1, 1), (2, 2), (3, 4), (5, 7)):
        g = gg.grid(r, c)
        deg = g.degrees()
        root = int(np.argmax(deg))
        rr, rc = divmod(root, c)
        L = np.array([abs(i // c - rr) + abs(i % c - rc) for i in range(r * c)])
        cases.append((g, 0, L, []))
    for a, b in ((1, 1), (2, 3), (4, 4), (3, 7)):
        cases.append((gg.complete_bipartite(a, b), 0, None, []))
    for leaves in (1, 6):
        cases.append((gg.star(leaves), 0, np.array([0] + [1] * leaves), []))
    for k in (1, 2, 5):
        g = gg.friendship(k)
        cases.append((g, k, np.array([0] + [1] * (2 * k)),
                      [(1 + 2 * t, 2 + 2 * t) for t in range(k)]))
    cases.append((gg.random_tree(40, 5), 0, None, []))
    cases.append((gg.empty(0), 0, np.zeros(0), []))
    cases.append((gg.empty(7), 0, np.zeros(7), []))
    u = gg.disjoint_union(gg.complete(6), gg.wheel(7), gg.empty(3), gg.cycle(3), gg.grid(3, 3))
    cases.append((u, comb(6, 3) + 7 + 1, None, None))
    return cases


def random_small_graphs():
    """Graphs small enough for the O(n^3) brute force (n <= 64)."""
    out = []
    for s in range(4):
        out.append(gg.rmat(5, 8, seed=100 + s))
        out.append(gg.rmat(6, 4, seed=200 + s, relabel_seed=300 + s))
        out.append(gg.erdos_renyi(40 + 6 * s, 0.2, seed=400 + s))
    out.append(gg.disjoint_union(gg.rmat(5, 4, seed=9), gg.erdos_renyi(20, 0.3, 11),
                                 gg.complete(7), gg.empty(2)))
    return out


def medium_graphs():
    """Graphs for the trace(A^3)/6 pin (n <= 512)."""
    return [gg.rmat(8, 16, seed=21), gg.rmat(9, 8, seed=22, relabel_seed=23),
            gg.erdos_renyi(300, 0.05, 24),
            gg.disjoint_union(gg.rmat(7, 16, seed=25), gg.erdos_renyi(100, 0.08, 26))]


# ---------------------------------------------------------------------------
# checks; each returns a list of failure strings (empty = pass)

def check_closed_forms(orc) -> list[str]:
    bad = []
    for g, T, L, H in closed_form_cases():
        r = orc.cetc(g)
        if r["T"] != T:
            bad.append(f"{g.name}: cetc T={r['T']} expected {T}")
        if orc.plain_count(g) != T:
            bad.append(f"{g.name}: plain T expected {T}")
        if len(orc.triangles(g)) != T:
            bad.append(f"{g.name}: enumerator expected {T}")
        if L is not None and not np.array_equal(r["levels"].astype(np.int64), np.asarray(L)):
            bad.append(f"{g.name}: levels {r['levels'].tolist()} expected {list(L)}")
        if H is not None and [tuple(map(int, x)) for x in r["H"]] != [tuple(x) for x in H]:
            bad.append(f"{g.name}: H {r['H'].tolist()} expected {H}")
    return bad


def check_brute_force(orc) -> list[str]:
    bad = []
    for g in random_small_graphs() + [c[0] for c in closed_form_cases() if c[0].n <= 64]:
        tris = brute_force_triangles(g)
        r = orc.cetc(g)
        if r["T"] != len(tris):
            bad.append(f"{g.name}: cetc {r['T']} brute {len(tris)}")
        if orc.plain_count(g) != len(tris):
            bad.append(f"{g.name}: plain vs brute")
        for th in (1, 3):
            if orc.cetc_count_mt(g, r["levels"], th) != len(tris):
                bad.append(f"{g.name}: all-core cetc ({th} threads) vs brute")
            if orc.plain_count_mt(g, th) != len(tris):
                bad.append(f"{g.name}: all-core plain ({th} threads) vs brute")
        lst = [tuple(map(int, t)) for t in orc.triangles(g)]
        if lst != tris:
            bad.append(f"{g.name}: enumerator list differs from brute force")
        # levels vs scipy with the root rule
        roots = root_rule_roots(g)
        if g.n and not np.array_equal(r["levels"].astype(np.int64), scipy_levels(g, roots)):
            bad.append(f"{g.name}: levels differ from scipy BFS distances")
        # Lemma 1/2 and Thm. 2 accounting
        Hs = set(map(tuple, r["H"].tolist()))
        L = r["levels"]
        for a, b, c in tris:
            nh = sum((x, y) in Hs for x, y in ((a, b), (a, c), (b, c)))
            if nh not in (1, 3):
                bad.append(f"{g.name}: triangle {a,b,c} has {nh} cover edges (Lemma 2)")
                break
        try:
            want = assigned_edge_counts(tris, L, r["H"].tolist())
            got = orc.cetc_edge_counts(g, L, r["H"]) if len(r["H"]) else np.zeros(0)
            if not np.array_equal(np.asarray(got, dtype=np.int64), want):
                bad.append(f"{g.name}: per-edge counts differ from Thm. 2 accounting")
            allc = orc.cetc_all_edge_counts_mt(g, L, len(want), 3)
            if not np.array_equal(np.asarray(allc, dtype=np.int64), want):
                bad.append(f"{g.name}: all-core per-edge counts differ from Thm. 2 accounting")
        except (AssertionError, KeyError) as e:
            bad.append(f"{g.name}: {e!r}")
    return bad


def check_trace(orc) -> list[str]:
    bad = []
    for g in medium_graphs():
        t = trace_count(g)
        r = orc.cetc(g)
        if r["T"] != t:
            bad.append(f"{g.name}: cetc {r['T']} trace {t}")
        if orc.plain_count(g) != t:
            bad.append(f"{g.name}: plain vs trace")
        if orc.cetc_count_mt(g, r["levels"], 4) != t or orc.plain_count_mt(g, 4) != t:
            bad.append(f"{g.name}: all-core counts vs trace")
        roots = root_rule_roots(g)
        if not np.array_equal(r["levels"].astype(np.int64), scipy_levels(g, roots)):
            bad.append(f"{g.name}: levels vs scipy")
        if r["nlevels"] != int(r["levels"].max()) + 1:
            bad.append(f"{g.name}: nlevels")
    return bad


def check_root_invariance(orc, seed=5) -> list[str]:
    """Thm. 2 holds for any BFS: T must not depend on the roots, and the
    levels must be BFS distances from the effective roots."""
    bad = []
    rng = np.random.default_rng(seed)
    for g in medium_graphs()[:2] + random_small_graphs()[:3]:
        base = orc.cetc(g)["T"]
        for _ in range(3):
            roots = rng.choice(g.n, size=min(4, g.n), replace=False)
            L, _ = orc.bfs_levels(g, roots)
            eff = effective_roots(g, roots)
            if not np.array_equal(L.astype(np.int64), scipy_levels(g, eff)):
                bad.append(f"{g.name}: explicit-root levels vs scipy")
            if not is_bfs_labelling(g, L, eff):
                bad.append(f"{g.name}: not a BFS labelling")
            if orc.cetc_count(g, L) != base:
                bad.append(f"{g.name}: T depends on roots")
            if orc.cetc_count_mt(g, L, 2) != base:
                bad.append(f"{g.name}: all-core T depends on roots")
    return bad


def check_all(orc) -> list[str]:
    return (check_closed_forms(orc) + check_brute_force(orc) + check_trace(orc)
            + check_root_invariance(orc))
