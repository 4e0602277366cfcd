"""Seeded synthetic graph generators (inputs only).

Every graph is returned as a symmetric CSR with sorted, duplicate-free
adjacency and no self-loops: ``offsets`` int64[n+1], ``cols`` uint32[nnz].
This module holds no triangle-counting arithmetic; the CPU oracle and the
CUDA path both read what it produces.

The heavy generators (R-MAT, Chung-Lu, Erdos-Renyi) and the CSR builder are
plain C in ``gen.c`` driven through ctypes; the small closed-form families
(complete graphs, wheels, grids, ...) are written with numpy.  Randomness is
SplitMix64 keyed by (seed, counter), so a graph depends only on its seed.

Workload recipes (sizes and distributions of the paper's benchmark graphs):

* R-MAT, Graph500 parameters a/b/c/d = 0.57/0.19/0.19/0.05, n = 2^scale,
  m = edgefactor * n generated pairs (Sec. IV-A of the paper); optional
  Fisher-Yates relabelling.
* Chung-Lu power law, gamma = 2.1, mean degree 32, degree cap 65,536, plus
  10% of the vertices in disjoint Erdos-Renyi islands of 16-256 vertices and
  mean degree 6.
* The mixed batch of 4,096 small graphs (R-MAT / Erdos-Renyi / complete).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lib = None

RMAT_ABCD = (Fraction(57, 100), Fraction(19, 100), Fraction(19, 100))


def build(force: bool = False) -> str:
    """Compile gen.c into libgraphgen.so next to it (gcc, a second or so)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
           "-fvisibility=hidden", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.gg_splitmix64.restype = ctypes.c_uint64
        lib.gg_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_rmat_edges.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                      u32p, u32p, ctypes.c_int]
        lib.gg_permutation.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p]
        lib.gg_apply_permutation.argtypes = [u32p, u32p, ctypes.c_int64, ctypes.c_int]
        lib.gg_alias_table.argtypes = [f64p, ctypes.c_uint32, u32p, u32p]
        lib.gg_alias_edges.argtypes = [u32p, u32p, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_int64, ctypes.c_uint64, u32p, u32p,
                                       ctypes.c_int]
        lib.gg_er_edges.restype = ctypes.c_int64
        lib.gg_er_edges.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                    ctypes.c_uint64, u32p, u32p, ctypes.c_int64]
        lib.gg_csr_begin.restype = ctypes.c_void_p
        lib.gg_csr_begin.argtypes = [ctypes.c_uint32, ctypes.c_int64, u32p, u32p,
                                     ctypes.c_int, i64p]
        lib.gg_csr_finish.argtypes = [ctypes.c_void_p, i64p, u32p, ctypes.c_int]
        _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


@dataclass
class CSR:
    """Symmetric CSR: offsets int64[n+1], cols uint32[nnz] (sorted rows)."""
    n: int
    offsets: np.ndarray
    cols: np.ndarray
    generated_edges: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1]) if self.n > 0 else 0

    @property
    def num_edges(self) -> int:
        """Undirected edge count |E| after de-duplication (= nnz / 2)."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)

    def neighbors(self, v: int) -> np.ndarray:
        return self.cols[self.offsets[v]:self.offsets[v + 1]]


def splitmix64(seed: int, i: int) -> int:
    return int(_L().gg_splitmix64(seed & (2**64 - 1), i & (2**64 - 1)))


def from_edges(n: int, src, dst, name: str = "", generated: int | None = None) -> CSR:
    """Symmetrise an edge list, drop self-loops and duplicates, sort rows."""
    src = np.ascontiguousarray(np.asarray(src, dtype=np.uint32))
    dst = np.ascontiguousarray(np.asarray(dst, dtype=np.uint32))
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    m = int(src.size)
    if n < 0 or n > 2**32 - 1:
        raise ValueError("n out of range")
    lib = _L()
    nnz = ctypes.c_int64(0)
    h = lib.gg_csr_begin(n, m, _p(src, ctypes.c_uint32), _p(dst, ctypes.c_uint32),
                         _threads(), ctypes.byref(nnz))
    offsets = np.zeros(n + 1, dtype=np.int64)
    cols = np.zeros(max(nnz.value, 0), dtype=np.uint32)
    rc = lib.gg_csr_finish(h, _p(offsets, ctypes.c_int64), _p(cols, ctypes.c_uint32),
                           _threads())
    if rc != 0 or nnz.value < 0:
        raise ValueError("edge endpoint >= n")
    return CSR(n=n, offsets=offsets, cols=cols,
               generated_edges=m if generated is None else generated, name=name)


def _thr32(x: Fraction) -> int:
    return int(x * 2**32)


def permutation(n: int, seed: int) -> np.ndarray:
    perm = np.empty(n, dtype=np.uint32)
    _L().gg_permutation(n, seed & (2**64 - 1), _p(perm, ctypes.c_uint32))
    return perm


def rmat_edges(scale: int, edgefactor: int = 16, seed: int = 1,
               abc=RMAT_ABCD, relabel_seed: int | None = None):
    """Generated R-MAT pairs (before cleanup) as two uint32 arrays."""
    n = 1 << scale
    m = edgefactor * n
    a, b, c = abc
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    rc = _L().gg_rmat_edges(scale, m, seed & (2**64 - 1), _thr32(a), _thr32(a + b),
                            _thr32(a + b + c), _p(src, ctypes.c_uint32),
                            _p(dst, ctypes.c_uint32), _threads())
    if rc != 0:
        raise ValueError("bad R-MAT parameters")
    if relabel_seed is not None:
        perm = permutation(n, relabel_seed)
        for arr in (src, dst):
            _L().gg_apply_permutation(_p(perm, ctypes.c_uint32), _p(arr, ctypes.c_uint32),
                                      m, _threads())
    return n, src, dst


def rmat(scale: int, edgefactor: int = 16, seed: int = 1,
         relabel_seed: int | None = None, abc=RMAT_ABCD) -> CSR:
    """R-MAT graph, Graph500 quadrant probabilities by default."""
    n, src, dst = rmat_edges(scale, edgefactor, seed, abc, relabel_seed)
    g = from_edges(n, src, dst, name=f"rmat-s{scale}-ef{edgefactor}-seed{seed}"
                   + (f"-relabel{relabel_seed}" if relabel_seed is not None else ""))
    g.meta.update(kind="rmat", scale=scale, edgefactor=edgefactor, seed=seed,
                  relabel_seed=relabel_seed)
    return g


def _er_threshold(p: float) -> int:
    if p <= 0.0:
        return 0
    if p >= 1.0:
        return 2**64 - 1
    return int(Fraction(p) * 2**64)


def er_edges(k: int, p: float, seed: int, base: int = 0):
    lib = _L()
    thr = _er_threshold(p)
    cnt = lib.gg_er_edges(k, base, thr, seed & (2**64 - 1), None, None, -1)
    src = np.empty(max(cnt, 1), dtype=np.uint32)
    dst = np.empty(max(cnt, 1), dtype=np.uint32)
    got = lib.gg_er_edges(k, base, thr, seed & (2**64 - 1), _p(src, ctypes.c_uint32),
                          _p(dst, ctypes.c_uint32), cnt)
    assert got == cnt
    return src[:cnt], dst[:cnt]


def erdos_renyi(n: int, p: float, seed: int) -> CSR:
    src, dst = er_edges(n, p, seed)
    g = from_edges(n, src, dst, name=f"er-n{n}-p{p:.4g}-seed{seed}")
    g.meta.update(kind="er", n=n, p=p, seed=seed)
    return g


def chung_lu_islands(n: int = 1 << 23, gamma: float = 2.1, mean_degree: float = 32.0,
                     cap: float = 65536.0, island_frac: float = 0.1,
                     island_min: int = 16, island_max: int = 256,
                     island_mean_degree: float = 6.0, seed: int = 7) -> CSR:
    """Chung-Lu power-law core plus disjoint Erdos-Renyi islands.

    Core vertices 0..floor((1-island_frac) n)-1 get weight
    (i+10)^(-1/(gamma-1)), scaled to ``mean_degree`` and then capped at
    ``cap`` (no rescale after the cap); round(sum(w)/2) endpoint pairs are
    drawn proportionally to w through an alias table.  The remaining vertices
    are split into consecutive islands of size U[island_min, island_max]
    (the last island absorbs a remainder smaller than island_min), each an
    independent G(k, island_mean_degree/(k-1)).
    """
    lib = _L()
    n_core = int((1.0 - island_frac) * n)
    idx = np.arange(n_core, dtype=np.float64)
    w = np.power(idx + 10.0, -1.0 / (gamma - 1.0))
    w *= mean_degree * n_core / w.sum()
    w = np.minimum(w, cap)
    pairs = int(round(float(w.sum()) / 2.0))
    prob = np.empty(n_core, dtype=np.uint32)
    alias = np.empty(n_core, dtype=np.uint32)
    w = np.ascontiguousarray(w)
    if lib.gg_alias_table(_p(w, ctypes.c_double), n_core, _p(prob, ctypes.c_uint32),
                          _p(alias, ctypes.c_uint32)) != 0:
        raise ValueError("bad Chung-Lu weights")
    src = [np.empty(pairs, dtype=np.uint32)]
    dst = [np.empty(pairs, dtype=np.uint32)]
    lib.gg_alias_edges(_p(prob, ctypes.c_uint32), _p(alias, ctypes.c_uint32), n_core, 0,
                       pairs, splitmix64(seed, 0), _p(src[0], ctypes.c_uint32),
                       _p(dst[0], ctypes.c_uint32), _threads())
    # islands
    size_seed = splitmix64(seed, 1)
    er_seed = splitmix64(seed, 2)
    base = n_core
    remaining = n - n_core
    j = 0
    islands = []
    while remaining > 0:
        span = island_max - island_min + 1
        k = island_min + int(splitmix64(size_seed, j) % span)
        if remaining - k < island_min:
            k = remaining
        islands.append((base, k))
        p = island_mean_degree / (k - 1) if k > 1 else 0.0
        s, d = er_edges(k, p, splitmix64(er_seed, j), base)
        src.append(s)
        dst.append(d)
        base += k
        remaining -= k
        j += 1
    S = np.concatenate(src)
    D = np.concatenate(dst)
    g = from_edges(n, S, D, name=f"chunglu-n{n}-g{gamma}-seed{seed}")
    g.meta.update(kind="chung_lu", n=n, n_core=n_core, islands=len(islands),
                  pairs=pairs, seed=seed)
    return g


# ---------------------------------------------------------------------------
# small closed-form families (numpy)

def _edges_graph(n, pairs, name, **meta) -> CSR:
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    g = from_edges(n, pairs[:, 0], pairs[:, 1], name=name)
    g.meta.update(meta)
    return g


def empty(n: int) -> CSR:
    return _edges_graph(n, np.zeros((0, 2)), f"empty-{n}", kind="empty")


def complete(k: int) -> CSR:
    i, j = np.triu_indices(k, 1)
    return _edges_graph(k, np.stack([i, j], 1), f"K{k}", kind="complete", k=k)


def path(k: int) -> CSR:
    i = np.arange(max(k - 1, 0))
    return _edges_graph(k, np.stack([i, i + 1], 1), f"P{k}", kind="path", k=k)


def cycle(k: int) -> CSR:
    i = np.arange(k)
    return _edges_graph(k, np.stack([i, (i + 1) % k], 1), f"C{k}", kind="cycle", k=k)


def star(leaves: int) -> CSR:
    i = np.arange(1, leaves + 1)
    return _edges_graph(leaves + 1, np.stack([np.zeros_like(i), i], 1), f"S{leaves}",
                        kind="star", leaves=leaves)


def wheel(rim: int) -> CSR:
    """Hub 0 joined to every vertex of the rim cycle 1..rim."""
    i = np.arange(rim)
    spokes = np.stack([np.zeros(rim, dtype=np.int64), i + 1], 1)
    rimc = np.stack([i + 1, (i + 1) % rim + 1], 1)
    return _edges_graph(rim + 1, np.concatenate([spokes, rimc]), f"W{rim}",
                        kind="wheel", rim=rim)


def grid(rows: int, cols: int) -> CSR:
    vid = np.arange(rows * cols).reshape(rows, cols)
    h = np.stack([vid[:, :-1].ravel(), vid[:, 1:].ravel()], 1)
    v = np.stack([vid[:-1, :].ravel(), vid[1:, :].ravel()], 1)
    return _edges_graph(rows * cols, np.concatenate([h, v]), f"grid{rows}x{cols}",
                        kind="grid", rows=rows, cols=cols)


def complete_bipartite(a: int, b: int) -> CSR:
    i, j = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return _edges_graph(a + b, np.stack([i.ravel(), j.ravel()], 1), f"K{a},{b}",
                        kind="complete_bipartite", a=a, b=b)


def friendship(k: int) -> CSR:
    """k triangles sharing the centre vertex 0."""
    e = []
    for t in range(k):
        x, y = 1 + 2 * t, 2 + 2 * t
        e += [(0, x), (0, y), (x, y)]
    return _edges_graph(2 * k + 1, np.array(e).reshape(-1, 2), f"F{k}", kind="friendship", k=k)


def random_tree(k: int, seed: int) -> CSR:
    parents = [int(splitmix64(seed, i) % i) for i in range(1, k)]
    pairs = np.stack([np.arange(1, k), np.array(parents, dtype=np.int64)], 1) if k > 1 \
        else np.zeros((0, 2))
    return _edges_graph(k, pairs, f"tree{k}-seed{seed}", kind="tree", k=k)


def disjoint_union(*graphs: CSR) -> CSR:
    src, dst, base = [], [], 0
    for g in graphs:
        rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets))
        src.append(rows + base)
        dst.append(g.cols.astype(np.int64) + base)
        base += g.n
    S = np.concatenate(src) if src else np.zeros(0, dtype=np.int64)
    D = np.concatenate(dst) if dst else np.zeros(0, dtype=np.int64)
    g = from_edges(base, S, D, name="+".join(x.name for x in graphs))
    g.meta.update(kind="union", parts=[x.name for x in graphs])
    return g


def relabel(g: CSR, seed: int) -> CSR:
    """Apply the Fisher-Yates permutation of stream ``seed`` to vertex ids."""
    perm = permutation(g.n, seed).astype(np.int64)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets))
    h = from_edges(g.n, perm[rows], perm[g.cols.astype(np.int64)],
                   name=g.name + f"-relabel{seed}")
    h.meta.update(g.meta)
    h.meta["relabel"] = seed
    return h


def to_edge_list(g: CSR):
    """Undirected edges (u < v) in CSR order."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets))
    c = g.cols.astype(np.int64)
    keep = rows < c
    return rows[keep], c[keep]


# ---------------------------------------------------------------------------
# workload recipes

def mixed_graph_specs(count: int = 4096, seed: int = 3, large_rmat_frac: float = 0.0):
    """Specs of the mixed small-graph batch.

    Exact quotas: 1% complete graphs K_m (m ~ U{20..200}), 10% Erdos-Renyi
    G(n, 10/(n-1)) with n ~ U{256..4096}, the rest R-MAT with scale ~ U{6..14}
    and edgefactor ~ U{8..32}; with ``large_rmat_frac`` > 0 that fraction of
    all graphs is taken out of the R-MAT share as R-MAT scale ~ U{18..22}.
    Kinds are shuffled with a Fisher-Yates pass of the same stream.
    """
    n_k = max(0, round(0.01 * count))
    n_er = max(0, round(0.10 * count))
    n_big = int(round(large_rmat_frac * count))
    n_rmat = count - n_k - n_er - n_big
    kinds = ["rmat"] * n_rmat + ["rmat_large"] * n_big + ["er"] * n_er + ["complete"] * n_k
    # shuffle
    for i in range(len(kinds) - 1, 0, -1):
        j = int(splitmix64(seed, i) % (i + 1))
        kinds[i], kinds[j] = kinds[j], kinds[i]
    specs = []
    s2 = splitmix64(seed, 1 << 40)
    for idx, kind in enumerate(kinds):
        r0 = splitmix64(s2, 4 * idx)
        r1 = splitmix64(s2, 4 * idx + 1)
        gseed = splitmix64(s2, 4 * idx + 2)
        if kind == "rmat":
            specs.append(dict(kind="rmat", scale=6 + int(r0 % 9), edgefactor=8 + int(r1 % 25),
                              seed=gseed))
        elif kind == "rmat_large":
            specs.append(dict(kind="rmat", scale=18 + int(r0 % 5), edgefactor=16, seed=gseed))
        elif kind == "er":
            n = 256 + int(r0 % (4096 - 256 + 1))
            specs.append(dict(kind="er", n=n, p=10.0 / (n - 1), seed=gseed))
        else:
            specs.append(dict(kind="complete", k=20 + int(r0 % 181)))
    return specs


def graph_from_spec(spec: dict) -> CSR:
    kind = spec["kind"]
    if kind == "rmat":
        return rmat(spec["scale"], spec["edgefactor"], spec["seed"], spec.get("relabel_seed"))
    if kind == "er":
        return erdos_renyi(spec["n"], spec["p"], spec["seed"])
    if kind == "complete":
        return complete(spec["k"])
    raise ValueError(kind)


# Named workloads (sizes and seeds of the benchmark configurations)
def rmat_s10() -> CSR:
    """R-MAT scale 10, edgefactor 16, seed 1, no relabel."""
    return rmat(10, 16, 1)


def rmat_s22() -> CSR:
    """R-MAT scale 22, edgefactor 16, edge seed 2, relabel stream 2 + 2^32."""
    return rmat(22, 16, 2, relabel_seed=2 + 2**32)


def rmat_s26() -> CSR:
    """R-MAT scale 26, edgefactor 16, edge seed 5, relabel stream 5 + 2^32."""
    return rmat(26, 16, 5, relabel_seed=5 + 2**32)


def chung_lu_2_23() -> CSR:
    return chung_lu_islands(1 << 23, seed=7)


def serve_large_specs() -> list[dict]:
    """The serving stream's large requests: two R-MAT graphs per scale
    18..22, edgefactor 16, edge seed 1000 + 10 scale + k, relabel stream
    2000 + 10 scale + k (k = 0, 1)."""
    return [dict(kind="rmat", scale=sc, edgefactor=16, seed=1000 + 10 * sc + k,
                 relabel_seed=2000 + 10 * sc + k) for sc in range(18, 23) for k in range(2)]
