"""CPU oracle for cover-edge triangle counting — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct restatement of the paper's Alg. 1
(D. A. Bader et al., "Triangle Counting Through Cover-Edges",
arXiv 2210.00389), written in C (``oracle.c``) and driven through ctypes.
Only the tests, the package smoke check and the benchmark's CPU-baseline
leg may import this module.  The CUDA library never calls it and shares no
code with it.

Functions (each cites the passage it follows in ``oracle.c``):

* :func:`bfs_levels` — Def. 2 / Alg. 1, with the root rule
  "maximum-degree vertex first (lowest id on ties), then every other
  component rooted at its lowest id".
* :func:`cover_edges` — Thm. 1 / Alg. 1.
* :func:`cetc_count`, :func:`cetc_edge_counts` — Alg. 1.
* :func:`plain_count` — the direction-oriented edge iterator (Sec. I, V-A).
* :func:`triangles` — triangle finding (lists {a < b < c}).
* :func:`cetc_count_mt`, :func:`plain_count_mt`, :func:`cetc_all_edge_counts_mt`
  — the same counting loops with the outer loop over vertices shared among
  the host's cores (OpenMP), for the benchmark-size graphs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def compile_source(src: str, out: str) -> str:
    """Compile an oracle C source file into a shared library at ``out``."""
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(out) or ".")
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                    "-fvisibility=hidden", src, "-o", tmp], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, well under a second)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


class Oracle:
    """ctypes binding of one oracle build (the default one, or a test's
    deliberately mutated copy)."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.or_bfs_levels.restype = ctypes.c_int64
        lib.or_bfs_levels.argtypes = [ctypes.c_uint32, i64p, u32p, u32p, ctypes.c_uint32, u32p]
        lib.or_cover_edges.restype = ctypes.c_int64
        lib.or_cover_edges.argtypes = [ctypes.c_uint32, i64p, u32p, u32p, u32p, ctypes.c_int64]
        lib.or_cetc_count.restype = ctypes.c_uint64
        lib.or_cetc_count.argtypes = [ctypes.c_uint32, i64p, u32p, u32p]
        lib.or_cetc_edge_counts.restype = ctypes.c_int
        lib.or_cetc_edge_counts.argtypes = [ctypes.c_uint32, i64p, u32p, u32p, u32p,
                                            ctypes.c_int64, u32p]
        lib.or_plain_count.restype = ctypes.c_uint64
        lib.or_plain_count.argtypes = [ctypes.c_uint32, i64p, u32p]
        lib.or_cetc_count_mt.restype = ctypes.c_uint64
        lib.or_cetc_count_mt.argtypes = [ctypes.c_uint32, i64p, u32p, u32p, ctypes.c_int]
        lib.or_plain_count_mt.restype = ctypes.c_uint64
        lib.or_plain_count_mt.argtypes = [ctypes.c_uint32, i64p, u32p, ctypes.c_int]
        lib.or_cetc_all_edge_counts_mt.restype = ctypes.c_int64
        lib.or_cetc_all_edge_counts_mt.argtypes = [ctypes.c_uint32, i64p, u32p, u32p, u32p,
                                                   ctypes.c_int64, ctypes.c_int]
        lib.or_triangles.restype = ctypes.c_int64
        lib.or_triangles.argtypes = [ctypes.c_uint32, i64p, u32p, u32p, ctypes.c_int64]
        self.lib = lib

    def bfs_levels(self, g, roots=None):
        """Levels L[n] (uint32) and the number of levels (Def. 2, Alg. 1)."""
        off, cols = _csr(g)
        L = np.empty(max(g.n, 1), dtype=np.uint32)
        if roots is None:
            r, nr = None, 0
        else:
            r = np.ascontiguousarray(roots, dtype=np.uint32)
            nr = int(r.size)
        nl = self.lib.or_bfs_levels(g.n, _i64(off), _u32(cols),
                                    _u32(r) if r is not None and nr else None, nr, _u32(L))
        if nl < 0:
            raise ValueError("bad roots")
        return L[:g.n], int(nl)

    def cover_edges(self, g, L) -> np.ndarray:
        """H as an (|H|, 2) uint32 array in ascending (u, v) order (Thm. 1)."""
        off, cols = _csr(g)
        L = np.ascontiguousarray(L, dtype=np.uint32)
        if L.size == 0:
            L = np.zeros(1, dtype=np.uint32)
        h = self.lib.or_cover_edges(g.n, _i64(off), _u32(cols), _u32(L), None, 0)
        uv = np.empty((max(h, 1), 2), dtype=np.uint32)
        h2 = self.lib.or_cover_edges(g.n, _i64(off), _u32(cols), _u32(L), _u32(uv), h)
        assert h2 == h
        return uv[:h]

    def num_cover(self, g, L) -> int:
        """|H| without listing H (Thm. 1)."""
        off, cols = _csr(g)
        L = np.ascontiguousarray(L, dtype=np.uint32)
        if L.size == 0:
            return 0
        return int(self.lib.or_cover_edges(g.n, _i64(off), _u32(cols), _u32(L), None, 0))

    def cetc_count(self, g, L) -> int:
        """T by Alg. 1 (exact uint64)."""
        off, cols = _csr(g)
        L = np.ascontiguousarray(L, dtype=np.uint32)
        if L.size == 0:
            return 0
        return int(self.lib.or_cetc_count(g.n, _i64(off), _u32(cols), _u32(L)))

    def cetc_edge_counts(self, g, L, uv) -> np.ndarray:
        """Per-cover-edge counts (Alg. 1) for the given (k, 2) edge list."""
        off, cols = _csr(g)
        L = np.ascontiguousarray(L, dtype=np.uint32)
        uv = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
        out = np.zeros(max(uv.shape[0], 1), dtype=np.uint32)
        if uv.shape[0] == 0:
            return out[:0]
        rc = self.lib.or_cetc_edge_counts(g.n, _i64(off), _u32(cols), _u32(L), _u32(uv),
                                          uv.shape[0], _u32(out))
        if rc != 0:
            raise ValueError("not a cover edge")
        return out

    def plain_count(self, g) -> int:
        """T by the direction-oriented edge iterator (u < v, w > v)."""
        off, cols = _csr(g)
        return int(self.lib.or_plain_count(g.n, _i64(off), _u32(cols)))

    # all-core forms (OpenMP over the rows; threads = 0: all host cores)

    def cetc_count_mt(self, g, L, threads: int = 0) -> int:
        """T by Alg. 1, the outer loop shared among host threads."""
        off, cols = _csr(g)
        L = np.ascontiguousarray(L, dtype=np.uint32)
        if L.size == 0:
            return 0
        return int(self.lib.or_cetc_count_mt(g.n, _i64(off), _u32(cols), _u32(L), threads))

    def plain_count_mt(self, g, threads: int = 0) -> int:
        """The plain edge iterator's T, the outer loop shared among threads."""
        off, cols = _csr(g)
        return int(self.lib.or_plain_count_mt(g.n, _i64(off), _u32(cols), threads))

    def cetc_all_edge_counts_mt(self, g, L, num_cover: int, threads: int = 0) -> np.ndarray:
        """Alg. 1's count of every cover edge, in H's ascending (u, v) order."""
        off, cols = _csr(g)
        L = np.ascontiguousarray(L, dtype=np.uint32)
        out = np.zeros(max(num_cover, 1), dtype=np.uint32)
        if g.n == 0:
            return out[:0]
        h = self.lib.or_cetc_all_edge_counts_mt(g.n, _i64(off), _u32(cols), _u32(L), _u32(out),
                                                num_cover, threads)
        if h != num_cover:
            raise ValueError(f"|H| = {h}, expected {num_cover}")
        return out[:h]

    def triangles(self, g) -> np.ndarray:
        """All triangles as an (T, 3) uint32 array of a < b < c."""
        off, cols = _csr(g)
        t = self.lib.or_triangles(g.n, _i64(off), _u32(cols), None, 0)
        abc = np.empty((max(t, 1), 3), dtype=np.uint32)
        self.lib.or_triangles(g.n, _i64(off), _u32(cols), _u32(abc), t)
        return abc[:t]

    def cetc(self, g, roots=None) -> dict:
        """Alg. 1 end to end: levels, number of levels, H and T."""
        L, nl = self.bfs_levels(g, roots)
        return dict(levels=L, nlevels=nl, H=self.cover_edges(g, L), T=self.cetc_count(g, L))


def _default() -> Oracle:
    global _lib
    if _lib is None:
        _lib = Oracle(build())
    return _lib


def _u32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _i64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _csr(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    cols = np.ascontiguousarray(g.cols, dtype=np.uint32)
    if cols.size == 0:
        cols = np.zeros(1, dtype=np.uint32)
    return off, cols


def bfs_levels(g, roots=None):
    return _default().bfs_levels(g, roots)


def cover_edges(g, L):
    return _default().cover_edges(g, L)


def cetc_count(g, L):
    return _default().cetc_count(g, L)


def num_cover(g, L):
    return _default().num_cover(g, L)


def cetc_edge_counts(g, L, uv):
    return _default().cetc_edge_counts(g, L, uv)


def plain_count(g):
    return _default().plain_count(g)


def triangles(g):
    return _default().triangles(g)


def cetc_count_mt(g, L, threads: int = 0):
    return _default().cetc_count_mt(g, L, threads)


def plain_count_mt(g, threads: int = 0):
    return _default().plain_count_mt(g, threads)


def cetc_all_edge_counts_mt(g, L, num_cover: int, threads: int = 0):
    return _default().cetc_all_edge_counts_mt(g, L, num_cover, threads)


def cetc(g, roots=None) -> dict:
    return _default().cetc(g, roots)
