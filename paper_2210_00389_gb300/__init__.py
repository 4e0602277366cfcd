"""Python binding of libcetc, the GB300 cover-edge triangle-counting library.

Thin ctypes marshalling over the C ABI declared in ``include/tc.h``: every
function here has the name of the C entry point it calls and does no
computation of its own.  Buffers may be numpy arrays (host memory) or torch
tensors (host or CUDA); streams may be ``torch.cuda.Stream`` objects or raw
``cudaStream_t`` handles.

Method: D. A. Bader et al., "Triangle Counting Through Cover-Edges"
(arXiv 2210.00389), Alg. 1: BFS levels (Def. 2), horizontal cover edges
(Thm. 1), intersection with the count-once rule (Thm. 2).

The library must be built first (``python paper_2210_00389_gb300/build.py``
or ``__graft_entry__.build()``); importing without it raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcetc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libcetc.so is not built ({LIB_PATH} missing): run "
        "`python paper_2210_00389_gb300/build.py` on a machine with nvcc")

_lib = ctypes.CDLL(LIB_PATH)

TC_OK = 0
TC_ERR_INVALID_ARG = -1
TC_ERR_INVALID_GRAPH = -2
TC_ERR_OOM = -3
TC_ERR_CUDA = -4
TC_ERR_CAPACITY = -5
TC_ERR_TIMEOUT = -6
TC_ERR_AGAIN = -7
TC_ERR_NOT_FOUND = -8
TC_ERR_CANCELLED = -9

TC_GRAPH_VALIDATE = 1
TC_GRAPH_CHECK_SYM = 2
TC_GRAPH_BORROW = 4

TC_MODE_COVER = 0
TC_MODE_PLAIN = 1
TC_INTERSECT_MERGE = 0x10


class CSRView(ctypes.Structure):
    _fields_ = [("offsets", ctypes.c_void_p), ("cols", ctypes.c_void_p),
                ("n", ctypes.c_uint32), ("nnz", ctypes.c_int64), ("on_device", ctypes.c_int)]


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("nnz", ctypes.c_int64), ("num_edges", ctypes.c_int64),
                ("max_degree", ctypes.c_uint32), ("nlevels", ctypes.c_int64),
                ("num_cover", ctypes.c_int64), ("num_roots", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("ms_validate", ctypes.c_float), ("ms_bfs", ctypes.c_float),
                ("ms_cover", ctypes.c_float), ("ms_bucket", ctypes.c_float),
                ("ms_intersect", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("bfs_levels", ctypes.c_uint32), ("bfs_bottom_up", ctypes.c_uint32),
                ("edges_intersected", ctypes.c_int64), ("list_elems", ctypes.c_int64),
                ("reserved0", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint32),
                ("ms_main_kernel", ctypes.c_float)]


class Options(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("skew", ctypes.c_int32), ("tiny_max_nnz", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("slots", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("wait_limit_ms", ctypes.c_int32),
                ("fail_admitted", ctypes.c_int32), ("borrow_views", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


_vp = ctypes.c_void_p
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_ip = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "tc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "tc_last_error": (ctypes.c_char_p, []),
    "tc_version": (ctypes.c_int, []),
    "tc_kernel_launches": (ctypes.c_uint64, []),
    "tc_set_allocator": (ctypes.c_int, [_vp, _vp, _vp]),
    "tc_graph_create": (ctypes.c_int, [ctypes.POINTER(CSRView), ctypes.c_uint32, _vp,
                                       ctypes.POINTER(_vp)]),
    "tc_graph_destroy": (ctypes.c_int, [_vp]),
    "tc_graph_invalidate": (ctypes.c_int, [_vp]),
    "tc_graph_info": (ctypes.c_int, [_vp, ctypes.POINTER(GraphInfo)]),
    "tc_graph_stats": (ctypes.c_int, [_vp, ctypes.POINTER(Stats)]),
    "tc_bfs_levels": (ctypes.c_int, [_vp, _vp, ctypes.c_uint32, _vp, _u32p]),
    "tc_cover_edges": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _i64p]),
    "tc_count": (ctypes.c_int, [_vp, ctypes.c_int, _u64p]),
    "tc_cover_edge_counts": (ctypes.c_int, [_vp, _vp, ctypes.c_int64]),
    "tc_shard_bounds": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int32, _vp]),
    "tc_vertex_counts": (ctypes.c_int, [_vp, _vp]),
    "tc_list_triangles": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _i64p]),
    "tc_count_range": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _u64p]),
    "tc_count_plain_static": (ctypes.c_int, [_vp, _vp, ctypes.c_uint32, ctypes.c_int64, _vp, _vp]),
    "tc_count_batch": (ctypes.c_int, [ctypes.POINTER(CSRView), ctypes.c_int32, ctypes.c_int,
                                      ctypes.POINTER(Options), _vp, _u64p, _ip]),
    "tc_serve_create": (ctypes.c_int, [ctypes.POINTER(ServeConfig), ctypes.POINTER(_vp)]),
    "tc_serve_register": (ctypes.c_int, [_vp, ctypes.POINTER(CSRView), _u64p]),
    "tc_serve_submit": (ctypes.c_int, [_vp, ctypes.POINTER(CSRView), ctypes.c_uint64,
                                       ctypes.c_int, _u64p]),
    "tc_serve_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, _ip, _u64p, _ip]),
    "tc_serve_destroy": (ctypes.c_int, [_vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class TCError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.tc_last_error().decode(errors="replace")
        name = _lib.tc_strerror(status).decode()
        super().__init__(f"{where}: {name} ({status}): {msg}")


def _check(status: int, where: str) -> None:
    if status != TC_OK:
        raise TCError(status, where)


# ---------------------------------------------------------------- marshalling

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(address, on_device) of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None, False
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), bool(x.is_cuda)
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, False
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_handle(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def csr_view(offsets, cols, n: int | None = None):
    """CSRView over caller buffers (int64 offsets[n+1], uint32 cols[nnz])."""
    op, od = _ptr(offsets)
    cp, cd = _ptr(cols)
    if n is None:
        n = (offsets.shape[0] if hasattr(offsets, "shape") else len(offsets)) - 1
    nnz = cols.shape[0] if hasattr(cols, "shape") else len(cols)
    _check_dtype(offsets, "int64")
    _check_dtype(cols, "uint32")
    v = CSRView(op, cp if nnz > 0 else (cp or 0), n, nnz, 1 if (od and (cd or nnz == 0)) else 0)
    return v


def _check_dtype(x, want: str):
    name = str(x.dtype).replace("torch.", "")
    if name != want:
        raise TypeError(f"expected dtype {want}, got {name}")


# ---------------------------------------------------------------- C ABI names

def tc_version() -> int:
    return _lib.tc_version()


def tc_kernel_launches() -> int:
    return _lib.tc_kernel_launches()


def tc_strerror(status: int) -> str:
    return _lib.tc_strerror(status).decode()


def tc_last_error() -> str:
    return _lib.tc_last_error().decode(errors="replace")


def tc_set_allocator(alloc_fn=None, free_fn=None, ctx=None) -> None:
    """alloc_fn / free_fn are ctypes function pointers (or None to reset)."""
    _check(_lib.tc_set_allocator(alloc_fn, free_fn, ctx), "tc_set_allocator")


def tc_graph_create(offsets, cols, n: int | None = None, flags: int = 0, stream=None) -> int:
    """Create a graph object from a CSR; returns the opaque handle."""
    v = csr_view(offsets, cols, n)
    h = _vp()
    _check(_lib.tc_graph_create(ctypes.byref(v), flags, _stream_handle(stream), ctypes.byref(h)),
           "tc_graph_create")
    return h.value


def tc_graph_destroy(g: int) -> None:
    _check(_lib.tc_graph_destroy(g), "tc_graph_destroy")


def tc_graph_invalidate(g: int) -> None:
    _check(_lib.tc_graph_invalidate(g), "tc_graph_invalidate")


def tc_graph_info(g: int) -> dict:
    info = GraphInfo()
    _check(_lib.tc_graph_info(g, ctypes.byref(info)), "tc_graph_info")
    return {k: getattr(info, k) for k, _ in GraphInfo._fields_}


def tc_graph_stats(g: int) -> dict:
    st = Stats()
    _check(_lib.tc_graph_stats(g, ctypes.byref(st)), "tc_graph_stats")
    return {k: getattr(st, k) for k, _ in Stats._fields_}


def tc_bfs_levels(g: int, roots=None, out=None):
    """BFS levels (Def. 2).  Returns (levels, nlevels); `out` may be a
    uint32 numpy array / torch tensor of length n (host or CUDA)."""
    n = tc_graph_info(g)["n"]
    if out is None:
        out = np.empty(n, dtype=np.uint32)
    op, _ = _ptr(out)
    r = None
    nr = 0
    if roots is not None:
        r = np.ascontiguousarray(np.asarray(roots, dtype=np.uint32))
        nr = int(r.size)
    nl = ctypes.c_uint32(0)
    _check(_lib.tc_bfs_levels(g, r.ctypes.data if nr else None, nr, op if n else None,
                              ctypes.byref(nl)), "tc_bfs_levels")
    return out, nl.value


def tc_cover_edge_count(g: int) -> int:
    """|H| (Thm. 1) without copying the cover edges out (tc_cover_edges with
    uv_out = NULL)."""
    cnt = ctypes.c_int64(0)
    _check(_lib.tc_cover_edges(g, None, 0, ctypes.byref(cnt)), "tc_cover_edges")
    return cnt.value


def tc_cover_edges(g: int, out=None):
    """Cover-edge set H (Thm. 1) as a (|H|, 2) uint32 array (or into `out`)."""
    cnt = ctypes.c_int64(0)
    _check(_lib.tc_cover_edges(g, None, 0, ctypes.byref(cnt)), "tc_cover_edges")
    if out is None:
        out = np.empty((max(cnt.value, 1), 2), dtype=np.uint32)
    op, _ = _ptr(out)
    cap = (out.numel() if _is_torch(out) else out.size) // 2
    _check(_lib.tc_cover_edges(g, op, cap, ctypes.byref(cnt)), "tc_cover_edges")
    return out[:cnt.value]


def tc_count(g: int, mode: int = TC_MODE_COVER) -> int:
    c = ctypes.c_uint64(0)
    _check(_lib.tc_count(g, mode, ctypes.byref(c)), "tc_count")
    return c.value


def tc_vertex_counts(g: int, out=None):
    """uint64[n]: triangles containing each vertex (host numpy, or into a
    given numpy array / CUDA tensor)."""
    n = tc_graph_info(g)["n"]
    if out is None:
        out = np.zeros(n, dtype=np.uint64)
    op, _ = _ptr(out)
    _check(_lib.tc_vertex_counts(g, op if n else None), "tc_vertex_counts")
    return out


def tc_list_triangles(g: int) -> np.ndarray:
    """(T, 3) uint32 array of the triangles as (u, v, w): (u, v) the cover
    edge the count-once rule attributes the triangle to, w the apex."""
    cnt = ctypes.c_int64(0)
    _check(_lib.tc_list_triangles(g, None, 0, ctypes.byref(cnt)), "tc_list_triangles")
    out = np.empty((max(cnt.value, 1), 3), dtype=np.uint32)
    _check(_lib.tc_list_triangles(g, out.ctypes.data, cnt.value, ctypes.byref(cnt)),
           "tc_list_triangles")
    return out[:cnt.value]


def tc_shard_bounds(g: int, mode: int, nshards: int) -> np.ndarray:
    """int64[nshards + 1] work-balanced bounds of the mode's edge index space."""
    b = np.zeros(nshards + 1, dtype=np.int64)
    _check(_lib.tc_shard_bounds(g, mode, nshards, b.ctypes.data), "tc_shard_bounds")
    return b


def tc_count_range(g: int, mode: int, begin: int, end: int) -> int:
    c = ctypes.c_uint64(0)
    _check(_lib.tc_count_range(g, mode, begin, end, ctypes.byref(c)), "tc_count_range")
    return c.value


def tc_cover_edge_counts(g: int, out=None):
    cnt = ctypes.c_int64(0)
    _check(_lib.tc_cover_edges(g, None, 0, ctypes.byref(cnt)), "tc_cover_edges")
    if out is None:
        out = np.empty(max(cnt.value, 1), dtype=np.uint32)
    op, _ = _ptr(out)
    cap = out.numel() if _is_torch(out) else out.size
    _check(_lib.tc_cover_edge_counts(g, op, cap), "tc_cover_edge_counts")
    return out[:cnt.value]


def tc_count_plain_static(offsets, cols, count_out, n: int | None = None, stream=None) -> None:
    """Plain all-edge count of a device CSR into the device tensor
    ``count_out`` (int64/uint64, one element) without any device
    allocation; asynchronous on ``stream``."""
    op, od = _ptr(offsets)
    cp, cd = _ptr(cols)
    outp, outd = _ptr(count_out)
    if n is None:
        n = offsets.shape[0] - 1
    _check(_lib.tc_count_plain_static(op, cp, n, cols.shape[0], outp, _stream_handle(stream)),
           "tc_count_plain_static")


def autotuned_options() -> Options | None:
    """The batched kernel's setting chosen by autotune.py (None if absent)."""
    path = os.path.join(_HERE, "autotune.json")
    try:
        import json
        b = json.load(open(path))["batch"]
        return Options(int(b["block_threads"]), int(b["blocks_per_sm"]), int(b["skew"]),
                       int(b.get("tiny_max_nnz", 0)))
    except (OSError, KeyError, ValueError):
        return None


def tc_count_batch(graphs, mode: int = TC_MODE_COVER, opt: Options | None = None, stream=None):
    """Count a list of (offsets, cols) CSRs; returns (counts uint64[], status int32[]).
    Without ``opt`` the autotuned setting is used when autotune.json exists."""
    if opt is None:
        opt = autotuned_options()
    k = len(graphs)
    views = (CSRView * max(k, 1))()
    for i, (off, cols) in enumerate(graphs):
        views[i] = csr_view(off, cols)
    counts = np.zeros(max(k, 1), dtype=np.uint64)
    status = np.zeros(max(k, 1), dtype=np.int32)
    _check(_lib.tc_count_batch(views, k, mode, ctypes.byref(opt) if opt is not None else None,
                               _stream_handle(stream),
                               counts.ctypes.data_as(_u64p), status.ctypes.data_as(_ip)),
           "tc_count_batch")
    return counts[:k], status[:k]


def tc_serve_create(hbm_budget_bytes: int, slots: int = 64, queue_capacity: int = 4096,
                    wait_limit_ms: int = 0, fail_request: int = 0,
                    borrow_views: bool = False) -> int:
    """``fail_request`` = k > 0 injects a host-side allocation failure into the
    k-th admitted request (tests of failure handling).  With ``borrow_views``
    the server keeps the submitted arrays instead of copying them: the caller
    keeps them alive and unchanged until the request is reported done."""
    cfg = ServeConfig(hbm_budget_bytes, slots, queue_capacity, wait_limit_ms, fail_request,
                      1 if borrow_views else 0, (ctypes.c_int32 * 2)(0, 0))
    h = _vp()
    _check(_lib.tc_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "tc_serve_create")
    return h.value


def tc_serve_register(s: int, offsets, cols) -> int:
    v = csr_view(offsets, cols)
    gid = ctypes.c_uint64(0)
    _check(_lib.tc_serve_register(s, ctypes.byref(v), ctypes.byref(gid)), "tc_serve_register")
    return gid.value


def tc_serve_submit(s: int, csr=None, graph_id: int = 0, mode: int = TC_MODE_COVER):
    """Returns a ticket, or None when the queue is full (TC_ERR_AGAIN)."""
    t = ctypes.c_uint64(0)
    vp = None
    if csr is not None:
        v = csr_view(*csr)
        vp = ctypes.byref(v)
    st = _lib.tc_serve_submit(s, vp, graph_id, mode, ctypes.byref(t))
    if st == TC_ERR_AGAIN:
        return None
    _check(st, "tc_serve_submit")
    return t.value


def tc_serve_poll(s: int, ticket: int):
    """(done, count, status) of a ticket."""
    done, st = ctypes.c_int(0), ctypes.c_int(0)
    c = ctypes.c_uint64(0)
    _check(_lib.tc_serve_poll(s, ticket, ctypes.byref(done), ctypes.byref(c), ctypes.byref(st)),
           "tc_serve_poll")
    return bool(done.value), c.value, st.value


def tc_serve_destroy(s: int) -> None:
    _check(_lib.tc_serve_destroy(s), "tc_serve_destroy")


# ---------------------------------------------------------------- convenience

class Graph:
    """Owning wrapper: ``with Graph(offsets, cols) as g: g.count()``."""

    def __init__(self, offsets, cols, n: int | None = None, flags: int = 0, stream=None):
        self._keep = (offsets, cols) if flags & TC_GRAPH_BORROW else None
        self.handle = tc_graph_create(offsets, cols, n, flags, stream)

    def close(self):
        if self.handle:
            tc_graph_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def count(self, mode: int = TC_MODE_COVER) -> int:
        return tc_count(self.handle, mode)

    def levels(self, roots=None, out=None):
        return tc_bfs_levels(self.handle, roots, out)

    def vertex_counts(self, out=None):
        return tc_vertex_counts(self.handle, out)

    def list_triangles(self) -> np.ndarray:
        return tc_list_triangles(self.handle)

    def shard_bounds(self, mode: int, nshards: int) -> np.ndarray:
        return tc_shard_bounds(self.handle, mode, nshards)

    def count_range(self, mode: int, begin: int, end: int) -> int:
        return tc_count_range(self.handle, mode, begin, end)

    def cover_edges(self, out=None):
        return tc_cover_edges(self.handle, out)

    def cover_edge_count(self) -> int:
        return tc_cover_edge_count(self.handle)

    def cover_edge_counts(self, out=None):
        return tc_cover_edge_counts(self.handle, out)

    def info(self) -> dict:
        return tc_graph_info(self.handle)

    def stats(self) -> dict:
        return tc_graph_stats(self.handle)

    def invalidate(self):
        tc_graph_invalidate(self.handle)
