"""The C-ABI library loads and exports every entry point include/tc.h
declares; argument errors are reported without touching a GPU (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._load_build_module().build()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^TC_API\s+[\w\s\*]*?\b(tc_\w+)\s*\(", text, re.M))
    return sorted(names)


def test_header_declares_the_path():
    names = declared_symbols()
    for want in ("tc_graph_create", "tc_bfs_levels", "tc_cover_edges", "tc_count",
                 "tc_count_batch", "tc_serve_submit", "tc_serve_poll"):
        assert want in names


def test_every_declared_symbol_is_exported(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert missing == []


def test_binding_names_match_abi(lib_path):
    import paper_2210_00389_gb300 as tc
    for s in declared_symbols():
        assert hasattr(tc, s), f"binding lacks {s}"


def test_status_strings_and_argument_errors(lib_path):
    import paper_2210_00389_gb300 as tc
    assert tc.tc_strerror(tc.TC_OK) == "ok"
    assert tc.tc_strerror(tc.TC_ERR_CAPACITY) == "output buffer too small"
    assert tc.tc_version() >= 100
    lib = tc._lib
    out = ctypes.c_void_p()
    assert lib.tc_graph_create(None, 0, None, ctypes.byref(out)) == tc.TC_ERR_INVALID_ARG
    assert "NULL" in tc.tc_last_error()
    c = ctypes.c_uint64()
    assert lib.tc_count(None, 0, ctypes.byref(c)) == tc.TC_ERR_INVALID_ARG
    assert lib.tc_graph_destroy(None) == tc.TC_OK
    with pytest.raises(tc.TCError):
        tc.tc_graph_create(np.zeros(3, dtype=np.int64), np.zeros(0, dtype=np.uint32),
                           flags=tc.TC_GRAPH_BORROW)
    with pytest.raises(TypeError):
        tc.csr_view(np.zeros(3, dtype=np.int32), np.zeros(0, dtype=np.uint32))
    assert lib.tc_set_allocator(ctypes.c_void_p(1), None, None) == tc.TC_ERR_INVALID_ARG
