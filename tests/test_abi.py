"""The C-ABI library loads, exports every symbol include/*.h declares, and
rejects bad arguments on the host without touching a GPU."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

import paper_2509_03653_b300 as ns
from paper_2509_03653_b300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ns_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_builds_and_loads():
    L = _native.load()
    assert os.path.exists(_native.lib_path())
    assert L is not None


def test_every_declared_symbol_is_exported():
    L = _native.load()
    names = declared_functions()
    assert "ns_window_build" in names and "ns_network_stats" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_every_declared_symbol_has_a_binding():
    names = declared_functions()
    missing = [n for n in names if n not in _native.SIGNATURES]
    assert not missing, missing


def test_status_strings():
    L = _native.load()
    assert L.ns_status_string(0) == b"NS_OK"
    assert L.ns_status_string(1) == b"NS_ERR_INVALID"
    assert L.ns_status_string(5) == b"NS_ERR_TIMEOUT"
    assert L.ns_status_string(8) == b"NS_ERR_IO"


def test_null_arguments_are_invalid_without_gpu():
    L = _native.load()
    P = ctypes.c_void_p
    assert L.ns_create(None, None, 0) == 1
    assert b"NULL" in L.ns_last_error()
    assert L.ns_window_build(None, None, None, 5, None, None) == 1
    assert L.ns_window_build_host(None, None, None, 5, None, None, None) == 1
    assert L.ns_accumulate(None, None, None, None) == 1
    assert L.ns_window_ingest(None, None, None, None, 3, None) == 1
    assert L.ns_network_stats(None, None, None, None) == 1
    assert L.ns_network_stats_async(None, None, None, None) == 1
    assert L.ns_matrix_export(None, None, None, 0, None, None) == 1
    assert L.ns_matrix_nnz(None, None, None) == 1
    assert L.ns_matrix_create(None, None) == 1
    assert L.ns_matrix_reserve(None, 10, None) == 1
    assert L.ns_matrix_clear(None, None) == 1
    assert L.ns_sync(None, None) == 1
    assert L.ns_matrix_save(None, None, None) == 1
    assert L.ns_matrix_load(None, None, None, None) == 1
    L.ns_destroy(None)
    L.ns_matrix_free(None)


def test_error_raises_in_python_binding():
    with pytest.raises(ns.NsError) as e:
        _native.check(1, "where")
    assert e.value.name == "NS_ERR_INVALID"


def test_matrix_after_its_context_closed_raises_without_a_library_call():
    """A matrix whose context (or owning slider) is gone must not reach the
    library, which would follow the context's freed memory."""
    class Closed:
        handle = None

    m = object.__new__(ns.Matrix)
    m._L = _native.load()
    m.ctx = Closed()
    m.handle = ctypes.c_void_p(1)  # never passed on
    for call in (lambda: ns.matrix_nnz(m), lambda: ns.matrix_clear(m), lambda: ns.matrix_reserve(m, 16),
                 lambda: ns.matrix_export(m)):
        with pytest.raises(RuntimeError, match="context has been closed"):
            call()
    m.handle = None
    with pytest.raises(RuntimeError, match="freed"):
        ns.matrix_nnz(m)

    class Open:
        handle = ctypes.c_void_p(1)
        device = 0

    b = ns._BorrowedMatrix.__new__(ns._BorrowedMatrix)
    b._L, b.ctx, b.handle, b.owner = _native.load(), Open(), ctypes.c_void_p(1), Closed()
    with pytest.raises(RuntimeError, match="owner has been freed"):
        ns.matrix_nnz(b)
