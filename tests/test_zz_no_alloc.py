"""ns_window_stats_static: the window statistics for callers that cannot
allocate device memory when they need them (for example when another
framework's caching allocator already holds the GPU's memory, or in a loop
that must not block in cudaMalloc/cudaFree).  It keeps its tables in one
fixed device array inside the library.

Checked through the C ABI, on two calls in a row -- a large window of
distinct links followed by a small skewed one, so that leftovers from the
first call would show up in the second -- against the CPU oracle and against
the ordinary entry points (ns_window_build + ns_network_stats), with exact
equality, the tolerance every count in this library is held to.  Collected
last on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from paper_2509_03653_b300 import _native

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def _row(t):
    v = t.cpu().numpy().view(np.uint64)
    return {f: int(x) for f, x in zip(ns.FIELDS, v[:9])}


def test_static_entry_matches_oracle_and_window_build_twice():
    L = _native.load()
    ctx = ns.Context(0, path="hash")
    windows = [W.rmat_stream(ns.STATIC_MAX_PACKETS), W.single_window(1000)]
    stream = torch.cuda.current_stream()
    for s, d in windows:
        ds, dd = _dev(s), _dev(d)
        out = torch.full((16,), -1, dtype=torch.int64, device="cuda")
        st = L.ns_window_stats_static(ctypes.c_void_p(ds.data_ptr()), ctypes.c_void_p(dd.data_ptr()), s.size,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, L.ns_last_error()
        torch.cuda.synchronize()
        assert _row(out) == oracle.stats_of_packets(s, d)
        m = ns.Matrix(ctx)
        ns.window_build(ctx, ds, dd, m)
        want = ns.network_stats(ctx, m)
        m.free()
        assert _row(out) == want
    ctx.close()


def test_static_entry_rejects_oversized_window():
    L = _native.load()
    n = ns.STATIC_MAX_PACKETS + 1
    src = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    st = L.ns_window_stats_static(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(src.data_ptr()), n,
                                  ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1  # NS_ERR_INVALID, nothing enqueued
    assert b"exceeds" in L.ns_last_error()
    torch.cuda.synchronize()
    assert int(out.abs().sum()) == 0
