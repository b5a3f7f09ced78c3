"""Parity of the CUDA path with the CPU oracle, element by element.

Every quantity and A's sorted nonzero list must match bit-exactly (all values
are uint64 counts).  Sizes span several tiles with ragged tails;
edge cases cover the empty window, one packet, a single repeated key, the
extreme keys 0 and 2^64-1, a star, self-loops and an all-distinct window.
Both aggregation paths (sort, hash) are checked, the sort path in both of
its per-destination forms, and the windowed forms (build + accumulate,
fused ingest) are checked after every window.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen
import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import assert_matrix_equal, export_np, stats_row, to_dev

pytestmark = pytest.mark.gpu

# "sort_pairs": the sort path with its per-destination side forced onto
# (dst, count) pairs, the form it takes from 2^32 packets on.  "hash_dense":
# the hash path with tables sized at load 0.9, so that probe sequences run
# long throughout.
PATHS = ["hash", "sort", "sort_pairs", "hash_dense"]


@pytest.fixture(scope="module")
def ctxs():
    c = {"hash": ns.Context(0, path="hash"), "sort": ns.Context(0, path="sort"),
         "sort_pairs": ns.Context(0, path="sort", column_sort="pairs"),
         "hash_dense": ns.Context(0, path="hash", hash_load=0.9)}
    yield c
    for x in c.values():
        x.close()


def check_window(ctx, s, d):
    m = ns.Matrix(ctx)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)
    got = ns.network_stats(ctx, m)
    wk, wc = oracle.build_matrix(s, d)
    assert got == oracle.stats(wk, wc)
    assert_matrix_equal(m, wk, wc)
    m.free()


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n", [0, 1, 2, 31, 4095, 4096, 4097, 12289, 100003, 1 << 17])
def test_window_zipf(ctxs, path, n):
    s, d = W.single_window(n)
    check_window(ctxs[path], s, d)


@pytest.mark.parametrize("path", PATHS)
def test_window_rmat(ctxs, path):
    s, d = W.rmat_stream(70001)
    check_window(ctxs[path], s, d)


@pytest.mark.parametrize("path", PATHS)
def test_edge_all_identical(ctxs, path):
    n = 50000
    check_window(ctxs[path], np.full(n, 7, np.uint32), np.full(n, 9, np.uint32))


@pytest.mark.parametrize("path", PATHS)
def test_edge_extreme_keys(ctxs, path):
    # keys 0 (src = dst = 0) and 2^64 - 1 (src = dst = 0xFFFFFFFF) with others
    s = np.array([0, 0xFFFFFFFF, 0, 5, 0xFFFFFFFF, 0, 0xFFFFFFFF, 1] * 1000, np.uint32)
    d = np.array([0, 0xFFFFFFFF, 0, 5, 0xFFFFFFFF, 1, 0, 0xFFFFFFFF] * 1000, np.uint32)
    check_window(ctxs[path], s, d)


@pytest.mark.parametrize("path", PATHS)
def test_edge_star_and_self_loops(ctxs, path):
    n = 30000
    s = np.full(n, 0xABCDEF01, np.uint32)
    d = np.arange(n, dtype=np.uint32)
    s2 = np.arange(5000, dtype=np.uint32)
    check_window(ctxs[path], np.concatenate([s, s2]), np.concatenate([d, s2]))


@pytest.mark.parametrize("path", PATHS)
def test_edge_all_distinct(ctxs, path):
    n = 1 << 16
    s = gen.feistel(np.arange(n, dtype=np.uint32), 11)
    d = gen.feistel(np.arange(n, dtype=np.uint32), 12)
    check_window(ctxs[path], s, d)


@pytest.mark.parametrize("path", PATHS)
def test_edge_tiny_address_space(ctxs, path):
    # heavy collisions: 8-bit addresses widened to 32 bits
    s8, d8 = gen.uniform_pairs(90001, 8, 5)
    w = lambda a: (a.astype(np.uint32) * np.uint32(0x01010101)).astype(np.uint32)
    check_window(ctxs[path], w(s8), w(d8))


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("mode", ["build_accumulate", "ingest"])
def test_windows_accumulate(ctxs, path, mode):
    ctx = ctxs[path]
    sizes = [4096, 1, 0, 12289, 7000, 4097, 30000, 3]
    total = sum(sizes)
    s, d = W.rmat_stream(total)
    # make some links repeat across windows
    s[total // 2:] = s[: total - total // 2]
    acc = ns.Matrix(ctx)
    tmp = ns.Matrix(ctx)
    off = 0
    want = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for n in sizes:
        ws, wd = s[off:off + n], d[off:off + n]
        off += n
        if mode == "ingest":
            ns.window_ingest(ctx, acc, to_dev(ws), to_dev(wd))
        else:
            ns.window_build(ctx, to_dev(ws), to_dev(wd), tmp)
            ns.accumulate(ctx, acc, tmp)
        want = oracle.accumulate(want, oracle.build_matrix(ws, wd))
        got = ns.network_stats(ctx, acc)
        assert got == oracle.stats(*want)
    assert_matrix_equal(acc, *want)


def test_mixed_formats_accumulate(ctxs):
    """Sorted-list windows (sort path) summed into a hash accumulator, and a
    sorted accumulator converted on its first accumulate."""
    s, d = W.single_window(20000)
    a1 = ns.Matrix(ctxs["sort"])
    ns.window_build(ctxs["sort"], to_dev(s[:9000]), to_dev(d[:9000]), a1)
    a2 = ns.Matrix(ctxs["sort"])
    ns.window_build(ctxs["sort"], to_dev(s[9000:]), to_dev(d[9000:]), a2)
    ns.accumulate(ctxs["sort"], a1, a2)  # list accumulator -> hash
    want = oracle.build_matrix(s, d)
    assert ns.network_stats(ctxs["sort"], a1) == oracle.stats(*want)
    assert_matrix_equal(a1, *want)


@pytest.mark.parametrize("path", PATHS)
def test_async_stats_match_blocking(ctxs, path):
    ctx = ctxs[path]
    s, d = W.single_window(1 << 15)
    m = ns.Matrix(ctx)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    ns.network_stats_async(ctx, m, out)
    torch.cuda.synchronize()
    assert stats_row(out) == ns.network_stats(ctx, m)


@pytest.mark.parametrize("path", PATHS)
def test_rebuild_reuses_matrix(ctxs, path):
    """A matrix rebuilt from a different window forgets the old one."""
    ctx = ctxs[path]
    m = ns.Matrix(ctx)
    s, d = W.single_window(50000)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)
    s2, d2 = W.rmat_stream(3000)
    ns.window_build(ctx, to_dev(s2), to_dev(d2), m)
    want = oracle.build_matrix(s2, d2)
    assert ns.network_stats(ctx, m) == oracle.stats(*want)
    assert_matrix_equal(m, *want)


def test_hash_accumulator_grows(ctxs):
    """An accumulator sized for a small window grows (rehash) as windows add
    new links, without changing any result."""
    ctx = ctxs["hash"]
    acc = ns.Matrix(ctx)
    ns.matrix_reserve(acc, 1000)
    s, d = W.rmat_stream(200000)
    for i in range(4):
        ns.window_ingest(ctx, acc, to_dev(s[i * 50000:(i + 1) * 50000]), to_dev(d[i * 50000:(i + 1) * 50000]))
    want = oracle.build_matrix(s, d)
    assert ns.network_stats(ctx, acc) == oracle.stats(*want)
    assert_matrix_equal(acc, *want)


def test_export_capacity_error(ctxs):
    ctx = ctxs["hash"]
    m = ns.Matrix(ctx)
    s, d = W.single_window(5000)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)
    keys = torch.empty(4, dtype=torch.int64, device="cuda")
    import ctypes
    got = ctypes.c_uint64()
    st = ctx._L.ns_matrix_export(m.handle, ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(keys.data_ptr()),
                                 4, ctypes.byref(got), None)
    assert st == 3  # NS_ERR_CAPACITY, nothing written
    assert got.value == oracle.stats(*oracle.build_matrix(s, d))["unique_links"]


def test_ingest_stats_after_every_window(ctxs):
    """ns_window_ingest_stats: the running quantities written by the last CTA
    of each window's launch equal the oracle's quantities of the prefix."""
    ctx = ctxs["hash"]
    sizes = [4096, 0, 1, 70001, 12289, 3, 40000]
    s, d = W.rmat_stream(sum(sizes))
    s[60000:] = s[:sum(sizes) - 60000]  # repeated sources across windows
    acc = ns.Matrix(ctx)
    rows = torch.zeros(len(sizes), 16, dtype=torch.int64, device="cuda")
    off = 0
    want_rows = []
    want = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for w, n in enumerate(sizes):
        ns.window_ingest_stats(ctx, acc, to_dev(s[off:off + n]), to_dev(d[off:off + n]), rows[w])
        want = oracle.accumulate(want, oracle.build_matrix(s[off:off + n], d[off:off + n]))
        want_rows.append(oracle.stats(*want))
        off += n
    torch.cuda.synchronize()
    for w in range(len(sizes)):
        assert stats_row(rows[w]) == want_rows[w], w
    assert ns.network_stats(ctx, acc) == want_rows[-1]
    assert_matrix_equal(acc, *want)


@pytest.mark.parametrize("form", ["sort", "sort_pairs"])
def test_trace_counts_kernels(ctxs, form):
    """Eight 64-bit digit passes for the links; the per-destination side adds
    four passes over one u64 word per link, or four over (dst, count) pairs."""
    ctx = ctxs[form]
    ns.trace_enable(ctx, True)
    m = ns.Matrix(ctx)
    s, d = W.single_window(50000)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)
    tr = ns.trace_read(ctx)
    ns.trace_enable(ctx, False)
    if form == "sort":
        assert tr["k_onesweep<u64 key>"][0] == 8
        assert tr["k_onesweep<u64 key, by dst>"][0] == 4
        assert "k_onesweep<u32 key, u64 value>" not in tr
    else:
        assert tr["k_onesweep<u64 key>"][0] == 8
        assert tr["k_onesweep<u32 key, u64 value>"][0] == 4
    assert tr["k_runs<links>"][0] == 1 and tr["k_run_stats<cols>"][0] == 1
    assert all(v[1] >= 0 and v[2] >= 0 for v in tr.values())
    assert ns.trace_read(ctx) == {}


def test_export_into_unaligned_buffers(ctxs):
    """ns_matrix_export into caller buffers that start 8 bytes past a 16-byte
    boundary (the sort stages such buffers with plain loads)."""
    import ctypes
    for path in PATHS:
        ctx = ctxs[path]
        s, d = W.single_window(30000)
        m = ns.Matrix(ctx)
        ns.window_build(ctx, to_dev(s), to_dev(d), m)
        want = oracle.build_matrix(s, d)
        nnz = want[0].size
        kb = torch.zeros(nnz + 2, dtype=torch.int64, device="cuda")
        cb = torch.zeros(nnz + 2, dtype=torch.int64, device="cuda")
        got = ctypes.c_uint64()
        st = ctx._L.ns_matrix_export(m.handle, ctypes.c_void_p(kb.data_ptr() + 8), ctypes.c_void_p(cb.data_ptr() + 8),
                                     nnz, ctypes.byref(got), None)
        assert st == 0 and got.value == nnz
        torch.cuda.synchronize()
        np.testing.assert_array_equal(kb[1:nnz + 1].cpu().numpy().view(np.uint64), want[0])
        np.testing.assert_array_equal(cb[1:nnz + 1].cpu().numpy().view(np.uint64), want[1])


@pytest.mark.parametrize("path", PATHS)
def test_window_from_unaligned_columns(ctxs, path):
    """Packet columns that start 4 bytes past a 16-byte boundary."""
    s, d = W.single_window(20001)
    ds = to_dev(np.concatenate([[0], s]).astype(np.uint32))[1:]
    dd = to_dev(np.concatenate([[0], d]).astype(np.uint32))[1:]
    ctx = ctxs[path]
    m = ns.Matrix(ctx)
    ns.window_build(ctx, ds, dd, m)
    want = oracle.build_matrix(s, d)
    assert ns.network_stats(ctx, m) == oracle.stats(*want)
    assert_matrix_equal(m, *want)


@pytest.mark.parametrize("cache", ["on", "off"])
@pytest.mark.parametrize("s_exp,K,n", [(1.5, 1 << 10, 1 << 20), (1.1, 1 << 14, 300007), (0.6, 1 << 20, 200003)])
def test_skewed_windows_cache_modes(cache, s_exp, K, n):
    """Very hot links/sources (Zipf 1.5 over 2^10: the top source carries a
    third of the packets, across hundreds of CTAs), a cache-overflowing
    mix, and near-uniform traffic -- with and without the per-CTA cache."""
    ctx = ns.Context(0, path="hash", cta_cache=cache)
    s, d = W.zipf_window(n, s_exp, K, 0x5EED + n)
    check_window(ctx, s, d)
    # and as two windows accumulated
    acc = ns.Matrix(ctx)
    ns.window_ingest(ctx, acc, to_dev(s[: n // 3]), to_dev(d[: n // 3]))
    ns.window_ingest(ctx, acc, to_dev(s[n // 3:]), to_dev(d[n // 3:]))
    want = oracle.build_matrix(s, d)
    assert ns.network_stats(ctx, acc) == oracle.stats(*want)
    assert_matrix_equal(acc, *want)


def test_sort_contexts_on_two_host_threads():
    """Two host threads, each with its own sort-path context, build windows at
    the same time.  The library's per-kernel launch shapes are shared between
    them (and locked); every result must equal the oracle's."""
    import threading
    cases = [W.zipf_window(300007, 1.1, 1 << 14, 0xA11CE), W.zipf_window(500009, 1.3, 1 << 16, 0xB0B)]
    devs = [(to_dev(s), to_dev(d)) for s, d in cases]
    torch.cuda.synchronize()
    results, errors = [None, None], []

    def work(t):
        try:
            ctx = ns.Context(0, path="sort")
            out = []
            for _ in range(3):
                m = ns.Matrix(ctx)
                ns.window_build(ctx, devs[t][0], devs[t][1], m)
                out.append((ns.network_stats(ctx, m), export_np(m)))
                m.free()
            ctx.close()
            results[t] = out
        except Exception as e:  # reported below, on the test's thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(t,)) for t in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for t, (s, d) in enumerate(cases):
        wk, wc = oracle.build_matrix(s, d)
        want = oracle.stats(wk, wc)
        for st, (k, c) in results[t]:
            assert st == want
            np.testing.assert_array_equal(k, wk)
            np.testing.assert_array_equal(c, wc)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_device_waits_time_out(which):
    """A look-back on a status word nobody publishes (one thread, and a whole
    warp), and an mbarrier phase expecting bytes no copy delivers: the
    bounded waits give up with NS_ERR_TIMEOUT within seconds and the device
    stays usable."""
    import ctypes
    import time
    from paper_2509_03653_b300 import _native
    L = _native.load()
    t0 = time.time()
    st = L.ns_diag_wait_timeout(which, None)
    el = time.time() - t0
    assert st == 5, L.ns_last_error()  # NS_ERR_TIMEOUT
    assert el < 10.0
    # the context still works afterwards
    ctx = ns.Context(0, path="sort")
    s, d = W.single_window(5000)
    m = ns.Matrix(ctx)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)
    assert ns.network_stats(ctx, m) == oracle.stats(*oracle.build_matrix(s, d))


def test_random_atomic_ceiling_diagnostic():
    us = ns.diag_random_atomics(1 << 20, 1 << 14, 2)
    assert 0.0 < us < 1e6
    with pytest.raises(ns.NsError):
        ns.diag_random_atomics(1000, 10, 1)  # not a power of two


@pytest.mark.parametrize("mode", ["claim", "claim_add", "claim_stale"])
def test_random_claim_ceiling_diagnostic(mode):
    us = ns.diag_random_claims(1 << 16, 1 << 14, mode, 2)
    assert 0.0 < us < 1e6
    with pytest.raises(ns.NsError):
        ns.diag_random_claims(1 << 16 | 1, 10, mode, 1)  # not a power of two


@pytest.mark.parametrize("load", [0.01, 0.95, -1.0])
def test_hash_load_out_of_range(load):
    with pytest.raises(ns.NsError) as e:
        ns.Context(0, path="hash", hash_load=load)
    assert e.value.name == "NS_ERR_INVALID"


def test_accumulator_growth_at_high_load():
    """An accumulator sized at load 0.9 that outgrows its tables is rehashed
    and stays exact."""
    ctx = ns.Context(0, path="hash", hash_load=0.9)
    acc = ns.Matrix(ctx)
    ns.matrix_reserve(acc, 1000)
    want = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for w in range(4):
        s, d = W.rmat_stream(30000, i0=w * 30000)
        ns.window_ingest(ctx, acc, to_dev(s), to_dev(d))
        want = oracle.accumulate(want, oracle.build_matrix(s, d))
    assert ns.network_stats(ctx, acc) == oracle.stats(*want)
    assert_matrix_equal(acc, *want)
