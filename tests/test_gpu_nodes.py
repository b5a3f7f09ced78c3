"""Per-entity vectors (ns_matrix_nodes) and address anonymization
(ns_anonymize), bit-exact against the CPU oracle on the same seeded inputs,
from hash and sort matrices, with ragged sizes spanning several tiles, the
extreme addresses, empty inputs and the capacity errors."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen
import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def windows():
    yield W.single_window(1 << 17)
    yield W.rmat_stream(70001)
    yield W.zipf_window(12289, 1.3, 1 << 10, 77)
    s = np.array([0, 0xFFFFFFFF, 5, 0xFFFFFFFF, 5, 0], np.uint32)
    yield s, np.array([0xFFFFFFFF, 0, 5, 0xFFFFFFFF, 7, 0], np.uint32)
    yield np.array([3], np.uint32), np.array([3], np.uint32)


@pytest.mark.parametrize("path", ["hash", "sort"])
def test_nodes_match_oracle(path):
    ctx = ns.Context(0, path=path)
    for s, d in windows():
        m = ns.Matrix(ctx)
        ns.window_build(ctx, to_dev(s), to_dev(d), m)
        k, c = oracle.build_matrix(s, d)
        for which, ref in (("src", oracle.rows(k, c)), ("dst", oracle.cols(k, c))):
            ids, pk, dg = ns.matrix_nodes(m, which)
            np.testing.assert_array_equal(u32(ids), ref[0])
            np.testing.assert_array_equal(u64(pk), ref[1])
            np.testing.assert_array_equal(u64(dg), ref[2])
        np.testing.assert_array_equal(u32(ns.matrix_nodes(m, "any")), oracle.unique_addresses(k))
        m.free()


def test_nodes_of_accumulated_matrix_and_empty():
    ctx = ns.Context(0, path="hash")
    acc = ns.Matrix(ctx)
    assert ns.matrix_nodes(acc, "any").numel() == 0
    want = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for w in range(3):
        s, d = W.rmat_stream(20000, i0=w * 20000)
        ns.window_ingest(ctx, acc, to_dev(s), to_dev(d))
        want = oracle.accumulate(want, oracle.build_matrix(s, d))
    ids, pk, dg = ns.matrix_nodes(acc, "dst")
    ref = oracle.cols(*want)
    np.testing.assert_array_equal(u32(ids), ref[0])
    np.testing.assert_array_equal(u64(pk), ref[1])
    np.testing.assert_array_equal(u64(dg), ref[2])
    st = ns.network_stats(ctx, acc)
    assert ids.numel() == st["unique_destinations"] and int(u64(pk).max()) == st["max_dst_packets"]


def test_nodes_capacity_error():
    import ctypes
    ctx = ns.Context(0, path="sort")
    s, d = W.single_window(5000)
    m = ns.Matrix(ctx)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)
    S = ns.network_stats(ctx, m)["unique_sources"]
    ids = torch.zeros(S - 1, dtype=torch.int32, device="cuda")
    got = ctypes.c_uint64()
    L = ctx._L
    st = L.ns_matrix_nodes(ctx.handle, m.handle, 0, ctypes.c_void_p(ids.data_ptr()), None, None, S - 1,
                           ctypes.byref(got), None)
    assert st == 3 and got.value == S  # NS_ERR_CAPACITY, count reported
    want = oracle.rows(*oracle.build_matrix(s, d))[0][: S - 1]
    np.testing.assert_array_equal(u32(ids), want)  # the first cap entries


@pytest.mark.parametrize("case", ["zipf", "rmat", "edges", "one"])
def test_anonymize_matches_oracle(case):
    ctx = ns.Context(0)
    s, d = {"zipf": lambda: W.single_window(1 << 17), "rmat": lambda: W.rmat_stream(100003),
            "edges": lambda: (np.array([0, 0xFFFFFFFF, 7, 7], np.uint32), np.array([7, 0, 0xFFFFFFFF, 7], np.uint32)),
            "one": lambda: (np.array([9], np.uint32), np.array([9], np.uint32))}[case]()
    rnd = gen.random_u64(2 * s.size, 12345, 7)
    ws, wd, wn = oracle.anonymize(s, d, rnd)
    r = torch.from_numpy(rnd.view(np.int64)).cuda()
    gs, gd, gn = ns.anonymize(ctx, to_dev(s), to_dev(d), r)
    assert gn == wn
    np.testing.assert_array_equal(u32(gs), ws)
    np.testing.assert_array_equal(u32(gd), wd)


def test_anonymize_golden_in_place_and_errors():
    from golden_io import read_anonymize_example
    ctx = ns.Context(0)
    s, d, rnd, want_s, want_d = read_anonymize_example()
    ds, dd = to_dev(s), to_dev(d)
    r = torch.from_numpy(rnd.view(np.int64)).cuda()
    _, _, nu = ns.anonymize(ctx, ds, dd, r, out_src=ds, out_dst=dd)  # in place
    assert nu == 4
    np.testing.assert_array_equal(u32(ds), want_s)
    np.testing.assert_array_equal(u32(dd), want_d)
    # fewer random keys than distinct addresses
    with pytest.raises(ns.NsError) as e:
        ns.anonymize(ctx, to_dev(s), to_dev(d), r[:3])
    assert e.value.name == "NS_ERR_CAPACITY"
    # empty input
    z = torch.zeros(0, dtype=torch.int32, device="cuda")
    assert ns.anonymize(ctx, z, z, r)[2] == 0


def test_anonymized_stream_keeps_the_quantities():
    """Anonymizing is a relabelling: the nine quantities of the anonymized
    packets equal those of the original ones (on the GPU path end to end)."""
    ctx = ns.Context(0, path="hash")
    s, d = W.rmat_stream(1 << 18)
    rnd = gen.random_u64(2 * s.size, 99, 1)
    gs, gd, _ = ns.anonymize(ctx, to_dev(s), to_dev(d), torch.from_numpy(rnd.view(np.int64)).cuda())
    a, b = ns.Matrix(ctx), ns.Matrix(ctx)
    ns.window_build(ctx, to_dev(s), to_dev(d), a)
    ns.window_build(ctx, gs, gd, b)
    assert ns.network_stats(ctx, a) == ns.network_stats(ctx, b)


@pytest.mark.slow
def test_anonymize_high_cardinality_retries_the_set():
    """2^24 packets of uniform 32-bit addresses: more than 2^24 distinct
    addresses overflow the first address set, and the retry with a table
    for all of them still gives the oracle's labels."""
    s, d = gen.uniform_pairs(1 << 24, 32, 4242)
    rnd = gen.random_u64(2 * s.size, 4243, 5)
    ws, wd, wn = oracle.anonymize(s, d, rnd)
    assert wn > (1 << 24)
    ctx = ns.Context(0)
    gs, gd, gn = ns.anonymize(ctx, to_dev(s), to_dev(d), torch.from_numpy(rnd.view(np.int64)).cuda())
    assert gn == wn
    np.testing.assert_array_equal(u32(gs), ws)
    np.testing.assert_array_equal(u32(gd), wd)
