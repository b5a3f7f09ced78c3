"""Checkpoint and resume of a traffic matrix (ns_matrix_save / ns_matrix_load).

A stream is accumulated for a few windows, saved, loaded into a matrix of a
fresh context, and both copies are fed the rest of the stream: after every
window they must agree with each other and with the oracle, bit for bit.
Malformed checkpoints are rejected and leave the target matrix unchanged."""
from __future__ import annotations

import os
import struct

import numpy as np
import pytest

import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import assert_matrix_equal, export_np, to_dev

pytestmark = pytest.mark.gpu

WIN = 1 << 14


@pytest.mark.parametrize("path", ["hash", "sort"])
def test_save_load_resume_equals_uninterrupted(tmp_path, path):
    n_win = 6
    s, d = W.rmat_stream(n_win * WIN)
    ctx = ns.Context(0, path=path)
    acc = ns.Matrix(ctx)
    for w in range(3):
        ns.window_ingest(ctx, acc, to_dev(s[w * WIN:(w + 1) * WIN]), to_dev(d[w * WIN:(w + 1) * WIN]))
    ck = str(tmp_path / "a.nsm")
    ns.matrix_save(acc, ck)
    want3 = oracle.build_matrix(s[:3 * WIN], d[:3 * WIN])
    # the file: header, then keys and counts
    raw = open(ck, "rb").read()
    assert raw[:8] == b"NSMATRIX" and struct.unpack_from("<II", raw, 8) == (1, 128)
    assert struct.unpack_from("<Q", raw, 16)[0] == want3[0].size
    assert len(raw) == 128 + 16 * want3[0].size
    # resume in a fresh context
    ctx2 = ns.Context(0, path="hash")
    res = ns.Matrix(ctx2)
    ns.matrix_load(ctx2, ck, res)
    assert ns.network_stats(ctx2, res) == oracle.stats(*want3)
    assert_matrix_equal(res, *want3)
    for w in range(3, n_win):
        a, b = w * WIN, (w + 1) * WIN
        ns.window_ingest(ctx, acc, to_dev(s[a:b]), to_dev(d[a:b]))
        ns.window_ingest(ctx2, res, to_dev(s[a:b]), to_dev(d[a:b]))
        want = oracle.build_matrix(s[:b], d[:b])
        assert ns.network_stats(ctx, acc) == ns.network_stats(ctx2, res) == oracle.stats(*want)
    k1, c1 = export_np(acc)
    k2, c2 = export_np(res)
    np.testing.assert_array_equal(k1, k2)
    np.testing.assert_array_equal(c1, c2)
    res.free()
    acc.free()
    ctx2.close()
    ctx.close()


def test_sorted_list_matrix_and_empty_matrix_round_trip(tmp_path):
    ctx = ns.Context(0, path="sort")
    s, d = W.single_window(50001)
    m = ns.Matrix(ctx)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)  # a sorted-list matrix
    ck = str(tmp_path / "b.nsm")
    ns.matrix_save(m, ck)
    r = ns.Matrix(ctx)
    ns.matrix_load(ctx, ck, r)
    want = oracle.build_matrix(s, d)
    assert ns.network_stats(ctx, r) == oracle.stats(*want)
    assert_matrix_equal(r, *want)
    # an empty matrix saves and loads as empty
    e = ns.Matrix(ctx)
    ns.matrix_save(e, str(tmp_path / "e.nsm"))
    ns.matrix_load(ctx, str(tmp_path / "e.nsm"), r)
    assert ns.network_stats(ctx, r) == oracle.stats(np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for x in (m, r, e):
        x.free()
    ctx.close()


def test_load_on_a_side_stream(tmp_path):
    """Loading on a non-blocking stream: the entries' copies are ordered
    with the insert that reads them, so the loaded matrix is exact however
    busy the device is (a large kernel is queued on the same stream first)."""
    import torch

    ctx = ns.Context(0, path="hash")
    s, d = W.rmat_stream(1 << 20)
    m = ns.Matrix(ctx)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)
    ck = str(tmp_path / "side.nsm")
    ns.matrix_save(m, ck)
    want = oracle.build_matrix(s, d)
    side = torch.cuda.Stream()
    busy = torch.empty(1 << 26, dtype=torch.float32, device="cuda")
    for _ in range(3):
        r = ns.Matrix(ctx)
        with torch.cuda.stream(side):
            busy.uniform_()  # keeps the side stream busy ahead of the load
            ns.matrix_load(ctx, ck, r, stream=side)
            got = ns.network_stats(ctx, r, stream=side)
        assert got == oracle.stats(*want)
        assert_matrix_equal(r, *want)
        r.free()
    m.free()
    ctx.close()


def test_malformed_checkpoints_are_rejected(tmp_path):
    ctx = ns.Context(0, path="hash")
    s, d = W.single_window(20000)
    m = ns.Matrix(ctx)
    ns.window_ingest(ctx, m, to_dev(s), to_dev(d))
    ck = str(tmp_path / "c.nsm")
    ns.matrix_save(m, ck)
    raw = bytearray(open(ck, "rb").read())
    nnz = struct.unpack_from("<Q", raw, 16)[0]
    target = ns.Matrix(ctx)
    ns.window_ingest(ctx, target, to_dev(s[:100]), to_dev(d[:100]))
    before = ns.network_stats(ctx, target)

    def load(data, name):
        p = str(tmp_path / name)
        with open(p, "wb") as f:
            f.write(bytes(data))
        with pytest.raises(ns.NsError) as e:
            ns.matrix_load(ctx, p, target)
        return e.value

    bad = raw.copy()
    bad[0] = ord("X")
    assert load(bad, "magic.nsm").name == "NS_ERR_INVALID"
    bad = raw.copy()
    struct.pack_into("<I", bad, 8, 99)
    assert load(bad, "version.nsm").name == "NS_ERR_INVALID"
    assert load(raw[:-8], "short.nsm").name == "NS_ERR_INVALID"
    bad = raw.copy()  # two keys swapped: not ascending
    k0, k1 = struct.unpack_from("<QQ", bad, 128)
    struct.pack_into("<QQ", bad, 128, k1, k0)
    assert load(bad, "order.nsm").name == "NS_ERR_INVALID"
    bad = raw.copy()  # a zero count
    struct.pack_into("<Q", bad, 128 + 8 * nnz, 0)
    assert load(bad, "zero.nsm").name == "NS_ERR_INVALID"
    assert ns.network_stats(ctx, target) == before  # rejected files leave the matrix unchanged
    bad = raw.copy()  # a count raised by one: the recomputed valid packets differ from the header
    c0 = struct.unpack_from("<Q", bad, 128 + 8 * nnz)[0]
    struct.pack_into("<Q", bad, 128 + 8 * nnz, c0 + 1)
    assert load(bad, "count.nsm").name == "NS_ERR_INVALID"
    with pytest.raises(ns.NsError) as e:
        ns.matrix_load(ctx, str(tmp_path / "missing.nsm"), target)
    assert e.value.name == "NS_ERR_IO"
    # the intact file still loads
    ns.matrix_load(ctx, ck, target)
    assert ns.network_stats(ctx, target) == oracle.stats_of_packets(s, d)
    assert not os.path.exists(ck + ".partial")
    m.free()
    target.free()
    ctx.close()
