"""Batched windows (ns_batch_*): per-window quantities and the running
aggregate, bit-exact against the CPU oracle; chunking of the arena; the
autotuner and its cache; replay from a captured CUDA graph."""
from __future__ import annotations

import json
import os
import tempfile

import numpy as np
import pytest
import torch

import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import assert_matrix_equal, to_dev

pytestmark = pytest.mark.gpu


def make_batch(sizes, seed0=0):
    srcs, dsts = [], []
    for w, n in enumerate(sizes):
        s, d = W.batched_window(seed0 + w, int(n), 0.8 + 0.05 * (w % 12), K=1 << 12)
        srcs.append(s)
        dsts.append(d)
    src = np.concatenate(srcs) if srcs else np.zeros(0, np.uint32)
    dst = np.concatenate(dsts) if dsts else np.zeros(0, np.uint32)
    off = np.zeros(len(sizes) + 1, np.uint64)
    off[1:] = np.cumsum(np.asarray(sizes, np.uint64))
    return src, dst, off


def rows_of(t, W_):
    v = t.cpu().numpy().view(np.uint64).reshape(-1, 9)[:W_]
    return [{f: int(x) for f, x in zip(oracle.FIELDS, r)} for r in v]


def expected(src, dst, off):
    per, acc = [], (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for w in range(off.size - 1):
        a, b = int(off[w]), int(off[w + 1])
        m = oracle.build_matrix(src[a:b], dst[a:b])
        per.append(oracle.stats(*m))
        acc = oracle.accumulate(acc, m)
    return per, acc


SIZES = [0, 1, 4095, 4096, 4097, 30000, 5, 0, 70001, 2, 12289, 1023]


def run_batch(ctx, src, dst, off, acc=None, params=None):
    b = ns.Batch(ctx, off.size - 1, int(off[-1]) + 1)
    if params:
        b.set_params(*params)
    out = torch.full(((off.size - 1) * 9,), -1, dtype=torch.int64, device="cuda")
    keep = ns.batch_run(ctx, b, to_dev(src), to_dev(dst), off, out, acc)
    torch.cuda.synchronize()
    del keep
    return b, out


@pytest.mark.parametrize("params", [None, (1024, 8, 0.5), (256, 16, 0.9), (16384, 4, 0.7)])
def test_batch_per_window_and_aggregate(params):
    ctx = ns.Context(0, path="hash")
    src, dst, off = make_batch(SIZES)
    acc = ns.Matrix(ctx)
    b, out = run_batch(ctx, src, dst, off, acc, params)
    per, want_acc = expected(src, dst, off)
    assert rows_of(out, len(SIZES)) == per
    assert ns.network_stats(ctx, acc) == oracle.stats(*want_acc)
    assert_matrix_equal(acc, *want_acc)
    b.free()


def test_batch_equals_plain_per_window_calls():
    ctx = ns.Context(0, path="hash")
    src, dst, off = make_batch([3000, 0, 9000, 17, 40000], seed0=50)
    b, out = run_batch(ctx, src, dst, off)
    got = rows_of(out, 5)
    m = ns.Matrix(ctx)
    for w in range(5):
        a, c = int(off[w]), int(off[w + 1])
        ns.window_build(ctx, to_dev(src[a:c]), to_dev(dst[a:c]), m)
        assert ns.network_stats(ctx, m) == got[w]


def test_batch_many_chunks():
    """A small HBM budget forces the arena to hold a few windows at a time."""
    ctx = ns.Context(0, path="hash", hbm_budget_bytes=48 * (1 << 18))  # 2^18 slots of 48 bytes
    sizes = [20000, 30000, 1, 0, 25000, 40000, 5000]
    src, dst, off = make_batch(sizes, seed0=7)
    acc = ns.Matrix(ctx)
    b, out = run_batch(ctx, src, dst, off, acc)
    per, want_acc = expected(src, dst, off)
    assert rows_of(out, len(sizes)) == per
    assert ns.network_stats(ctx, acc) == oracle.stats(*want_acc)


def test_batch_window_too_large_for_arena():
    ctx = ns.Context(0, path="hash", hbm_budget_bytes=48 * 4096)
    src, dst, off = make_batch([100000], seed0=3)
    b = ns.Batch(ctx, 1, 100001)
    out = torch.zeros(9, dtype=torch.int64, device="cuda")
    with pytest.raises(ns.NsError) as e:
        ns.batch_run(ctx, b, to_dev(src), to_dev(dst), off, out)
    assert e.value.name == "NS_ERR_CAPACITY"


def test_batch_autotune_and_cache():
    with tempfile.TemporaryDirectory() as tmp:
        cache = os.path.join(tmp, "tuner.json")
        ctx = ns.Context(0, path="hash", tuner_cache=cache)
        src, dst, off = make_batch([5000] * 16, seed0=11)
        b = ns.Batch(ctx, 16, int(off[-1]))
        p = ns.batch_tune(ctx, b, to_dev(src), to_dev(dst), off)
        assert p["tile_packets"] in (1024, 2048, 4096, 8192, 16384)
        assert p["ctas_per_sm"] in (4, 8, 16) and p["max_load"] in (0.5, 0.7)
        assert b.params == p
        entries = json.load(open(cache))
        assert len(entries) == 1
        key = next(iter(entries))
        assert "|batch|" in key
        # a new plan of the same shape starts from the cached choice
        b2 = ns.Batch(ctx, 16, int(off[-1]))
        assert b2.params["tile_packets"] == p["tile_packets"]
        assert b2.params["ctas_per_sm"] == p["ctas_per_sm"]
        # and still computes the right answer
        out = torch.zeros(16 * 9, dtype=torch.int64, device="cuda")
        ns.batch_run(ctx, b2, to_dev(src), to_dev(dst), off, out)
        torch.cuda.synchronize()
        assert rows_of(out, 16) == expected(src, dst, off)[0]


def test_batch_in_cuda_graph():
    ctx = ns.Context(0, path="hash")
    src, dst, off = make_batch([7000, 0, 12000, 3, 50000], seed0=21)
    b = ns.Batch(ctx, 5, int(off[-1]))
    acc = ns.Matrix(ctx)
    ns.matrix_reserve(acc, int(off[-1]))
    ds, dd = to_dev(src), to_dev(dst)
    out = torch.zeros(5 * 9, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ns.batch_run(ctx, b, ds, dd, off, out)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ns.matrix_clear(acc)
        keep = ns.batch_run(ctx, b, ds, dd, off, out, acc)
    per, want_acc = expected(src, dst, off)
    for _ in range(2):
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert rows_of(out, 5) == per
        assert ns.network_stats(ctx, acc) == oracle.stats(*want_acc)
    del keep


def test_device_offsets_new_layout_without_recapture():
    """ns_batch_run_device in a captured CUDA graph: one capture, replayed
    with two different window layouts written into the device offsets (the
    same packets cut differently), each equal to the oracle per window and
    in the running aggregate; then offsets past the plan are refused."""
    src, dst, off_a = make_batch([9000, 1, 0, 25000, 4097, 12000, 333], seed0=70)
    total = int(off_a[-1])
    cuts = np.sort(np.random.default_rng(4).integers(0, total, size=6).astype(np.uint64))
    off_b = np.concatenate([[0], cuts, [total]]).astype(np.uint64)  # 7 windows again, other sizes
    Wn = off_a.size - 1
    ctx = ns.Context(0, path="hash")
    b = ns.Batch(ctx, Wn, total)
    acc = ns.Matrix(ctx)
    ns.matrix_reserve(acc, total)
    ds, dd = to_dev(src), to_dev(dst)
    d_off = torch.from_numpy(off_a.view(np.int64).copy()).cuda()
    out = torch.full((Wn * 9,), -1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ns.matrix_clear(acc)
        ns.batch_run_device(ctx, b, ds, dd, d_off, out, acc)  # warm-up outside capture
    torch.cuda.synchronize()
    ns.batch_sync(b)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ns.matrix_clear(acc)
        ns.batch_run_device(ctx, b, ds, dd, d_off, out, acc)
    for off in (off_a, off_b, off_a):
        d_off.copy_(torch.from_numpy(off.view(np.int64).copy()))
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        ns.batch_sync(b)
        per, want_acc = expected(src, dst, off)
        assert rows_of(out, Wn) == per
        assert ns.network_stats(ctx, acc) == oracle.stats(*want_acc)
        assert_matrix_equal(acc, *want_acc)
    # more packets than the plan allows: the run does nothing and reports it
    bad = off_a.copy()
    bad[-1] = total + 1
    d_off.copy_(torch.from_numpy(bad.view(np.int64).copy()))
    g.replay()
    torch.cuda.synchronize()
    with pytest.raises(ns.NsError) as e:
        ns.batch_sync(b)
    assert e.value.name == "NS_ERR_CAPACITY"
    del g
    b.free()
    acc.free()
    ctx.close()


def test_batch_aggregate_by_one_sort_build():
    """A context on the sort path: an empty aggregate receives the batch's
    matrix from one sort-path build of all its packets; a second batch into
    the now non-empty aggregate adds its windows' tables instead.  Per-window
    quantities and the aggregate equal the oracle both times."""
    ctx = ns.Context(0, path="sort")
    src, dst, off = make_batch(SIZES, seed0=90)
    acc = ns.Matrix(ctx)
    b, out = run_batch(ctx, src, dst, off, acc)
    per, want_acc = expected(src, dst, off)
    assert rows_of(out, len(SIZES)) == per
    assert ns.network_stats(ctx, acc) == oracle.stats(*want_acc)
    assert_matrix_equal(acc, *want_acc)
    src2, dst2, off2 = make_batch([30000, 7, 0, 9999], seed0=95)
    b2, out2 = run_batch(ctx, src2, dst2, off2, acc)
    per2, want2 = expected(src2, dst2, off2)
    assert rows_of(out2, 4) == per2
    total = oracle.accumulate(want_acc, want2)
    assert ns.network_stats(ctx, acc) == oracle.stats(*total)
    assert_matrix_equal(acc, *total)
    b.free()
    b2.free()


@pytest.mark.parametrize("digits", ["8", "wide"])
def test_batch_aggregate_by_sort_in_cuda_graph_with_new_packets(digits):
    """The same, captured in a CUDA graph (aggregate cleared inside it) and
    replayed on packets with new contents but the same window layout, with
    either digit plan."""
    ctx = ns.Context(0, path="sort", sort_split="on", sort_digits=digits)
    sizes = [70000, 0, 5000, 131072, 3]
    src, dst, off = make_batch(sizes, seed0=101)
    src2, dst2, _ = make_batch(sizes, seed0=202)
    Wn, total = len(sizes), int(off[-1])
    b = ns.Batch(ctx, Wn, total)
    acc = ns.Matrix(ctx)
    ds, dd = to_dev(src), to_dev(dst)
    out = torch.full((Wn * 9,), -1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ns.matrix_clear(acc)
        ns.batch_run(ctx, b, ds, dd, off, out, acc)  # outside capture: every buffer reaches its size
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ns.matrix_clear(acc)
        keep = ns.batch_run(ctx, b, ds, dd, off, out, acc)
    for a, c in ((src2, dst2), (src, dst), (src2, dst2)):
        ds.copy_(to_dev(a))
        dd.copy_(to_dev(c))
        out.fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        per, want_acc = expected(a, c, off)
        assert rows_of(out, Wn) == per
        assert ns.network_stats(ctx, acc) == oracle.stats(*want_acc)
        assert_matrix_equal(acc, *want_acc)
    del keep
    b.free()
