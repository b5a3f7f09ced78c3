"""Streaming service (ns_server / ns_stream_*): every window's results are
the same alone and in the mix -- per-window quantities equal the oracle's
for that window, running quantities equal the oracle's for the windows
submitted up to it -- plus the timeout and admission-budget paths."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import assert_matrix_equal

pytestmark = pytest.mark.gpu


def windows():
    out = []
    sizes = [4096, 1, 0, 70001, 12289, 300000, 5, 65536, 200000, 777]
    for w, n in enumerate(sizes):
        if w % 2:
            s, d = W.serving_window(w, n)
        else:
            s, d = W.zipf_window(n, 1.2, 1 << 12, 900 + w)
        out.append((s, d))
    return out


def expected(ws):
    per, run = [], []
    acc = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for s, d in ws:
        m = oracle.build_matrix(s, d)
        per.append(oracle.stats(*m))
        acc = oracle.accumulate(acc, m)
        run.append(oracle.stats(*acc))
    return per, run, acc


def serve(ws, slots, alone, pinned=False):
    ctx = ns.Context(0, path="hash", max_slots=slots)
    acc = ns.Matrix(ctx)
    srv = ns.Server(ctx, acc)
    results = []
    host = []
    for s, d in ws:
        if pinned:
            s = torch.from_numpy(s.view(np.int32)).pin_memory()
            d = torch.from_numpy(d.view(np.int32)).pin_memory()
        host.append((s, d))
    if alone:
        for w, (s, d) in enumerate(host):
            t = ns.stream_submit(srv, s, d, window_id=w)
            results.append(ns.stream_wait(srv, t))
    else:
        tickets = [ns.stream_submit(srv, s, d, window_id=w) for w, (s, d) in enumerate(host)]
        results = [ns.stream_wait(srv, t) for t in tickets]
    srv.close()
    return ctx, acc, results


@pytest.mark.parametrize("pinned", [False, True])
def test_alone_and_in_the_mix_agree(pinned):
    ws = windows()
    per, run, want_acc = expected(ws)
    ctx1, acc1, alone = serve(ws, 1, True, pinned)
    ctx4, acc4, mix = serve(ws, 4, False, pinned)
    for w in range(len(ws)):
        assert alone[w][0] == per[w] and mix[w][0] == per[w], w
        assert alone[w][1] == run[w] and mix[w][1] == run[w], w
        for _, _, tm in (alone[w], mix[w]):
            assert tm["window_id"] == w
            assert tm["submit_us"] <= tm["admit_us"] <= tm["complete_us"]
    assert ns.network_stats(ctx4, acc4) == oracle.stats(*want_acc)
    assert_matrix_equal(acc4, *want_acc)
    assert_matrix_equal(acc1, *want_acc)


def test_wait_timeout_keeps_ticket():
    ctx = ns.Context(0, path="hash", max_slots=2)
    acc = ns.Matrix(ctx)
    srv = ns.Server(ctx, acc)
    s, d = W.serving_window(1, 1 << 22)
    t = ns.stream_submit(srv, s, d)
    try:
        ns.stream_wait(srv, t, timeout_us=0)
        timed_out = False
    except ns.NsError as e:
        assert e.name == "NS_ERR_TIMEOUT"
        timed_out = True
    if timed_out:
        pw, rn, _ = ns.stream_wait(srv, t)
        assert pw["valid_packets"] == 1 << 22 and rn == pw
    srv.close()


def test_window_over_budget_is_rejected():
    ctx = ns.Context(0, path="hash", max_slots=2, hbm_budget_bytes=1 << 20)
    acc = ns.Matrix(ctx)
    srv = ns.Server(ctx, acc)
    s, d = W.serving_window(2, 1 << 18)
    t = ns.stream_submit(srv, s, d)
    with pytest.raises(ns.NsError) as e:
        ns.stream_wait(srv, t)
    assert e.value.name == "NS_ERR_OOM"
    # a window that fits still works afterwards
    s2, d2 = W.serving_window(3, 1000)
    t2 = ns.stream_submit(srv, s2, d2)
    pw, rn, _ = ns.stream_wait(srv, t2)
    assert pw == oracle.stats(*oracle.build_matrix(s2, d2))
    srv.close()


def test_server_reserve_then_windows_match_oracle():
    """Slots sized up front (ns_server_reserve) serve windows up to that size
    with the oracle's per-window and running quantities; reserving again
    once the service is idle is allowed."""
    ctx = ns.Context(0, path="hash")
    acc = ns.Matrix(ctx)
    srv = ns.Server(ctx, acc)
    sizes = [30000, 1, 0, 65536, 12345]
    srv.reserve(max(sizes))
    want = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for w, n in enumerate(sizes):
        s, d = W.serving_window(w, n)
        pw, run, _ = ns.stream_wait(srv, ns.stream_submit(srv, s, d, w))
        m = oracle.build_matrix(s, d)
        want = oracle.accumulate(want, m)
        assert pw == oracle.stats(*m) and run == oracle.stats(*want), w
    srv.reserve(1 << 18)  # idle again: allowed
    srv.clear()  # A = 0: the next window's running quantities are its own
    s, d = W.serving_window(99, 4000)
    pw, run, _ = ns.stream_wait(srv, ns.stream_submit(srv, s, d, 99))
    assert pw == run == oracle.stats_of_packets(s, d)
    srv.close()


def test_slots_regrow_mid_stream_without_reserve():
    """No ns_server_reserve: window sizes keep growing, so every slot frees
    and regrows its buffers and tables (stream-ordered, on its own stream)
    while other slots have windows in flight.  Every window's results still
    equal the oracle's, alone and running."""
    sizes = [int(64 * 1.6 ** k) for k in range(24)]  # 64 .. ~5.7e6 packets
    ws = []
    for w, n in enumerate(sizes):
        ws.append(W.serving_window(w, n) if w % 3 else W.zipf_window(n, 1.1, 1 << 16, 77 + w))
    per, run, acc_want = expected(ws)
    ctx = ns.Context(0, path="hash", max_slots=4)
    acc = ns.Matrix(ctx)
    srv = ns.Server(ctx, acc)
    host = [(torch.from_numpy(s.view(np.int32)).pin_memory(), torch.from_numpy(d.view(np.int32)).pin_memory())
            for s, d in ws]
    tickets = []
    for w, (s, d) in enumerate(host):
        while True:
            try:
                tickets.append(ns.stream_submit(srv, s, d, window_id=w))
                break
            except ns.NsError as e:
                assert e.name == "NS_ERR_BUSY"
                torch.cuda.synchronize()
    results = [ns.stream_wait(srv, t) for t in tickets]
    srv.close()
    for w, (pw, rn, _) in enumerate(results):
        assert pw == per[w], w
        assert rn == run[w], w
    assert_matrix_equal(acc, *acc_want)
    acc.free()
    ctx.close()

