"""Parity at the full workload sizes, in the launch configurations bench.py
times.  The oracle's all-cores variant (pinned to the single-thread oracle on
the CPU) computes the whole-workload references; per-window references run
the single-thread oracle on a pool of host threads (the oracle's C calls
release the interpreter lock).  Where a reference would take too long even
so (every prefix of a stream), sampled windows are compared and properties
that hold at any size are checked for the rest."""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import export_np, stats_row, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def oracle_per_window(windows):
    """oracle.stats_of_packets of every (src, dst) window, on all host cores."""
    with ThreadPoolExecutor(max_workers=oracle.hardware_threads()) as ex:
        return list(ex.map(lambda sd: oracle.stats_of_packets(*sd), windows))


def pinned_pair(n):
    s = torch.empty(n, dtype=torch.int32).pin_memory()
    d = torch.empty(n, dtype=torch.int32).pin_memory()
    return s, d, s.numpy().view(np.uint32), d.numpy().view(np.uint32)


def test_stream_512_windows_of_2p17():
    """Workload 2 as bench.py runs it: one ns_window_ingest_stats launch per
    window.  Exact A after all windows; exact running quantities after
    sampled windows; invariants after every window."""
    NW, WIN = W.W2_WINDOWS, W.W2_WINDOW
    N = NW * WIN
    hs, hd, s, d = pinned_pair(N)
    W.rmat_stream(N, src=s, dst=d)
    ds, dd = hs.cuda(), hd.cuda()
    ctx = ns.Context(0, path="hash", hash_load=0.25)  # bench.py's table sizing
    A = ns.Matrix(ctx)
    ns.matrix_reserve(A, N)
    rows = torch.zeros(NW, 16, dtype=torch.int64, device="cuda")
    for w in range(NW):
        sl = slice(w * WIN, (w + 1) * WIN)
        ns.window_ingest_stats(ctx, A, ds[sl], dd[sl], rows[w])
    torch.cuda.synchronize()
    got = rows.cpu().numpy().view(np.uint64)[:, :9]
    # invariants after every window
    assert np.array_equal(got[:, 0], (np.arange(NW, dtype=np.uint64) + 1) * WIN)
    assert np.all(np.diff(got.astype(np.int64), axis=0) >= 0)  # monotone running quantities
    assert np.all(got[:, 1] <= got[:, 0]) and np.all(got[:, 5] <= got[:, 3]) and np.all(got[:, 7] <= got[:, 2])
    # sampled windows against the oracle's prefix
    for w in (0, 1, 2, 100, 255):
        k, c = oracle.build_matrix(s[: (w + 1) * WIN], d[: (w + 1) * WIN])
        assert stats_row(rows[w]) == oracle.stats(k, c), w
    # the whole stream: A's nonzeros and the last window's quantities
    k, c = oracle.build_matrix(s, d)
    assert stats_row(rows[NW - 1]) == oracle.stats(k, c)
    gk, gc = export_np(A)
    np.testing.assert_array_equal(gk, k)
    np.testing.assert_array_equal(gc, c)


def test_oneshot_2p30_both_paths():
    """Workload 3: 2^30 packets, in the configuration bench.py times.  Both
    paths (the sort path with each digit plan) against the oracle: the nine
    quantities and A's sorted nonzero list, element by element."""
    N = W.W3_N
    hs, hd, s, d = pinned_pair(N)
    W.large_build(N, src=s, dst=d)
    wk, wc = oracle.build_matrix_parallel(s, d)
    want = oracle.stats_parallel(wk, wc)
    assert want["valid_packets"] == N
    ds, dd = hs.cuda(), hd.cuda()
    for path, digits in (("sort", "8"), ("sort", "wide"), ("hash", "auto")):
        ctx = ns.Context(0, path=path, sort_digits=digits)
        m = ns.Matrix(ctx)
        ns.window_build(ctx, ds, dd, m)
        assert ns.network_stats(ctx, m) == want, (path, digits)
        k, c = export_np(m)
        assert k.size == wk.size, (path, digits)
        np.testing.assert_array_equal(k, wk)
        np.testing.assert_array_equal(c, wc)
        del k, c
        m.free()
        ctx.close()
        torch.cuda.empty_cache()


def test_batched_8192_windows():
    """Workload 4: the batched launch against the oracle on every window and
    on the running aggregate (its nine quantities and its nonzero list), and
    against plain per-window launches."""
    sizes, svals = W.batched_plan()
    Wn = sizes.size
    off = np.zeros(Wn + 1, np.uint64)
    off[1:] = np.cumsum(sizes)
    total = int(off[-1])
    hs, hd, s, d = pinned_pair(total)
    for w in range(Wn):
        a, b = int(off[w]), int(off[w + 1])
        W.batched_window(w, b - a, float(svals[w]), src=s[a:b], dst=d[a:b])
    ds, dd = hs.cuda(), hd.cuda()
    ctx = ns.Context(0, path="hash", hbm_budget_bytes=96 << 30)
    acc = ns.Matrix(ctx)
    ns.matrix_reserve_ex(acc, total, 1 << 21)
    batch = ns.Batch(ctx, Wn, total)
    out_b = torch.zeros(Wn * 9, dtype=torch.int64, device="cuda")
    ns.batch_run(ctx, batch, ds, dd, off, out_b, acc)
    torch.cuda.synchronize()
    agg_b = ns.network_stats(ctx, acc)
    batch.free()
    # plain per-window launches
    out_p = torch.zeros(Wn * 9, dtype=torch.int64, device="cuda")
    ns.matrix_clear(acc)
    At = ns.Matrix(ctx)
    for w in range(Wn):
        a, b = int(off[w]), int(off[w + 1])
        ns.window_build(ctx, ds[a:b], dd[a:b], At)
        ns.network_stats_async(ctx, At, out_p[w * 9:(w + 1) * 9])
        ns.accumulate(ctx, acc, At)
    torch.cuda.synchronize()
    assert torch.equal(out_b, out_p)
    assert ns.network_stats(ctx, acc) == agg_b
    assert agg_b["valid_packets"] == total
    rows = out_b.cpu().numpy().view(np.uint64).reshape(Wn, 9)
    assert np.array_equal(rows[:, 0], sizes.astype(np.uint64))
    # every window against the oracle
    wants = oracle_per_window([(s[int(off[w]):int(off[w + 1])], d[int(off[w]):int(off[w + 1])]) for w in range(Wn)])
    for w in range(Wn):
        assert {f: int(x) for f, x in zip(oracle.FIELDS, rows[w])} == wants[w], w
    # the running aggregate: the matrix of the concatenated windows
    wk, wc = oracle.build_matrix_parallel(s, d)
    assert agg_b == oracle.stats_parallel(wk, wc)
    gk, gc = export_np(acc)
    np.testing.assert_array_equal(gk, wk)
    np.testing.assert_array_equal(gc, wc)


def test_serving_448_windows():
    """Workload 5 windows through the service (8 slots): every window's
    per-window quantities equal the oracle's and an independent build; the
    running quantities after sampled windows and after the last one equal
    the oracle's for the concatenated windows."""
    Wn = 448
    sizes, _ = W.serving_plan(Wn, 1.0)
    wins = []
    for w in range(Wn):
        s, d = W.serving_window(w, int(sizes[w]))
        wins.append((torch.from_numpy(s.view(np.int32)).pin_memory(), torch.from_numpy(d.view(np.int32)).pin_memory()))
    ctx = ns.Context(0, path="hash", max_slots=8, hbm_budget_bytes=64 << 30)
    acc = ns.Matrix(ctx)
    ns.matrix_reserve(acc, int(sizes.sum()))
    srv = ns.Server(ctx, acc)
    results = [None] * Wn
    pending = []  # (window, ticket) in submission order
    for w, (s, d) in enumerate(wins):
        while True:
            try:
                pending.append((w, ns.stream_submit(srv, s, d, w)))
                break
            except ns.NsError as e:  # queue full: wait for the oldest window
                assert e.name == "NS_ERR_BUSY"
                pw, t = pending.pop(0)
                results[pw] = ns.stream_wait(srv, t)
    for pw, t in pending:
        results[pw] = ns.stream_wait(srv, t)
    srv.close()
    ref = ns.Context(0, path="hash")
    m, tot = ns.Matrix(ref), ns.Matrix(ref)
    for w, (s, d) in enumerate(wins):
        ds, dd = s.cuda(), d.cuda()
        ns.window_build(ref, ds, dd, m)
        assert results[w][0] == ns.network_stats(ref, m), w
        ns.window_ingest(ref, tot, ds, dd)
    assert results[-1][1] == ns.network_stats(ref, tot)
    # every window's own quantities against the oracle
    host = [(s.numpy().view(np.uint32), d.numpy().view(np.uint32)) for s, d in wins]
    wants = oracle_per_window(host)
    for w in range(Wn):
        assert results[w][0] == wants[w], w
    # running quantities: A after sampled windows and after the last one
    for w in (0, 7, 200, Wn - 1):
        k, c = oracle.build_matrix_parallel(np.concatenate([h[0] for h in host[:w + 1]]),
                                            np.concatenate([h[1] for h in host[:w + 1]]))
        assert results[w][1] == oracle.stats_parallel(k, c), w


def test_anonymize_2p30():
    """Anonymization of the one-shot build's 2^30 packets, as bench.py times
    it.  The distinct-address count equals numpy's; sampled packets carry the
    label their address's random key ranks to (computed one by one from the
    definition); labels are a bijection; the nine quantities are unchanged."""
    import gen
    N = W.W3_N
    hs, hd, s, d = pinned_pair(N)
    W.large_build(N, src=s, dst=d)
    rnd = torch.empty(2 * N, dtype=torch.int64).pin_memory()
    gen.random_u64(2 * N, W.seed_of(3), 9, out=rnd.numpy().view(np.uint64))
    ds, dd, dr = hs.cuda(), hd.cuda(), rnd.cuda()
    ctx = ns.Context(0)
    os_, od, nu = ns.anonymize(ctx, ds, dd, dr)
    u = np.union1d(np.unique(s), np.unique(d))
    assert nu == u.size
    r = rnd.numpy().view(np.uint64)[:nu]
    rank = np.empty(nu, np.int64)
    rank[np.argsort(r, kind="stable")] = np.arange(nu)
    rng = np.random.default_rng(5)
    pick = rng.integers(0, N, 4096)
    got_s = os_[torch.from_numpy(pick).cuda()].cpu().numpy().view(np.uint32)
    got_d = od[torch.from_numpy(pick).cuda()].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got_s, rank[np.searchsorted(u, s[pick])].astype(np.uint32))
    np.testing.assert_array_equal(got_d, rank[np.searchsorted(u, d[pick])].astype(np.uint32))
    # labels stay below nu, and the relabelled build has the same quantities
    assert int(os_.view(torch.int32).max().item()) < nu or nu > 2**31
    ctx_s = ns.Context(0, path="sort")
    a, b = ns.Matrix(ctx_s), ns.Matrix(ctx_s)
    ns.window_build(ctx_s, ds, dd, a)
    ns.window_build(ctx_s, os_, od, b)
    assert ns.network_stats(ctx_s, a) == ns.network_stats(ctx_s, b)


def test_slide_512_windows_k8():
    """The slide workload as bench.py runs it (512 windows of 2^17 RMAT
    packets, K = 8, no CTA staging): sampled windows' own and sliding-window
    quantities against the oracle; every window's valid counts."""
    NW, WIN, K = W.W2_WINDOWS, W.W2_WINDOW, 8
    N = NW * WIN
    hs, hd, s, d = pinned_pair(N)
    W.rmat_stream(N, src=s, dst=d)
    ds, dd = hs.cuda(), hd.cuda()
    ctx = ns.Context(0, path="hash", cta_cache="off")
    sl = ns.Slider(ctx, K)
    ow = torch.zeros(NW, 16, dtype=torch.int64, device="cuda")
    osl = torch.zeros(NW, 16, dtype=torch.int64, device="cuda")
    for w in range(NW):
        a = w * WIN
        ns.slider_push(ctx, sl, ds[a:a + WIN], dd[a:a + WIN], ow[w], osl[w])
    torch.cuda.synchronize()
    rw = ow.cpu().numpy().view(np.uint64)[:, :9]
    rs = osl.cpu().numpy().view(np.uint64)[:, :9]
    assert np.all(rw[:, 0] == WIN)
    assert np.array_equal(rs[:, 0], np.minimum(np.arange(NW) + 1, K).astype(np.uint64) * WIN)
    for w in (0, 3, 7, 8, 300, NW - 1):
        a, b = max(0, w + 1 - K) * WIN, (w + 1) * WIN
        assert {f: int(x) for f, x in zip(oracle.FIELDS, rs[w])} == oracle.stats_of_packets(s[a:b], d[a:b]), w
        c = w * WIN
        assert {f: int(x) for f, x in zip(oracle.FIELDS, rw[w])} == oracle.stats_of_packets(s[c:c + WIN], d[c:c + WIN]), w


def test_sort_one_repeated_key_2p28():
    """2^28 copies of one packet through the sort path: the closed form
    (N, 1, 1, 1, N, 1, N, 1) with max link N, and A = [(key, N)].  At this
    size every histogram CTA flushes its shared counters mid-launch, and
    each 16-bit half reaches its bound (one digit value takes every count);
    the stable passes see one digit per warp and the unstable first pass
    sends every key to one cursor."""
    N = 1 << 28
    s_val, d_val = 0xDEADBEEF, 0x12345678
    ds = torch.full((N,), s_val - (1 << 32), dtype=torch.int32, device="cuda")
    dd = torch.full((N,), d_val, dtype=torch.int32, device="cuda")
    ctx = ns.Context(0, path="sort")
    m = ns.Matrix(ctx)
    ns.window_build(ctx, ds, dd, m)
    st = ns.network_stats(ctx, m)
    assert st == {"valid_packets": N, "unique_links": 1, "unique_sources": 1, "unique_destinations": 1,
                  "max_src_packets": N, "max_src_fanout": 1, "max_dst_packets": N, "max_dst_fanin": 1,
                  "max_link_packets": N}
    k, c = export_np(m)
    np.testing.assert_array_equal(k, np.array([(s_val << 32) | d_val], dtype=np.uint64))
    np.testing.assert_array_equal(c, np.array([N], dtype=np.uint64))
