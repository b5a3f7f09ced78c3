"""The sort path's hot-key split against the oracle: A's sorted nonzero list
and the nine quantities, element by element, with the split forced on and
off, on skewed and uniform windows of several sizes (ragged tails, sizes at
the split's lower bound), unaligned columns, and the degenerate cases --
every packet hot (nothing left to sort), no key hot, the extreme keys 0 and
2^64 - 1 heavy (2^64 - 1 marks a free slot of the hot table and is never
made hot)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen
import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import export_np, to_dev

pytestmark = pytest.mark.gpu


def check(ctx, s, d, m=None):
    m = m or ns.Matrix(ctx)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)
    got = ns.network_stats(ctx, m)
    wk, wc = oracle.build_matrix(s, d)
    assert got == oracle.stats(wk, wc)
    k, c = export_np(m)
    np.testing.assert_array_equal(k, wk)
    np.testing.assert_array_equal(c, wc)
    return ns.sort_split_info(ctx)


@pytest.mark.parametrize("n", [1 << 16, (1 << 16) + 1, 300001, 1 << 20, 3 * (1 << 20) + 17])
@pytest.mark.parametrize("split", ["on", "off"])
def test_split_matches_oracle_zipf(n, split):
    ctx = ns.Context(0, path="sort", sort_split=split)
    s, d = W.zipf_window(n, 1.2, 1 << 16, 77 + n)
    info = check(ctx, s, d)
    assert info["used"] == (split == "on")
    if split == "on":
        assert info["hot_keys"] > 0
        assert 0 <= info["cold_packets"] < n
    ctx.close()


def test_split_small_window_never_splits():
    ctx = ns.Context(0, path="sort", sort_split="on")
    s, d = W.zipf_window((1 << 16) - 1, 1.2, 1 << 10, 5)
    assert not check(ctx, s, d)["used"]
    ctx.close()


def test_split_uniform_has_no_hot_keys():
    ctx = ns.Context(0, path="sort", sort_split="on")
    s, d = gen.uniform_pairs(1 << 20, 32, 9)
    info = check(ctx, s, d)
    assert info["used"] and info["hot_keys"] == 0 and info["cold_packets"] == 1 << 20
    ctx.close()


def test_split_every_packet_hot():
    n = (1 << 18) + 3
    s = np.full(n, 0xDEADBEEF, np.uint32)
    d = np.full(n, 0x01020304, np.uint32)
    ctx = ns.Context(0, path="sort", sort_split="on")
    info = check(ctx, s, d)
    assert info["hot_keys"] == 1 and info["cold_packets"] == 0
    ctx.close()


def test_split_extreme_keys_heavy():
    n = 1 << 20
    s, d = W.zipf_window(n, 1.1, 1 << 12, 13)
    s, d = s.copy(), d.copy()
    s[::3] = 0xFFFFFFFF  # key 2^64 - 1 on a third of the packets
    d[::3] = 0xFFFFFFFF
    s[1::5] = 0  # key 0 on a fifth
    d[1::5] = 0
    ctx = ns.Context(0, path="sort", sort_split="on")
    info = check(ctx, s, d)
    assert info["hot_keys"] > 0
    ctx.close()


def test_split_unaligned_columns_and_rebuild():
    n = (1 << 20) + 5
    s, d = W.zipf_window(n + 1, 1.3, 1 << 14, 21)
    ts, td = to_dev(s), to_dev(d)
    ctx = ns.Context(0, path="sort", sort_split="on")
    m = ns.Matrix(ctx)
    for off in (1, 0):  # 4-byte offset: the split loads packets one by one
        ns.window_build(ctx, ts[off:off + n], td[off:off + n], m)
        wk, wc = oracle.build_matrix(s[off:off + n], d[off:off + n])
        assert ns.network_stats(ctx, m) == oracle.stats(wk, wc)
        k, c = export_np(m)
        np.testing.assert_array_equal(k, wk)
        np.testing.assert_array_equal(c, wc)
    ctx.close()


def test_split_rmat_and_accumulate():
    """An RMAT window through the split, then summed with a second one."""
    ctx = ns.Context(0, path="sort", sort_split="on")
    s, d = W.rmat_stream(1 << 21)
    a, b = ns.Matrix(ctx), ns.Matrix(ctx)
    half = 1 << 20
    ns.window_build(ctx, to_dev(s[:half]), to_dev(d[:half]), a)
    ns.window_build(ctx, to_dev(s[half:]), to_dev(d[half:]), b)
    ns.accumulate(ctx, a, b)
    wk, wc = oracle.build_matrix(s, d)
    assert ns.network_stats(ctx, a) == oracle.stats(wk, wc)
    k, c = export_np(a)
    np.testing.assert_array_equal(k, wk)
    np.testing.assert_array_equal(c, wc)
    ctx.close()


def test_path_tune_records_split_choice(tmp_path):
    cache = str(tmp_path / "tuner.json")
    ctx = ns.Context(0, tuner_cache=cache)
    s, d = W.zipf_window(1 << 22, 1.2, 1 << 20, 3)
    ns.path_tune(ctx, to_dev(s), to_dev(d))
    text = open(cache).read()
    assert '"sort_split"' in text and '"sort_split_ms"' in text and '"sort_tile"' in text
    # a context on the same cache takes the recorded choices, and still builds exactly
    ctx2 = ns.Context(0, tuner_cache=cache)
    check(ctx2, s, d)
    ctx.close()
    ctx2.close()


@pytest.mark.parametrize("tile", ["512x16", "512x12", "256x16"])
@pytest.mark.parametrize("split", ["on", "off"])
def test_every_tile_shape_matches_oracle(tile, split):
    """Each digit-pass tile the path tuner can choose (threads x keys per
    thread), with and without the split, on a ragged skewed window and on a
    window of all-distinct links."""
    ctx = ns.Context(0, path="sort", sort_split=split, sort_tile=tile)
    s, d = W.zipf_window((1 << 20) + 77, 1.2, 1 << 16, 31)
    check(ctx, s, d)
    s, d = gen.uniform_pairs(300007, 32, 12)
    check(ctx, s, d)
    ctx.close()


def test_split_second_tier_takes_warm_keys():
    """More heavy links than the shared-memory tier holds (6144 keys): the
    global-memory tier takes the next ones, and A is still exact."""
    s, d = W.zipf_window(1 << 22, 1.1, 1 << 18, 41)
    ctx = ns.Context(0, path="sort", sort_split="on")
    info = check(ctx, s, d)
    assert info["hot_keys"] > 6144
    ctx.close()


def test_split_tiers_with_tied_sample_counts():
    """60,000 links of exactly 32 packets each, shuffled into uniform filler:
    the sample sees them all about equally often, so the tier thresholds
    fall inside a histogram bin's ties; whatever each tier takes, A is
    exact."""
    rng = np.random.default_rng(5)
    k = 60000
    hs = rng.integers(0, 1 << 32, k, dtype=np.uint64).astype(np.uint32)
    hd = rng.integers(0, 1 << 32, k, dtype=np.uint64).astype(np.uint32)
    n = 1 << 21
    s = np.empty(n, np.uint32)
    d = np.empty(n, np.uint32)
    s[:32 * k] = np.repeat(hs, 32)
    d[:32 * k] = np.repeat(hd, 32)
    s[32 * k:] = rng.integers(0, 1 << 32, n - 32 * k, dtype=np.uint64).astype(np.uint32)
    d[32 * k:] = rng.integers(0, 1 << 32, n - 32 * k, dtype=np.uint64).astype(np.uint32)
    p = rng.permutation(n)
    s, d = s[p], d[p]
    ctx = ns.Context(0, path="sort", sort_split="on")
    info = check(ctx, s, d)
    assert info["hot_keys"] > 6144 and info["cold_packets"] < n
    ctx.close()


def test_split_extreme_keys_in_second_tier():
    """Keys 0 and 2^64 - 1 at middling frequency (one packet in 500 each),
    below the heaviest links: 0 can be a tier-2 key, 2^64 - 1 never is (it
    marks free slots), and both still count exactly."""
    n = 1 << 22
    s, d = W.zipf_window(n, 1.2, 1 << 16, 23)
    s, d = s.copy(), d.copy()
    s[::500] = 0xFFFFFFFF
    d[::500] = 0xFFFFFFFF
    s[7::500] = 0
    d[7::500] = 0
    ctx = ns.Context(0, path="sort", sort_split="on")
    info = check(ctx, s, d)
    assert info["hot_keys"] > 6144
    ctx.close()


def test_split_interleaved_sample_runs_are_harmless():
    """The sample is grouped by the upper half of each key times an odd
    constant c (mod 2^64).  For keys k + t c^-1 (t = 0, 1, 2) those products
    differ by t and share their upper half, so their sample occurrences
    interleave and each such key can become a candidate more than once, in
    one tier or in both.  Groups of them at frequencies spanning both tiers
    and the cold range: A stays exact."""
    c_inv = 0xF1DE83E19937733D  # the inverse of the sample's multiplier modulo 2^64
    rng = np.random.default_rng(11)
    n = 1 << 21
    keys = []
    for g in range(40):
        k = int(rng.integers(1, 1 << 62))
        f = max(8, int(20000 * 0.82 ** g))
        for t in range(3):
            keys += [(k + t * c_inv) % (1 << 64)] * f
    keys = np.array(keys, dtype=np.uint64)
    fill = rng.integers(0, 1 << 63, n - keys.size, dtype=np.uint64)
    allk = np.concatenate([keys, fill])[rng.permutation(n)]
    s = (allk >> np.uint64(32)).astype(np.uint32)
    d = (allk & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctx = ns.Context(0, path="sort", sort_split="on")
    info = check(ctx, s, d)
    assert info["hot_keys"] > 0
    ctx.close()


def test_column_split_heavy_destinations():
    """The column side's hot-destination split: a few destinations with
    fan-in in the hundreds of thousands (one of them 0xFFFFFFFF, which marks
    a free slot of the destination table and is never hot), under a skewed
    window.  Every column quantity, and A, equal the oracle's."""
    rng = np.random.default_rng(17)
    n = 1 << 22
    s, d = W.zipf_window(n, 1.2, 1 << 18, 29)
    s, d = s.copy(), d.copy()
    heavy = np.array([0xFFFFFFFF, 0x0A000001, 0xC0A80001, 0x00000000], np.uint32)
    for j, h in enumerate(heavy):
        sl = slice(j, n, 7)  # one packet in seven per heavy destination, from random sources
        d[sl] = h
        s[sl] = rng.integers(0, 1 << 32, s[sl].size, dtype=np.uint64).astype(np.uint32)
    ctx = ns.Context(0, path="sort", sort_split="on")
    check(ctx, s, d)
    ci = ns.column_split_info(ctx)
    assert ci["used"] and ci["hot_destinations"] > 0 and ci["cold_words"] > 0
    ctx.close()


def test_column_split_single_destination():
    """Every link into one destination: its column words all go one way, and
    its fan-in is the number of distinct sources."""
    rng = np.random.default_rng(19)
    n = 1 << 21
    s = rng.integers(0, 1 << 20, n, dtype=np.uint64).astype(np.uint32)
    d = np.full(n, 0x7F000001, np.uint32)
    ctx = ns.Context(0, path="sort", sort_split="on")
    check(ctx, s, d)
    ci = ns.column_split_info(ctx)
    assert ci["used"] and ci["hot_destinations"] == 1 and ci["cold_words"] == 0
    ctx.close()


def test_column_split_off_without_the_link_split():
    ctx = ns.Context(0, path="sort", sort_split="off")
    s, d = W.zipf_window(1 << 20, 1.2, 1 << 16, 3)
    check(ctx, s, d)
    assert not ns.column_split_info(ctx)["used"]
    ctx.close()
