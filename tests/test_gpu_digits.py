"""The sort path's two digit plans against the oracle: eight passes of 8-bit
digits, and the wide plan (a 10-bit first pass, then six 9-bit passes).  A's
sorted nonzero list and the nine quantities, element by element, for every
plan x digit-pass tile x hot-key split, on skewed and uniform windows; sizes
below, at and just past one tile, several tiles with a ragged tail, and the
empty window; keys that differ only at the wide plan's digit boundaries; the
path tuner's record of the plan and ns_sort_resolve's report of it."""
from __future__ import annotations

import json

import numpy as np
import pytest

import gen
import gen.workloads as W
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import export_np, to_dev

pytestmark = pytest.mark.gpu


def check(ctx, s, d):
    m = ns.Matrix(ctx)
    ns.window_build(ctx, to_dev(s), to_dev(d), m)
    got = ns.network_stats(ctx, m)
    wk, wc = oracle.build_matrix(s, d)
    assert got == oracle.stats(wk, wc)
    k, c = export_np(m)
    assert k.size == wk.size
    np.testing.assert_array_equal(k, wk)
    np.testing.assert_array_equal(c, wc)
    m.free()


@pytest.mark.parametrize("digits", ["8", "wide"])
@pytest.mark.parametrize("tile", ["512x16", "512x12", "256x16"])
@pytest.mark.parametrize("split", ["on", "off"])
def test_every_plan_and_tile_matches_oracle(digits, tile, split):
    ctx = ns.Context(0, path="sort", sort_split=split, sort_tile=tile, sort_digits=digits)
    assert ns.sort_resolve(ctx, 1 << 20) == {"split": split == "on", "tile": tile, "digits": digits}
    s, d = W.zipf_window((1 << 20) + 77, 1.2, 1 << 16, 31)
    check(ctx, s, d)
    s, d = gen.uniform_pairs(300007, 32, 12)
    check(ctx, s, d)
    ctx.close()


@pytest.mark.parametrize("n", [0, 1, 100, 4095, 4096, 6144, 8191, 8192, 8193, 5 * 8192 + 1, 123457])
def test_wide_plan_small_and_ragged_sizes(n):
    """Fewer keys than one tile, exactly one tile of each shape, one key past
    it, and several tiles with a ragged tail (no split below 2^16)."""
    for tile in ("512x16", "256x16"):
        ctx = ns.Context(0, path="sort", sort_tile=tile, sort_digits="wide")
        s, d = gen.uniform_pairs(n, 20, 40 + n) if n else (np.zeros(0, np.uint32), np.zeros(0, np.uint32))
        check(ctx, s, d)
        ctx.close()


@pytest.mark.parametrize("split", ["on", "off"])
def test_wide_plan_digit_boundaries(split):
    """Keys that differ only in the bits on either side of each of the wide
    plan's digit boundaries (9|10, 18|19, 27|28, 36|37, 45|46, 54|55) and in
    bit 63, with the extreme keys 0 and 2^64 - 1, repeated unevenly."""
    rng = np.random.default_rng(5)
    base = np.uint64(rng.integers(0, 1 << 62, dtype=np.uint64))
    bits = [0, 9, 10, 18, 19, 27, 28, 31, 32, 36, 37, 45, 46, 54, 55, 62, 63]
    keys = [np.uint64(0), np.uint64(0xFFFFFFFFFFFFFFFF)]
    for mask in range(1 << 6):
        k = base
        for j, b in enumerate(bits[:6]):
            if (mask >> j) & 1:
                k ^= np.uint64(1) << np.uint64(b)
        keys.append(k)
    for b in bits:
        keys.append(base ^ (np.uint64(1) << np.uint64(b)))
        keys.append(np.uint64(1) << np.uint64(b))
    keys = np.array(keys, dtype=np.uint64)
    n = (1 << 17) + 3
    pick = rng.zipf(1.3, n) % keys.size
    k = keys[pick]
    s = (k >> np.uint64(32)).astype(np.uint32)
    d = (k & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctx = ns.Context(0, path="sort", sort_split=split, sort_digits="wide")
    check(ctx, s, d)
    ctx.close()


def test_path_tune_records_digit_plan(tmp_path):
    cache = str(tmp_path / "tuner.json")
    ctx = ns.Context(0, tuner_cache=cache)
    s, d = W.zipf_window(1 << 22, 1.2, 1 << 20, 3)
    ns.path_tune(ctx, to_dev(s), to_dev(d))
    rec = next(iter(json.load(open(cache)).values()))
    assert rec["sort_digits"] in (0, 1)
    assert rec["sort_digits8_ms"] > 0 and rec["sort_wide_ms"] > 0
    want = "wide" if rec["sort_digits"] == 1 else "8"
    assert ns.sort_resolve(ctx, 1 << 22)["digits"] == want
    # a context on the same cache takes the recorded plan, and still builds exactly
    ctx2 = ns.Context(0, path="sort", tuner_cache=cache)
    assert ns.sort_resolve(ctx2, (1 << 22) + 5)["digits"] == want
    check(ctx2, s, d)
    # a forced plan wins over the record
    other = "8" if want == "wide" else "wide"
    ctx3 = ns.Context(0, path="sort", tuner_cache=cache, sort_digits=other)
    assert ns.sort_resolve(ctx3, 1 << 22)["digits"] == other
    ctx.close()
    ctx2.close()
    ctx3.close()


@pytest.mark.parametrize("split", ["on", "off"])
def test_wide_plan_many_tiles_per_cta(split):
    """Windows with far more tiles than resident CTAs, so that every CTA of a
    digit pass takes many tiles and every CTA of the histogram counts many
    rounds between flushes: a Zipf window with a ragged tail, and one in
    which a single link takes half of the packets (every count of one digit
    grows in every lane)."""
    n = (1 << 24) + 123
    ctx = ns.Context(0, path="sort", sort_split=split, sort_digits="wide")
    s, d = W.zipf_window(n, 1.2, 1 << 20, 91)
    check(ctx, s, d)
    s = s.copy()
    d = d.copy()
    s[::2] = 0x01020304
    d[::2] = 0x0A0B0C0D
    check(ctx, s, d)
    ctx.close()
