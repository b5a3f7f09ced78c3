"""Seeded randomized parity: windows of random sizes (0 to several tiles
plus ragged tails), address spaces from 2 addresses to the full 32 bits,
skew from uniform to heavy Zipf, both paths and all three hash-table
configurations, and random window sequences through build + accumulate and
the fused ingest -- every result bit-exact against the CPU oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2509_03653_b300 as ns
from gpu_util import assert_matrix_equal, to_dev

pytestmark = pytest.mark.gpu

CONFIGS = {
    "hash": dict(path="hash"),
    "hash_cache_on": dict(path="hash", cta_cache="on"),
    "hash_dense": dict(path="hash", hash_load=0.9, cta_cache="off"),
    "sort": dict(path="sort"),
    "sort_pairs": dict(path="sort", column_sort="pairs"),
}


def random_window(rng, n):
    kind = rng.integers(0, 4)
    seed = int(rng.integers(1, 1 << 40))
    if kind == 0:  # tiny address space: heavy collisions
        bits = int(rng.integers(1, 6))
        s, d = gen.uniform_pairs(n, bits, seed)
    elif kind == 1:  # Zipf over a random number of ranks
        K = int(2 ** rng.integers(2, 22))
        sexp = float(rng.uniform(0.6, 1.6))
        key = gen.bijection_key(seed)
        s = gen.zipf_addresses(n, sexp, K, seed, 1, key)
        d = gen.zipf_addresses(n, sexp, K, seed, 2, key)
    elif kind == 2:  # RMAT
        s, d = gen.rmat_pairs(n, seed, gen.bijection_key(seed))
    else:  # full 32-bit uniform, with the extreme addresses mixed in
        s, d = gen.uniform_pairs(n, 32, seed)
        if n:
            m = rng.integers(0, n, max(1, n // 50))
            s[m[::2]] = 0xFFFFFFFF
            d[m[1::2]] = 0
    return s.astype(np.uint32), d.astype(np.uint32)


def random_size(rng):
    return int(rng.choice([0, 1, 31, 4095, 4096, 4097, 8191, 8192, 8193,
                           int(rng.integers(2, 40000)), int(rng.integers(40000, 300000))]))


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("seed", [1, 2])
def test_random_windows(name, seed):
    rng = np.random.default_rng(1000 * seed + len(name))
    ctx = ns.Context(0, **CONFIGS[name])
    m = ns.Matrix(ctx)
    for _ in range(6):
        s, d = random_window(rng, random_size(rng))
        ns.window_build(ctx, to_dev(s), to_dev(d), m)
        k, c = oracle.build_matrix(s, d)
        assert ns.network_stats(ctx, m) == oracle.stats(k, c)
        assert_matrix_equal(m, k, c)


@pytest.mark.parametrize("name", ["hash", "sort", "hash_dense"])
def test_random_window_sequences(name):
    rng = np.random.default_rng(77 + len(name))
    ctx = ns.Context(0, **CONFIGS[name])
    acc_b, acc_i, at = ns.Matrix(ctx), ns.Matrix(ctx), ns.Matrix(ctx)
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    want = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for w in range(8):
        s, d = random_window(rng, random_size(rng))
        ns.window_build(ctx, to_dev(s), to_dev(d), at)
        ns.accumulate(ctx, acc_b, at)
        ns.window_ingest_stats(ctx, acc_i, to_dev(s), to_dev(d), out)
        want = oracle.accumulate(want, oracle.build_matrix(s, d))
        ref = oracle.stats(*want)
        assert ns.network_stats(ctx, acc_b) == ref, w
        torch.cuda.synchronize()
        assert {f: int(x) for f, x in zip(oracle.FIELDS, out.cpu().numpy().view(np.uint64)[:9])} == ref, w
    assert_matrix_equal(acc_b, *want)
    assert_matrix_equal(acc_i, *want)
