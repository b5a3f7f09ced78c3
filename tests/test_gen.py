"""The seeded input generators (CPU only).

Both the oracle and the CUDA path consume these arrays, so they are pinned
to their published definitions and to the properties the workloads rely on:
SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) restated here in Python, the
counter-based stream built on it, the Feistel relabelling being a bijection
with a working inverse, determinism and slice consistency of the
counter-based draws, and Zipf frequencies against their closed form."""
from __future__ import annotations

import numpy as np
import pytest

import gen
import gen.workloads as W

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64_ref(x: int) -> int:
    """SplitMix64's output step on state x + golden gamma, written out from
    the published algorithm (the state increment is the golden-ratio
    constant; the finaliser is two xor-shift-multiply rounds and a shift)."""
    z = (x + GOLDEN) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_matches_its_definition():
    rng = np.random.default_rng(1)
    xs = [0, 1, GOLDEN, M64, 1 << 40, 0x4E530001] + [int(v) for v in rng.integers(0, 2**63, 200)]
    for x in xs:
        assert gen.splitmix64(x) == splitmix64_ref(x), hex(x)
    # the generator's first outputs from state 0, as commonly published
    assert splitmix64_ref(0) == 0xE220A8397B1DCDAF
    assert splitmix64_ref(GOLDEN) == 0x6E789E6AA1B965F4


def test_random_keys_are_the_counter_based_stream():
    seed, stream, n = 0x4E530003, 7, 4096
    r = gen.random_u64(n, seed, stream)
    for i in (0, 1, 2, 1000, n - 1):
        assert int(r[i]) == splitmix64_ref(seed ^ (stream << 40) ^ i)
    assert np.array_equal(r, gen.random_u64(n, seed, stream))
    assert not np.array_equal(r, gen.random_u64(n, seed + 1, stream))
    assert not np.array_equal(r, gen.random_u64(n, seed, stream + 1))


def test_feistel_is_a_bijection_with_an_inverse():
    key = gen.bijection_key(0x4E530002)
    # injective on every 16-bit-aligned block tried, and on a wide sample
    for base in (0, 0x10000 * 12345, 0xFFFF0000):
        x = np.arange(base, base + 0x10000, dtype=np.uint64).astype(np.uint32)
        y = gen.feistel(x, key)
        assert np.unique(y).size == x.size
    x = np.random.default_rng(2).integers(0, 2**32, 1 << 20, dtype=np.uint64).astype(np.uint32)
    x = np.unique(x)
    assert np.unique(gen.feistel(x, key)).size == x.size
    # the inverse undoes it, including at the extremes
    for v in (0, 1, 0xFFFF, 0x10000, 0x7FFFFFFF, 0xFFFFFFFF, 123456789):
        y = int(gen.feistel(np.array([v], dtype=np.uint32), key)[0])
        assert gen.feistel_inv_scalar(y, key) == v
    # a different key gives a different relabelling
    x = np.arange(1024, dtype=np.uint32)
    assert not np.array_equal(gen.feistel(x, key), gen.feistel(x, key ^ 1))


def test_rmat_stream_is_deterministic_and_slice_consistent():
    key = gen.bijection_key(5)
    s, d = gen.rmat_pairs(1 << 16, 5, key)
    s2, d2 = gen.rmat_pairs(1 << 16, 5, key)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)
    # packet i depends only on (seed, i): a window drawn from offset i0 is
    # the same slice of the whole stream
    a = 12345
    ws, wd = gen.rmat_pairs(1000, 5, key, i0=a)
    assert np.array_equal(ws, s[a:a + 1000]) and np.array_equal(wd, d[a:a + 1000])
    # the stream workload is built the same way
    S, D = W.rmat_stream(1 << 12)
    S2, D2 = W.rmat_stream(1 << 12)
    assert np.array_equal(S, S2) and np.array_equal(D, D2)


@pytest.mark.parametrize("s,K", [(1.1, 1 << 14), (1.2, 1 << 10), (0.8, 1 << 12)])
def test_zipf_frequencies_match_the_closed_form(s, K):
    n = 1 << 20
    r = gen.zipf_ranks(n, s, K, 0x4E530001, 3)  # rank k is returned as k - 1
    assert r.max() <= K - 1
    H = float(np.sum(np.arange(1, K + 1, dtype=np.float64) ** -s))
    counts = np.bincount(r, minlength=K)
    for k in (1, 2, 3, 10, 100):
        p = k ** -s / H
        sigma = np.sqrt(p * (1 - p) / n)
        assert abs(counts[k - 1] / n - p) < 6 * sigma + 1e-6, (k, counts[k - 1] / n, p)
    assert np.array_equal(r, gen.zipf_ranks(n, s, K, 0x4E530001, 3))


def test_window_sizes_and_arrivals():
    sizes = gen.loguniform_sizes(8192, 10.0, 20.0, 9, 1)
    assert sizes.min() >= 2**10 and sizes.max() <= 2**20
    # log2 of the sizes is spread over the whole range
    lg = np.log2(sizes.astype(np.float64))
    assert abs(lg.mean() - 15.0) < 0.1
    t = gen.poisson_arrivals(1 << 16, 1000.0, 9, 2)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps >= 0)
    assert abs(gaps.mean() - 1e-3) < 3e-5  # mean gap 1/rate (about 8 standard errors for 2^16 exponential gaps)
