"""Synthetic workloads standing in for the challenge's packet capture.

The paper measures on one public graph of 2^30 packets (section "Graph
Challenge Setup", paragraph "Inputs") whose GraphBLAS release holds 128 x 64
matrices (section "Implementation", paragraph "GraphBLAS format"), i.e. 2^17
packets per matrix; addresses are anonymized by a random permutation (section
"Implementation", paragraph "IP Address Anonymization").  That dataset is not
available here, so every workload below is drawn by :mod:`gen` from a fixed
seed with the same shapes: uint32 src/dst columns, windows of 2^17 packets,
skewed (Zipf or RMAT) address popularity, addresses relabelled by a seeded
32-bit bijection.

Seeds: workload c (1..5) uses seed 0x4E530000 + c.
"""
from __future__ import annotations

import numpy as np

import gen

SEED_BASE = 0x4E530000

# Single window: 2^17 packets, src and dst independently Zipf(1.1) over 2^14.
W1_N = 1 << 17
W1_S = 1.1
W1_K = 1 << 14

# Accumulated stream: 512 windows of 2^17 RMAT scale-32 packets, 10% uniform.
W2_WINDOWS = 512
W2_WINDOW = 1 << 17
W2_N = W2_WINDOWS * W2_WINDOW

# Large one-shot build: 2^30 packets, Zipf(1.2) over 2^24 addresses.
W3_N = 1 << 30
W3_S = 1.2
W3_K = 1 << 24

# Batched: 8192 windows, sizes log-uniform in [2^10, 2^20], s ~ U[0.8, 1.4],
# K = 2^20.  Exponents are rounded to 0.01 (a draw, not a method parameter).
W4_WINDOWS = 8192
W4_K = 1 << 20

# Streaming serving: sizes log-uniform in [2^12, 2^22], RMAT pairs.
W5_LO, W5_HI = 12.0, 22.0


def seed_of(c: int) -> int:
    return SEED_BASE + c


def zipf_window(n: int, s: float, K: int, seed: int, src=None, dst=None):
    """One window whose src and dst are independent Zipf(s) draws over K."""
    key = gen.bijection_key(seed)
    src = gen.zipf_addresses(n, s, K, seed, 100, key, out=src)
    dst = gen.zipf_addresses(n, s, K, seed, 101, key, out=dst)
    return src, dst


def single_window(n: int = W1_N):
    """Workload 1: one window of n packets, Zipf(1.1) over 2^14 addresses."""
    return zipf_window(n, W1_S, W1_K, seed_of(1))


def rmat_stream(n: int = W2_N, i0: int = 0, src=None, dst=None, seed: int | None = None):
    """Workload 2 packets i0..i0+n-1: RMAT scale 32 (0.57, 0.19, 0.19, 0.05)
    with 10% uniform background pairs."""
    seed = seed_of(2) if seed is None else seed
    return gen.rmat_pairs(n, seed, gen.bijection_key(seed), i0=i0, src=src, dst=dst)


def large_build(n: int = W3_N, src=None, dst=None):
    """Workload 3: n packets, Zipf(1.2) over 2^24 addresses."""
    return zipf_window(n, W3_S, W3_K, seed_of(3), src=src, dst=dst)


def batched_plan(k: int = W4_WINDOWS, lo: float = 10.0, hi: float = 20.0):
    """Workload 4 window sizes and per-window Zipf exponents."""
    seed = seed_of(4)
    sizes = gen.loguniform_sizes(k, lo, hi, seed, 200)
    s = np.round(gen.uniform_doubles(k, 0.8, 1.4, seed, 201), 2)
    return sizes, s


def batched_window(w: int, n: int, s: float, K: int = W4_K, src=None, dst=None):
    """Window w of workload 4: its own Zipf draws (own seed), one anonymizing
    bijection shared by all windows."""
    seed = gen.splitmix64(seed_of(4) * 0x10001 + w)
    key = gen.bijection_key(seed_of(4))
    src = gen.zipf_addresses(n, s, K, seed, 100, key, out=src)
    dst = gen.zipf_addresses(n, s, K, seed, 101, key, out=dst)
    return src, dst


def serving_plan(k: int, rate: float):
    """Workload 5 window sizes (log-uniform in [2^12, 2^22]) and Poisson
    arrival times (seconds) at `rate` windows per second."""
    seed = seed_of(5)
    sizes = gen.loguniform_sizes(k, W5_LO, W5_HI, seed, 300)
    arrivals = gen.poisson_arrivals(k, rate, seed, 301)
    return sizes, arrivals


def serving_window(w: int, n: int, src=None, dst=None):
    seed = gen.splitmix64(seed_of(5) * 0x10001 + w)
    return gen.rmat_pairs(n, seed, gen.bijection_key(seed_of(5)), src=src, dst=dst)
