"""Host logic of bench.py that the reported fractions rest on: the sort
path's minimal-byte model against its closed forms (per packet, per link,
per node, per cold key and column word), the digit-pass count, and the
parsing of committed ncu summaries keyed by kernel sources."""
from __future__ import annotations

import os

import pytest

import bench


def test_plain_sort_bytes_closed_form():
    # histogram 8N, eight passes 128N, link runs 8N + 16U, link counts 16U,
    # rows 24U + 32S, column histogram/passes/runs 80U + 32D
    N, U, S, D = 1000, 700, 90, 80
    assert bench.sort_path_bytes(N, U, S, D, {}) == 144 * N + 136 * U + 32 * (S + D)


def test_split_sort_bytes_closed_form():
    N, U, S, D, C, H, Wc = 10_000, 5_000, 900, 800, 3_000, 40, 1_500
    info = {"cold_packets": C, "hot_keys": H, "cold_words": Wc}
    UC = U - H
    want = 8 * N + 152 * C + 32 * UC + 48 * U + 88 * Wc + 32 * (S + D)
    assert bench.sort_path_bytes(N, U, S, D, info) == want


def test_digit_passes_scale_the_pass_bytes():
    N, U, S, D = 1 << 20, 1 << 19, 1 << 10, 1 << 10
    # one pass fewer saves 16 bytes per sorted key
    assert bench.sort_path_bytes(N, U, S, D, {}, 8) - bench.sort_path_bytes(N, U, S, D, {}, 7) == 16 * N
    info = {"cold_packets": N // 3, "hot_keys": 7}
    assert (bench.sort_path_bytes(N, U, S, D, info, 8) - bench.sort_path_bytes(N, U, S, D, info, 7)
            == 16 * (N // 3))


def test_keyed_profile_traffic():
    names = ["ns_hash.cu", "ns_batch.cu", "ns_common.cuh"]
    prof = "k_batch_insert.batched_1024_windows.md"
    path = os.path.join(bench.ROOT, "profiles", prof)
    if not os.path.exists(path):
        pytest.skip("no committed summary")
    text = open(path).read()
    key = "4096,16,0.7,1"
    line = next(l for l in text.splitlines() if l.startswith(f"traffic_per_packet[{key}]:"))
    want = float(line.split(":", 1)[1])
    sha = next(l for l in text.splitlines() if l.startswith("source_sha256:")).split(":", 1)[1].strip()
    got = bench.profile_traffic_keyed(prof, names, key)
    if sha == bench.sources_sha(names):
        assert got == want
    else:
        assert got is None  # taken on other sources: not reported
    assert bench.profile_traffic_keyed(prof, ["ns_sort.cu"], key) is None
    assert bench.profile_traffic_keyed("no_such_profile.md", names, key) is None
