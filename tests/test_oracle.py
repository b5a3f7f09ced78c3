"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:
  * a hand-worked example (tests/golden/worked_example.txt, from the Table 2
    definitions),
  * dense brute force over a 2^8-address space: the matrix A is built as a
    dense 256 x 256 array and every quantity is evaluated straight from its
    Table 2 matrix-notation formula (sums, |.|_0 and max over rows/columns),
  * numpy's np.unique as an independent library routine for A's nonzeros,
  * closed forms (identical packets, a permutation, a complete bipartite
    block, a star, the empty stream),
  * invariants (row total = column total = packets, U <= N, fan-out <= D,
    fan-in <= S, concatenated windows = summed matrices, packet-order and
    address-relabelling invariance, src/dst exchange swaps the quantities,
    monotone running statistics),
  * per-source / per-destination vectors and the distinct addresses against
    the dense model's row and column sums and counts,
  * address anonymization: a hand-worked fixture
    (tests/golden/anonymize_example.txt), bijectivity, invariance of the nine
    quantities, and the order-preserving special case,
  * planted mistakes: variants of the oracle source with a dropped term, a
    transposed operand or a wrong index must each fail one of the pins.
"""
from __future__ import annotations

import os
import subprocess
import tempfile

import numpy as np
import pytest

import gen
import gen.workloads as W
import oracle
from golden_io import read_anonymize_example, read_worked_example

F = oracle.FIELDS


def tup(d):
    return tuple(d[f] for f in F)


# ---------------------------------------------------------------- dense model

def widen8(a8):
    """Order-preserving injection of 8-bit addresses into 32 bits (0 -> 0,
    255 -> 0xFFFFFFFF), so the extreme keys 0 and 2^64-1 occur."""
    return (a8.astype(np.uint32) * np.uint32(0x01010101)).astype(np.uint32)


def dense_matrix(s8, d8):
    M = np.zeros((256, 256), dtype=np.uint64)
    np.add.at(M, (s8.astype(np.int64), d8.astype(np.int64)), np.uint64(1))
    return M


def dense_stats(M):
    """Table 2, matrix notation, evaluated on a dense array."""
    nz = (M > 0).astype(np.uint64)
    row = M.sum(axis=1)          # A 1
    col = M.sum(axis=0)          # 1^T A
    rdeg = nz.sum(axis=1)        # |A|_0 1
    cdeg = nz.sum(axis=0)        # 1^T |A|_0
    return (int(M.sum()), int(nz.sum()), int((row > 0).sum()), int((col > 0).sum()),
            int(row.max()), int(rdeg.max()), int(col.max()), int(cdeg.max()), int(M.max()))


def dense_nonzeros(M):
    i, j = np.nonzero(M)  # row-major, i.e. ascending (src, dst)
    keys = (widen8(i.astype(np.uint32)).astype(np.uint64) << np.uint64(32)) | \
        widen8(j.astype(np.uint32)).astype(np.uint64)
    return keys, M[i, j].astype(np.uint64)


def skewed_pairs(n, seed):
    """src skewed (Zipf ranks), dst uniform, both 8-bit: asymmetric on purpose
    so that a src/dst mix-up changes the answer."""
    s8 = (gen.zipf_ranks(n, 1.3, 256, seed, 7) & 0xFF).astype(np.uint32) if n else \
        np.zeros(0, np.uint32)
    _, d8 = gen.uniform_pairs(n, 8, seed)
    return s8, d8


# ------------------------------------------------------------------ the pins

def check_golden(L):
    wins, (gk, gc), want = read_worked_example()
    acc = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for t, (s, d) in enumerate(wins):
        acc = oracle.accumulate(acc, oracle.build_matrix(s, d, L), L)
        assert tup(oracle.stats(*acc, L)) == want[t]
    np.testing.assert_array_equal(acc[0], gk)
    np.testing.assert_array_equal(acc[1], gc)


def check_bruteforce(L, n, seed):
    s8, d8 = skewed_pairs(n, seed)
    M = dense_matrix(s8, d8)
    k, c = oracle.build_matrix(widen8(s8), widen8(d8), L)
    dk, dc = dense_nonzeros(M)
    np.testing.assert_array_equal(k, dk)
    np.testing.assert_array_equal(c, dc)
    if n:
        assert tup(oracle.stats(k, c, L)) == dense_stats(M)
    else:
        assert tup(oracle.stats(k, c, L)) == (0,) * 9


def check_windows_bruteforce(L, sizes, seed):
    M = np.zeros((256, 256), dtype=np.uint64)
    acc = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    for w, n in enumerate(sizes):
        s8, d8 = skewed_pairs(n, seed + 1000 * w)
        M += dense_matrix(s8, d8)
        acc = oracle.accumulate(acc, oracle.build_matrix(widen8(s8), widen8(d8), L), L)
        dk, dc = dense_nonzeros(M)
        np.testing.assert_array_equal(acc[0], dk)
        np.testing.assert_array_equal(acc[1], dc)
        if M.sum():
            assert tup(oracle.stats(*acc, L)) == dense_stats(M)


def check_swap(L, seed):
    s, d = skewed_pairs(3000, seed)
    a = oracle.stats_of_packets(widen8(s), widen8(d), L)
    b = oracle.stats_of_packets(widen8(d), widen8(s), L)
    assert (a["unique_sources"], a["max_src_packets"], a["max_src_fanout"]) == \
        (b["unique_destinations"], b["max_dst_packets"], b["max_dst_fanin"])
    assert (a["unique_destinations"], a["max_dst_packets"], a["max_dst_fanin"]) == \
        (b["unique_sources"], b["max_src_packets"], b["max_src_fanout"])


def check_vectors_bruteforce(L, n, seed):
    """Per-source and per-destination vectors and the distinct addresses,
    against the dense matrix: row sums and row nonzero counts (A 1,
    |A|_0 1), column sums and counts (1^T A, 1^T |A|_0), and the union of
    live rows and live columns."""
    s8, d8 = skewed_pairs(n, seed)
    M = dense_matrix(s8, d8)
    k, c = oracle.build_matrix(widen8(s8), widen8(d8), L)
    live_r = np.nonzero(M.sum(axis=1))[0]
    live_c = np.nonzero(M.sum(axis=0))[0]
    src, pk, fo = oracle.rows(k, c, L)
    np.testing.assert_array_equal(src, widen8(live_r.astype(np.uint32)))
    np.testing.assert_array_equal(pk, M.sum(axis=1)[live_r])
    np.testing.assert_array_equal(fo, (M > 0).sum(axis=1)[live_r].astype(np.uint64))
    dst, cp, fi = oracle.cols(k, c, L)
    np.testing.assert_array_equal(dst, widen8(live_c.astype(np.uint32)))
    np.testing.assert_array_equal(cp, M.sum(axis=0)[live_c])
    np.testing.assert_array_equal(fi, (M > 0).sum(axis=0)[live_c].astype(np.uint64))
    both = np.union1d(live_r, live_c).astype(np.uint32)
    np.testing.assert_array_equal(oracle.unique_addresses(k, L), widen8(both))


def check_anonymize(L, seed):
    """The hand-worked fixture; then, on a skewed stream: the labels are a
    bijection of the distinct addresses onto 0..N-1, equal addresses get
    equal labels, the nine quantities are unchanged, and increasing keys
    give the order-preserving relabelling (labels = ranks)."""
    s, d, r, want_s, want_d = read_anonymize_example()
    got_s, got_d, nu = oracle.anonymize(s, d, r, L)
    np.testing.assert_array_equal(got_s, want_s)
    np.testing.assert_array_equal(got_d, want_d)
    assert nu == 4
    s8, d8 = skewed_pairs(20000, seed)
    src, dst = widen8(s8), widen8(d8)
    u = np.union1d(src, dst)
    rnd = gen.random_u64(u.size + 5, seed, 3)
    a_s, a_d, nu = oracle.anonymize(src, dst, rnd, L)
    assert nu == u.size
    lab = np.full(u.size, -1, np.int64)
    for addr, out in ((src, a_s), (dst, a_d)):
        idx = np.searchsorted(u, addr)
        assert np.all((lab[idx] == -1) | (lab[idx] == out))  # one label per address
        lab[idx] = out
    assert np.array_equal(np.sort(lab), np.arange(u.size))  # a permutation of 0..N-1
    assert tup(oracle.stats_of_packets(a_s, a_d, L)) == tup(oracle.stats_of_packets(src, dst, L))
    ranks_s, ranks_d, _ = oracle.anonymize(src, dst, np.arange(u.size, dtype=np.uint64), L)
    np.testing.assert_array_equal(ranks_s, np.searchsorted(u, src).astype(np.uint32))
    np.testing.assert_array_equal(ranks_d, np.searchsorted(u, dst).astype(np.uint32))


def check_parallel(L, seed):
    """The all-cores variants against the dense model (nonzero list and the
    nine quantities, heavy collisions, keys 0 and 2^64-1) with more threads
    than packets and with ragged chunks, and against the single-thread
    oracle on a skewed stream."""
    for n, threads in ((0, 4), (1, 4), (5, 16), (4099, 3), (40000, 7)):
        s8, d8 = skewed_pairs(n, seed + n)
        M = dense_matrix(s8, d8)
        k, c = oracle.build_matrix_parallel(widen8(s8), widen8(d8), threads, L)
        dk, dc = dense_nonzeros(M)
        np.testing.assert_array_equal(k, dk)
        np.testing.assert_array_equal(c, dc)
        want = dense_stats(M) if n else (0,) * 9
        assert tup(oracle.stats_parallel(k, c, threads, L)) == want
    s, d = W.large_build(1 << 16)
    k1, c1 = oracle.build_matrix(s, d, L)
    for threads in (2, 5, 0):
        k2, c2 = oracle.build_matrix_parallel(s, d, threads, L)
        np.testing.assert_array_equal(k2, k1)
        np.testing.assert_array_equal(c2, c1)
        assert oracle.stats_parallel(k1, c1, threads, L) == oracle.stats(k1, c1, L)


def all_pins(L):
    check_golden(L)
    check_parallel(L, 51)
    for n, seed in ((1, 1), (2, 2), (255, 3), (4099, 4), (40000, 5)):
        check_bruteforce(L, n, seed)
    check_windows_bruteforce(L, (700, 0, 1, 3000), 11)
    check_swap(L, 21)
    for n, seed in ((1, 31), (3000, 32), (30000, 33)):
        check_vectors_bruteforce(L, n, seed)
    check_anonymize(L, 41)


def test_golden_worked_example():
    check_golden(oracle.lib())


@pytest.mark.parametrize("n", [0, 1, 2, 31, 256, 4099, 65536, 200003])
@pytest.mark.parametrize("seed", [1, 2])
def test_bruteforce_dense(n, seed):
    check_bruteforce(oracle.lib(), n, seed)


def test_bruteforce_windows():
    check_windows_bruteforce(oracle.lib(), (5000, 1, 0, 777, 20000, 3), 42)


def test_numpy_unique_crosscheck():
    s, d = W.single_window(1 << 16)
    k, c = oracle.build_matrix(s, d)
    keys = (s.astype(np.uint64) << np.uint64(32)) | d.astype(np.uint64)
    uk, uc = np.unique(keys, return_counts=True)
    np.testing.assert_array_equal(k, uk)
    np.testing.assert_array_equal(c, uc.astype(np.uint64))


def test_rows_vector_bruteforce():
    s8, d8 = skewed_pairs(30000, 9)
    M = dense_matrix(s8, d8)
    k, c = oracle.build_matrix(widen8(s8), widen8(d8))
    src, pk, fo = oracle.rows(k, c)
    live = np.nonzero(M.sum(axis=1))[0]
    np.testing.assert_array_equal(src, widen8(live.astype(np.uint32)))
    np.testing.assert_array_equal(pk, M.sum(axis=1)[live])
    np.testing.assert_array_equal(fo, (M > 0).sum(axis=1)[live].astype(np.uint64))


# ------------------------------------------------------------- closed forms

def test_closed_all_identical():
    n = 1000
    s = np.full(n, 7, np.uint32)
    d = np.full(n, 9, np.uint32)
    assert tup(oracle.stats_of_packets(s, d)) == (n, 1, 1, 1, n, 1, n, 1, n)


def test_closed_permutation():
    n = 4096
    s = np.arange(n, dtype=np.uint32) * np.uint32(977)
    d = gen.feistel(np.arange(n, dtype=np.uint32), 5)
    assert tup(oracle.stats_of_packets(s, d)) == (n, n, n, n, 1, 1, 1, 1, 1)


def test_closed_complete_bipartite():
    k = 37
    s = np.repeat(np.arange(k, dtype=np.uint32) + 100, k)
    d = np.tile(np.arange(k, dtype=np.uint32) + 5000, k)
    order = np.argsort(gen.feistel(np.arange(k * k, dtype=np.uint32), 3))
    assert tup(oracle.stats_of_packets(s[order], d[order])) == (k * k, k * k, k, k, k, k, k, k, 1)


def test_closed_star():
    n = 5000
    s = np.full(n, 0xFFFFFFFF, np.uint32)
    d = np.arange(n, dtype=np.uint32)
    assert tup(oracle.stats_of_packets(s, d)) == (n, n, 1, n, n, n, 1, 1, 1)


def test_closed_empty():
    z = np.zeros(0, np.uint32)
    assert tup(oracle.stats_of_packets(z, z)) == (0,) * 9
    k, c = oracle.build_matrix(z, z)
    assert k.size == 0 and c.size == 0


# --------------------------------------------------------------- invariants

def _invariants(st, n):
    assert st["valid_packets"] == n
    assert st["unique_links"] <= n
    assert st["max_src_fanout"] <= st["unique_destinations"]
    assert st["max_dst_fanin"] <= st["unique_sources"]
    assert st["max_src_packets"] >= st["max_src_fanout"]
    assert st["max_dst_packets"] >= st["max_dst_fanin"]
    assert st["unique_sources"] <= st["unique_links"]
    assert st["unique_destinations"] <= st["unique_links"]
    assert st["max_link_packets"] <= min(st["max_src_packets"], st["max_dst_packets"])


@pytest.mark.parametrize("kind", ["zipf", "rmat"])
def test_invariants_and_totals(kind):
    n = 1 << 16
    s, d = W.single_window(n) if kind == "zipf" else W.rmat_stream(n)
    k, c = oracle.build_matrix(s, d)
    st = oracle.stats(k, c)
    _invariants(st, n)
    # row total = column total = N
    _, pk, _ = oracle.rows(k, c)
    assert int(pk.sum()) == n == int(c.sum())
    kt, ct = oracle.build_matrix(d, s)
    _, pkt, _ = oracle.rows(kt, ct)
    assert int(pkt.sum()) == n


def test_concat_equals_sum_and_monotone():
    n = 1 << 14
    s, d = W.rmat_stream(6 * n)
    acc = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    prev = (0,) * 9
    for w in range(6):
        acc = oracle.accumulate(acc, oracle.build_matrix(s[w * n:(w + 1) * n], d[w * n:(w + 1) * n]))
        cur = tup(oracle.stats(*acc))
        assert all(a >= b for a, b in zip(cur, prev))
        prev = cur
    k, c = oracle.build_matrix(s, d)
    np.testing.assert_array_equal(acc[0], k)
    np.testing.assert_array_equal(acc[1], c)


def test_packet_order_invariance():
    s, d = W.single_window(1 << 15)
    perm = np.argsort(gen.feistel(np.arange(s.size, dtype=np.uint32), 77))
    a = oracle.build_matrix(s, d)
    b = oracle.build_matrix(s[perm], d[perm])
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_relabel_invariance():
    s, d = W.single_window(1 << 15)
    key = 0xABCDEF
    a = oracle.build_matrix(s, d)
    b = oracle.build_matrix(gen.feistel(s, key), gen.feistel(d, key))
    assert oracle.stats(*a) == oracle.stats(*b)
    # nonzeros map under the bijection: same multiset of counts, relabelled keys
    ks = gen.feistel((a[0] >> np.uint64(32)).astype(np.uint32), key).astype(np.uint64)
    kd = gen.feistel((a[0] & np.uint64(0xFFFFFFFF)).astype(np.uint32), key).astype(np.uint64)
    mk = (ks << np.uint64(32)) | kd
    o = np.argsort(mk)
    np.testing.assert_array_equal(mk[o], b[0])
    np.testing.assert_array_equal(a[1][o], b[1])


def test_swap_exchanges_quantities():
    check_swap(oracle.lib(), 5)


def test_digest_order_independent():
    k, c = oracle.build_matrix(*W.single_window(1 << 12))
    p = np.argsort(gen.feistel(np.arange(k.size, dtype=np.uint32), 1))
    assert oracle.digest(k, c) == oracle.digest(k[p], c[p])
    c2 = c.copy()
    c2[0] += np.uint64(1)
    assert oracle.digest(k, c) != oracle.digest(k, c2)


# ---------------------------------------------------------- planted mistakes

MUTANTS = {
    # a dropped term: row packets count entries instead of packets
    "row_packets_counts_entries": ("packets += counts[u];", "packets += 1;"),
    # a transposed operand: columns grouped by the source half of the key
    "columns_by_source": ("(uint32_t)(keys[v] & 0xFFFFFFFFu)", "(uint32_t)(keys[v] >> 32)"),
    # fan-out accumulating packets instead of entries
    "fanout_sums_packets": ("fanout += 1;", "fanout += counts[u];"),
    # accumulate drops the second operand's count on equal keys
    "merge_drops_term": ("counts_out[u] = ca[i] + cb[j];", "counts_out[u] = ca[i];"),
    # key packed with src and dst exchanged
    "key_transposed": ("key[i] = ((uint64_t)src[i] << 32) | (uint64_t)dst[i];",
                       "key[i] = ((uint64_t)dst[i] << 32) | (uint64_t)src[i];"),
    # run length off by one
    "run_length_off_by_one": ("counts_out[u] = j - i;", "counts_out[u] = j - i + (j - i > 1);"),
    # fan-in maximum taken from the wrong running value
    "fanin_wrong_index": ("if (fanin > stats[MAX_DST_FANIN]) stats[MAX_DST_FANIN] = fanin;",
                          "if (fanin > stats[MAX_DST_FANIN]) stats[MAX_DST_FANIN] = packets;"),
    # unique sources counted per entry rather than per run
    "sources_per_entry": ("stats[UNIQUE_SOURCES] += 1;", "stats[UNIQUE_SOURCES] += fanout;"),
    # column fan-in summing packets instead of entries
    "cols_fanin_sums_packets": ("fanin += 1;\n            ++u;", "fanin += col[u].second;\n            ++u;"),
    # distinct addresses taken from the source half only
    "unique_addresses_src_only": ("a.push_back((uint32_t)keys[u]);", "a.push_back((uint32_t)(keys[u] >> 32));"),
    # the inverse permutation applied instead of the permutation
    "anonymize_inverse_permutation": ("label[order[t]] = (uint32_t)t;", "label[t] = (uint32_t)order[t];"),
    # random keys indexed from the end of the array
    "anonymize_wrong_random_index": ("return rnd[a] < rnd[b];", "return rnd[rnd_n - 1 - a] < rnd[rnd_n - 1 - b];"),
    # all-cores build: each chunk loses its last packet
    "parallel_chunk_short": ("oracle_build(src + a, dst + a, b - a,", "oracle_build(src + a, dst + a, b - a - (b > a),"),
    # all-cores build: an odd chunk matrix left out of the sum
    "parallel_drops_odd_chunk": ("if (part.size() & 1) next.back() = std::move(part.back());\n        part.swap(next);\n    }\n    const List&",
                                 "part.swap(next);\n    }\n    const List&"),
    # all-cores columns: merged destinations keep one side's fan-in
    "parallel_cols_merge_drops_entries": ("a[i].entries + b[j].entries", "a[i].entries"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    old, new = MUTANTS[name]
    with open(oracle._SRC) as f:
        text = f.read()
    assert text.count(old) >= 1, name  # the first occurrence is in oracle_stats/_build
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "mutant.cpp")
        with open(src, "w") as f:
            f.write(text.replace(old, new, 1))
        so = os.path.join(tmp, "libmutant.so")
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-pthread", "-shared", "-fPIC", "-o", so, src])
        L = oracle.load(so)
        with pytest.raises(AssertionError):
            all_pins(L)


def test_unmutated_passes_all_pins():
    all_pins(oracle.lib())
